"""Driver for the native serving loop: replays a request stream (arrival
times, mesh sizes, degrees, N(0,1) right-hand sides) against a Server and
reports latency percentiles and throughput.

Only argument marshalling and wall-clock bookkeeping happen here; admission,
context reuse, the interleaved CG iterations and the kernels run in the
library (csrc/serve.cpp, csrc/pmg.cu).
"""
import time

import numpy as np
import torch

from . import CARTESIAN, FP32, SERVE_FIFO, Server, make_config
from .inputs import interior_mask


def _rhs(dim, n, k, seed):
    """N(0,1) on the free nodes, zero on the boundary, as pinned CPU memory."""
    m = interior_mask(dim, n, k)
    b = torch.zeros(m.size, dtype=torch.float64).pin_memory()
    rng = np.random.default_rng(seed)
    b.numpy()[m] = rng.standard_normal(int(m.sum()))
    return b


def prepare(requests, dim=3):
    """Pinned host right-hand sides (N(0,1), seed rhs_seed) and solution
    buffers for ``requests``; pass the result to run() to reuse them."""
    out = []
    for r in requests:
        b = _rhs(dim, r["n"], r["k"], r["rhs_seed"])
        out.append((b, torch.zeros_like(b).pin_memory()))
    return out


def run(requests, dim=3, precision=FP32, geometry=CARTESIAN, max_active=8, budget=0, rtol=1e-8, maxit=300,
        time_scale=1.0, poll_sleep=0.0, policy=SERVE_FIFO, max_wait_s=2.0, small_work=0.0, buffers=None,
        group_work=0.0, max_group=8, **config):
    """Serve ``requests`` (dicts with t_arrival, n, k, rhs_seed) and return
    per-request records plus summary statistics.  policy / max_wait_s /
    small_work: the server's admission order (pmg_server_set_policy);
    group_work / max_group: grouped launches for requests up to that
    estimated work (pmg_server_set_grouping; 0 = off);
    buffers: prepare(requests) to reuse; config: further make_config
    arguments (e.g. outer_apply) for every request."""
    buffers = prepare(requests, dim) if buffers is None else buffers
    prepared = []
    for r, (b, x) in zip(requests, buffers):
        cfg = make_config(dim=dim, n_cells=r["n"], degree=r["k"], mg_precision=precision, geometry=geometry, **config)
        x.zero_()
        prepared.append((r, cfg, b, x))
    server = Server(budget, max_active, policy=policy, max_wait_s=max_wait_s, small_work=small_work,
                    group_work=group_work, max_group=max_group)
    ids = {}
    pending = list(range(len(prepared)))
    t0 = time.perf_counter()
    done = 0
    while done < len(prepared):
        now = time.perf_counter() - t0
        while pending and prepared[pending[0]][0]["t_arrival"] * time_scale <= now:
            i = pending.pop(0)
            r, cfg, b, x = prepared[i]
            ids[i] = server.submit(cfg, b, x, rtol=rtol, maxit=maxit)
        running, queued = server.poll()
        done = len(ids) - running - queued  # finished (done or failed): neither queued nor running
        if poll_sleep:
            time.sleep(poll_sleep)
    wall = time.perf_counter() - t0
    records = []
    for i, (r, cfg, b, x) in enumerate(prepared):
        res = server.result(ids[i])
        n1 = r["k"] * r["n"] + 1
        records.append(dict(r, dofs=n1 ** dim, latency_s=res["t_done"] - res["t_submit"],
                            queue_s=res["t_start"] - res["t_submit"], t_start=res["t_start"],
                            t_done=res["t_done"], state=res["state"],
                            iterations=res["iterations"], rel_residual=res["rel_residual"], x=x))
        server.release(ids[i])
    stats = server.stats()
    server.close()
    lat = np.array([rec["latency_s"] for rec in records])
    total_dofs = sum(rec["dofs"] for rec in records)
    summary = dict(requests=len(records), p50_ms=float(np.percentile(lat, 50) * 1e3),
                   p99_ms=float(np.percentile(lat, 99) * 1e3), mean_ms=float(lat.mean() * 1e3),
                   makespan_s=wall, dofs_per_s=total_dofs / wall, failed=sum(rec["state"] != 2 for rec in records),
                   max_iterations=max(rec["iterations"] for rec in records), **stats)
    return records, summary
