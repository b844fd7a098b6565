"""Serving loop: admission, concurrency, and the same result alone and in the
mix (through the native server and the C ABI)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2512_02577_gb300 as p
from paper_2512_02577_gb300 import serve
from paper_2512_02577_gb300.inputs import serving_requests

pytestmark = pytest.mark.gpu


def _stream(n_req, seed_shift=0, n_hi=16):
    return serving_requests(n_requests=n_req, rate=400.0, arrival_seed=7 + seed_shift, size_seed=11 + seed_shift,
                            n_lo=8, n_hi=n_hi, k_lo=2, k_hi=5)


def test_each_result_is_the_same_alone_and_in_the_mix():
    reqs = _stream(10)
    mix, summary = serve.run(reqs, precision=p.FP32, max_active=6)
    assert summary["failed"] == 0
    assert all(rec["rel_residual"] <= 1e-8 for rec in mix)
    for rec in mix[:4]:
        alone, _ = serve.run([dict(rec, t_arrival=0.0)], precision=p.FP32, max_active=1)
        a, m = alone[0]["x"], rec["x"]
        rel = float(torch.linalg.norm(a - m) / torch.linalg.norm(a))
        assert rel <= 1e-12, (rec["n"], rec["k"], rel)
        assert alone[0]["iterations"] == rec["iterations"]


def test_results_match_direct_solve():
    reqs = _stream(4, seed_shift=3)
    recs, _ = serve.run(reqs, precision=p.FP64, max_active=4)
    for rec in recs:
        ctx = p.Context(p.make_config(dim=3, n_cells=rec["n"], degree=rec["k"]), device="cuda:0")
        b = serve._rhs(3, rec["n"], rec["k"], rec["rhs_seed"]).cuda()
        x = torch.zeros_like(b)
        info = ctx.solve(b, x)
        assert info.iterations == rec["iterations"]
        assert torch.equal(x.cpu(), rec["x"])
        ctx.close()


def test_admission_by_memory_budget():
    # a budget that holds one context of the largest request at a time: the
    # others wait in the queue, all finish, and contexts are evicted/reused
    reqs = _stream(6, seed_shift=5)
    sizes = [p.bytes_required(p.make_config(dim=3, n_cells=r["n"], degree=r["k"], mg_precision=p.FP32))
             for r in reqs]
    recs, summary = serve.run(reqs, precision=p.FP32, max_active=6, budget=int(max(sizes) * 1.01))
    assert summary["failed"] == 0
    assert summary["used_bytes"] <= max(sizes) * 1.01
    assert all(rec["rel_residual"] <= 1e-8 for rec in recs)


def test_request_larger_than_budget_is_rejected():
    srv = p.Server(memory_budget_bytes=1 << 20, max_active=2)
    cfg = p.make_config(dim=3, n_cells=16, degree=4)
    n = (4 * 16 + 1) ** 3
    b = torch.zeros(n, dtype=torch.float64)
    with pytest.raises(p.PmgError) as e:
        srv.submit(cfg, b, torch.zeros_like(b))
    assert e.value.code == p.PMG_ERR_OOM
    srv.close()


def test_concurrent_requests_overlap():
    # six requests arriving together with six slots are all in flight at once
    reqs = [dict(id=i, t_arrival=0.0, n=16, k=4, rhs_seed=500 + i) for i in range(6)]
    recs, summary = serve.run(reqs, precision=p.FP32, max_active=6)
    assert summary["failed"] == 0
    assert max(r["t_start"] for r in recs) < min(r["t_done"] for r in recs)
    # one slot: strictly one after the other
    recs1, _ = serve.run(reqs, precision=p.FP32, max_active=1)
    order = sorted(recs1, key=lambda r: r["t_start"])
    assert all(a["t_done"] <= b["t_start"] + 1e-6 for a, b in zip(order, order[1:]))


def test_mixed_method_stream_same_alone_and_in_the_mix():
    # requests with different smoothers, local cycles, outer solvers and
    # geometries in one stream: each result equals its solve alone
    from paper_2512_02577_gb300.inputs import vertex_displacements
    disp = vertex_displacements(3, 8, 0.2, 7)
    cfgs = [p.make_config(dim=3, n_cells=8, degree=3, mg_precision=p.FP32),
            p.make_config(dim=3, n_cells=8, degree=3, mg_precision=p.FP32, smoother=p.MULTIPLICATIVE),
            p.make_config(dim=3, n_cells=8, degree=2, mg_precision=p.FP32, local_half=1),
            p.make_config(dim=3, n_cells=8, degree=2, geometry=p.DISTORTED, vertex_disp=disp,
                          mg_precision=p.FP32, local_half=1, smoother=p.MULTIPLICATIVE),
            p.make_config(dim=3, n_cells=4, degree=4, geometry=p.DEFORMED)]
    srv = p.Server(0, 5)
    jobs = []
    for i, cfg in enumerate(cfgs):
        b = serve._rhs(3, cfg.n_cells, cfg.degree, 700 + i)
        x = torch.zeros_like(b).pin_memory()
        jobs.append((cfg, b, x, srv.submit(cfg, b, x)))
    while any(srv.result(j[3])["state"] < 2 for j in jobs):
        srv.poll()
    for cfg, b, x, rid in jobs:
        res = srv.result(rid)
        assert res["state"] == 2 and res["rel_residual"] <= 1e-8
        ctx = p.Context(cfg, device="cuda:0")
        xa = torch.zeros(ctx.num_dofs(), dtype=torch.float64, device="cuda:0")
        info = ctx.solve(b.cuda(), xa)
        assert info.iterations == res["iterations"]
        assert torch.equal(xa.cpu(), x)
        ctx.close()
    srv.close()


def test_reuse_key_separates_amplitude_damping_and_displacements():
    # One slot, so each request finds the previous one's context idle: a
    # context may be reused only when it builds the same operator and
    # preconditioner.  Requests differ only in the deformation amplitude,
    # the damping, or the displacement values (the caller overwrites its
    # displacement array after the first submit); the last repeats the first
    # and reuses its context.
    from paper_2512_02577_gb300.inputs import vertex_displacements
    d, n, k = 3, 4, 3
    disp = vertex_displacements(d, n, 0.2, 21)
    disp_b = vertex_displacements(d, n, 0.2, 22)
    base = dict(dim=d, n_cells=n, degree=k, mg_precision=p.FP32)
    cfgs = [p.make_config(geometry=p.DEFORMED, deform_amp=0.05, **base),
            p.make_config(geometry=p.DEFORMED, deform_amp=0.1, **base),
            p.make_config(**base),
            p.make_config(omega_patch=0.12, **base),
            p.make_config(omega_jacobi=[1.0, 0.6], **base)]
    srv = p.Server(0, 1)
    jobs = []

    def submit(cfg, seed):
        b = serve._rhs(d, n, k, seed)
        x = torch.zeros_like(b).pin_memory()
        jobs.append((b, x, srv.submit(cfg, b, x)))

    for i, cfg in enumerate(cfgs):
        submit(cfg, 900 + i)
    arr = np.array(disp)                               # the caller's buffer
    cfg_a = p.make_config(geometry=p.DISTORTED, vertex_disp=arr, **base)
    cfg_a.vertex_disp = arr.ctypes.data                 # point at the buffer itself, not a copy
    submit(cfg_a, 905)
    arr[:] = disp_b                                     # reused before the request was admitted
    submit(cfg_a, 906)
    submit(cfgs[0], 907)
    while any(srv.result(j[2])["state"] < 2 for j in jobs):
        srv.poll()
    assert srv.stats()["created_contexts"] == 7
    solo_cfgs = cfgs + [p.make_config(geometry=p.DISTORTED, vertex_disp=disp, **base),
                        p.make_config(geometry=p.DISTORTED, vertex_disp=disp_b, **base), cfgs[0]]
    xs = []
    for cfg, (b, x, rid) in zip(solo_cfgs, jobs):
        res = srv.result(rid)
        assert res["state"] == 2 and res["rel_residual"] <= 1e-8
        ctx = p.Context(cfg, device="cuda:0")
        xa = torch.zeros(ctx.num_dofs(), dtype=torch.float64, device="cuda:0")
        info = ctx.solve(b.cuda(), xa)
        assert info.iterations == res["iterations"]
        assert torch.equal(xa.cpu(), x)
        ctx.close()
        srv.release(rid)
        xs.append(x)
    assert srv.result(jobs[0][2])["code"] == p.PMG_ERR_ARG   # released: unknown id
    assert not torch.equal(xs[0], xs[1]) and not torch.equal(xs[2], xs[3]) and not torch.equal(xs[5], xs[6])
    srv.close()


def test_release_refuses_a_running_request():
    srv = p.Server(0, 1)
    cfg = p.make_config(dim=3, n_cells=8, degree=2)
    b = serve._rhs(3, 8, 2, 1)
    x = torch.zeros_like(b).pin_memory()
    rid = srv.submit(cfg, b, x)
    with pytest.raises(p.PmgError) as e:
        srv.release(rid)                                # still queued
    assert e.value.code == p.PMG_ERR_STATE
    while srv.result(rid)["state"] < 2:
        srv.poll()
    srv.release(rid)
    srv.close()
