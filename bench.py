"""Benchmark: 3D Poisson, unit cube, 32^3 hexes, Q4 (2,146,689 DoFs), FP64.

One step = one pass of the whole hot path on the resident problem:
  operator apply (FP64) + one additive vertex-patch sweep with the local
  p-multigrid solver (FP64) + a full PCG solve with the geometric V-cycle
  preconditioner to ||r|| <= 1e-8 ||b|| (FP64 throughout, manufactured RHS).
value = DoFs / step time (whole job, summed over ranks).  L2 is flushed
between timed steps (a 512 MB write outside the timed events).

Also reported: apply and sweep throughput, FP64 and mixed (FP32 V-cycle)
solve times p50/p99, the roofline of the dominant kernel (the patch
smoother, FP64-ALU bound), the CPU oracle on a bounded sample, the
end-to-end number through the host-buffer C-ABI calls, and SM clocks.

--impl reference times the CPU oracle (the reference arm of this build).
Multi-GPU: replicas only (one independent problem per rank, no collective).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "3D unit cube, 32^3 hexes, Q4 (2,146,689 DoFs), FP64: apply + patch sweep + PCG/GMG solve to 1e-8"
METRIC = "DoFs/s of operator apply + patch smoother; solve time to 1e-8 residual, FP32-MG vs FP64; p50/p99"
D, NCELL, K = 3, 32, 4
# Coarsest level of the 32^3 hierarchies: the first mesh of the halving
# sequence with at most 4,096 free DoFs (4^3 cells at k = 4: 3,375), solved
# by the dense coarse inverse.  Coarsening further (to 2^3 and 1 cell) adds
# two levels whose patch launches hold one or a few blocks -- a block's
# latency each, about 0.2 ms in FP64 -- and no work worth the launch.
COARSE_DOFS = 4096
ORACLE_N = 4          # bounded CPU sample: same degree and dimension, 4^3 cells (4,913 DoFs)
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 (measured 1.255 with a project FMA probe)
FP32_PEAK_TFLOPS = 78.5  # measured FP32 FMA (128 lanes x 152 SMs x 2 x ~2.0 GHz)
# DRAM bytes (read + write) of one FP64 patch launch at 32^3 Q4, from one ncu
# capture of that launch (57.12 MB + 54.64 MB); to be re-taken whenever
# patch_cart_kernel changes.
PATCH64_TRAFFIC_BYTES = 111762432


# ----------------------------------------------------------------- flop model
def pnz(p, q, i, j):
    side = lambda pp, ii: 0 if ii < pp - 1 else (1 if ii == pp - 1 else 2)
    a, b = side(p, i), side(q, j)
    return not ((a == 0 and b == 2) or (a == 2 and b == 0))


def p_hierarchy(k):
    lv, p = [], 1
    while p < k:
        lv.append(p)
        p = 2 * p + 1
    return lv + [k]


def patch_flops(d, k, n_iter=1):
    """Floating-point operations of one Cartesian patch solve as executed by
    the patch kernel: gather, full p-multigrid V-cycle (two patch vmults per
    level), scatter.  Counts an FMA as 2."""
    levels = p_hierarchy(k)

    def vmult(p):
        m = 2 * p - 1
        nnz = sum(pnz(p, p, i, j) for i in range(m) for j in range(m))
        if d == 3:
            return m * m * (2 * nnz * 2 + (3 * 2 * nnz + m) + (2 * 2 * nnz + 3 * m))
        return m * (2 * 2 * nnz + (2 * 2 * nnz + 3 * m))

    def vcycle(l):
        if l == 0:
            return 1
        p = levels[l]
        m = 2 * p - 1
        S = m ** d
        f = 3 * S + vmult(p) + vcycle(l - 1) + 4 * S + vmult(p)
        pc = levels[l - 1]
        mc = 2 * pc - 1
        nnz_t = sum(pnz(p, pc, i, j) for i in range(m) for j in range(mc))
        lines_r = (m * m + mc * m + mc * mc) if d == 3 else (m + mc)
        f += 2 * 2 * nnz_t * lines_r + S  # restriction + prolongation (+ add)
        return f

    top = len(levels) - 1
    m = 2 * k - 1
    f = vcycle(top) * n_iter + (n_iter - 1) * (vmult(k) + m ** d)
    return f + 2 * m ** d  # scatter u += omega d


def apply_flops_per_dof(d, k):
    """Cartesian apply: each 1D matrix costs (K+1) FMAs per output plus
    (K+1) more at the cell vertex; 7 matrix applications in 3D (4 in 2D)."""
    per_seg = 2 * (k + 1) * k + 2 * (k + 1)
    mats = 7 if d == 3 else 4
    return mats * per_seg / k


# ----------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self):
        self.samples = []
        self._stop = threading.Event()
        self._proc = None

    def start(self):
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-i", os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0],
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self._proc = None
            return
        threading.Thread(target=self._read, daemon=True).start()

    def _read(self):
        for line in self._proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self._proc:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ----------------------------------------------------------------- CPU oracle
def oracle_child(seconds, n_steps=0, case="sample"):
    """Runs in a fresh single-threaded process: time the oracle's step
    (apply + sweep + PCG solve) on the bounded sample of the benchmark
    workload (case "sample": 3D Q4 on ORACLE_N^3 cells) or on the 2D 16x16 Q2
    three-level problem in full (case "cfg1"), set-up excluded; exactly
    n_steps steps if n_steps > 0, else for about ``seconds``."""
    import numpy as np
    from oracle import constants, fem, solver
    if case == "cfg1":
        d, n, k, L = 2, 16, 2, 3
    else:
        d, n, k = D, ORACLE_N, K
        L, nn = 1, n
        while nn % 2 == 0:
            nn //= 2
            L += 1
    m = fem.Mesh(d, n, k)
    h = solver.Hierarchy(m, L, constants.omega_jacobi(d, k), constants.omega_patch(d))
    b = fem.rhs_manufactured(m)[m.interior_index()]
    fine = h.levels[-1]
    times = []
    t_end = time.time() + seconds
    while (len(times) < n_steps) if n_steps > 0 else (time.time() < t_end or len(times) < 3):
        t0 = time.perf_counter()
        fine.A @ b
        fine.smooth(b, np.zeros_like(b))
        x, it, hist = solver.solve(h, b)
        times.append(time.perf_counter() - t0)
    print(json.dumps({"dofs": m.n_dofs, "times": times, "iterations": it}))


def run_oracle(seconds, n_steps=0, case="sample"):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-child", str(seconds),
                        "--oracle-steps", str(n_steps), "--oracle-case", case],
                       capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle child failed:\n" + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline_entry(res):
    t = statistics.median(res["times"])
    return {"value": res["dofs"] / t, "unit": "DoFs/s", "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": "same step (apply + sweep + PCG/GMG solve to 1e-8, FP64, Q4, 3D, manufactured RHS) on "
                      "4^3 cells (%d DoFs), set-up excluded, median of %d steps, single thread"
                      % (res["dofs"], len(res["times"]))}


# ----------------------------------------------------------------- extra sections
def _measured_hbm_gbs():
    """The machine's measured copy bandwidth (generated MEASURED_PEAKS.json
    beside this file), else the profiling recipe's fallback of 6.8 TB/s."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


HBM_GBS, HBM_PEAK_KIND = _measured_hbm_gbs()


def _timed_ms(torch, stream, flush, fn, reps=5):
    fn()
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def extra_sections(p, torch, dev, stream, flush):
    """Deformed 96^3 Q3 (24,137,569 DoFs, FP32 G_q, mixed precision) and a
    bounded serving sample; reported beside the headline, outside its timing."""
    out = {}
    n, k = 96, 3
    ctx = p.Context(p.make_config(dim=3, n_cells=n, degree=k, geometry=p.DEFORMED, mg_precision=p.FP32),
                    stream=stream, device=dev)
    N = ctx.num_dofs()
    b = torch.empty(N, dtype=torch.float64, device=dev)
    ctx.rhs_manufactured(b)
    b32 = b.float()
    y32 = torch.empty_like(b32)
    x = torch.zeros_like(b)
    t_apply32 = _timed_ms(torch, stream, flush, lambda: ctx.apply(b32, y32, prec=p.FP32))
    t_apply64 = _timed_ms(torch, stream, flush, lambda: ctx.apply(b, x, prec=p.FP64), reps=3)
    phases = ctx.smoother_phase_times(reps=3)
    ctx.solve(b, x)
    solves = []
    for _ in range(3):
        flush.zero_()
        torch.cuda.synchronize()
        solves.append(ctx.solve(b, x))
    err = ctx.l2_error_manufactured(x)
    ncell = n ** 3
    g_bytes = ncell * (k + 1) ** 3 * 6 * 4
    alg_bytes = 8 * N + g_bytes  # x read + y write (FP32) + G_q read
    out["deformed_96_q3_mixed"] = {
        "dofs": N, "solve_ms_p50": pct([s.time_ms for s in solves], 50), "iterations": solves[-1].iterations,
        "rel_residual": solves[-1].rel_residual, "l2_error": err,
        "apply_fp32_ms": t_apply32, "apply_fp64_ms": t_apply64,
        "apply_fp32_roofline": {"bound": "hbm", "achieved": alg_bytes / (t_apply32 * 1e-3) / 1e9, "peak": HBM_GBS,
                                "peak_kind": HBM_PEAK_KIND,
                                "unit": "GB/s", "frac": alg_bytes / (t_apply32 * 1e-3) / 1e9 / HBM_GBS,
                                "algorithmic_bytes": alg_bytes},
        "smoother_phases_ms": {"residual": phases[0], "patch": phases[1], "gather": phases[2]},
    }
    ctx.close()
    # the same solve with the quadrature-point tensors stored in FP64: time
    # and the difference the FP32 storage makes to the solution
    ctx64g = p.Context(p.make_config(dim=3, n_cells=n, degree=k, geometry=p.DEFORMED, mg_precision=p.FP32,
                                     geom_precision=p.FP64), stream=stream, device=dev)
    x64g = torch.zeros_like(b)
    ctx64g.solve(b, x64g)
    solves64g = []
    for _ in range(3):
        flush.zero_()
        torch.cuda.synchronize()
        solves64g.append(ctx64g.solve(b, x64g))
    out["deformed_96_q3_mixed"]["fp64_geometry"] = {
        "solve_ms_p50": pct([s_.time_ms for s_ in solves64g], 50), "iterations": solves64g[-1].iterations,
        "l2_error": ctx64g.l2_error_manufactured(x64g),
        "rel_diff_x_fp32_vs_fp64_geometry": float(torch.linalg.norm(x - x64g) / torch.linalg.norm(x64g))}
    ctx64g.close()
    # the same solve with the float-float outer operator
    ctxff = p.Context(p.make_config(dim=3, n_cells=n, degree=k, geometry=p.DEFORMED, mg_precision=p.FP32,
                                    outer_apply=p.APPLY_FLOAT_FLOAT), stream=stream, device=dev)
    xff = torch.zeros_like(b)
    ctxff.solve(b, xff)
    solvesff = []
    for _ in range(3):
        flush.zero_()
        torch.cuda.synchronize()
        solvesff.append(ctxff.solve(b, xff))
    t_applyff = _timed_ms(torch, stream, flush, lambda: ctxff.apply(b, x64g, prec=p.FP64), reps=3)
    out["deformed_96_q3_mixed"]["float_float_operator"] = {
        "solve_ms_p50": pct([s_.time_ms for s_ in solvesff], 50), "iterations": solvesff[-1].iterations,
        "apply_ms": t_applyff, "l2_error": ctxff.l2_error_manufactured(xff),
        "rel_diff_x_vs_fp64_operator": float(torch.linalg.norm(x - xff) / torch.linalg.norm(x))}
    ctxff.close()
    del b, b32, y32, x, x64g, xff
    out["outer_solvers_32_q4"] = outer_solver_section(p, torch, dev, stream, flush)
    out["distorted_64_q3_mixed"] = distorted_section(p, torch, dev, stream, flush)
    out["serving_cfg4"] = serving_section(p, torch)
    return out


def serving_section(p, torch):
    """The served configuration as stated: 256 Poisson solve requests,
    Poisson arrivals at 50/s (seed 7), n log-uniform in [8, 64] snapped to
    {8, 12, 16, 24, 32, 48, 64} for k <= 5 and to powers of two above (seed
    11), k uniform in 2..7, N(0,1) right-hand sides (seeds 1000 + i), FP32
    V-cycle, FP64 CG to 1e-8, 16 slots, a fresh server per pass.  Passes: the
    process's first (cold: kernel modules loaded, smoother layouts tuned,
    coarse inverses computed) and a warm one, both served shortest-first
    with the float-float outer operator, then warm passes with grouped
    launches below the median work, and in arrival order with the FP64
    outer operator, for comparison; and a stream of small requests served
    with and without grouping."""
    import numpy as np
    from paper_2512_02577_gb300 import serve
    from paper_2512_02577_gb300.inputs import serving_requests
    reqs = serving_requests(n_requests=256, rate=50.0, snap="coarse")
    t0 = time.perf_counter()
    bufs = serve.prepare(reqs)
    prep_s = time.perf_counter() - t0
    # shortest-first: requests below the median estimated work (nodes x
    # (k + 2)) also get high-priority streams
    small = float(np.median([(r["k"] * r["n"] + 1) ** 3 * (r["k"] + 2) for r in reqs]))
    best = dict(policy=p.SERVE_SHORTEST_FIRST, max_wait_s=2.0, small_work=small, outer_apply=p.APPLY_FLOAT_FLOAT)
    # for comparison: requests below the median work in groups (their
    # iterations share each launch with the other running requests of their
    # degree)
    grouped = dict(best, group_work=small, max_group=16)
    res = {"workload": "256 requests, Poisson arrivals 50/s, n log-uniform 8..64 snapped to "
                       "{8,12,16,24,32,48,64} (k <= 5) / {8,16,32,64} (k >= 6), k uniform 2..7, N(0,1) RHS, "
                       "FP32 V-cycle, FP64 CG to 1e-8, 16 slots",
           "served_as": "shortest-first admission with 2 s aging, high-priority streams below the median work, "
                        "float-float outer operator",
           "total_dofs": int(sum((r["k"] * r["n"] + 1) ** 3 for r in reqs)), "prepare_s": prep_s}
    for label, kw in (("cold", best), ("warm", best), ("warm_grouped", grouped),
                      ("warm_fifo_fp64_operator", {})):
        recs, summ = serve.run(reqs, precision=p.FP32, max_active=16, buffers=bufs, **kw)
        lat = np.array([r["latency_s"] for r in recs])
        res[label] = {k: summ[k] for k in ("p50_ms", "p99_ms", "mean_ms", "makespan_s", "dofs_per_s", "failed",
                                           "max_iterations", "created_contexts")}
        res[label]["queue_p50_ms"] = float(np.median([r["queue_s"] for r in recs]) * 1e3)
        small_lat = [r["latency_s"] for r in recs if (r["k"] * r["n"] + 1) ** 3 * (r["k"] + 2) < small]
        res[label]["p50_below_median_work_ms"] = float(np.median(small_lat) * 1e3)
    del bufs
    # a stream of small requests, where grouping matters most: 256 requests
    # arriving at 2,000/s, n log-uniform 4..16 (powers of two), k uniform 2..5,
    # FP32 V-cycle, 32 slots; one stream per request vs groups of up to 16
    reqs = serving_requests(n_requests=256, rate=2000.0, arrival_seed=17, size_seed=19, n_lo=4, n_hi=16, k_lo=2,
                            k_hi=5)
    bufs = serve.prepare(reqs)
    small_res = {"workload": "256 requests, Poisson arrivals 2000/s, n log-uniform 4..16 (powers of two), "
                             "k uniform 2..5, N(0,1) RHS, FP32 V-cycle, FP64 CG to 1e-8, 32 slots",
                 "total_dofs": int(sum((r["k"] * r["n"] + 1) ** 3 for r in reqs))}
    for label, kw in (("warmup", {}), ("streams", {}), ("grouped", dict(group_work=1e18, max_group=16))):
        recs, summ = serve.run(reqs, precision=p.FP32, max_active=32, buffers=bufs, **kw)
        if label != "warmup":
            small_res[label] = {k: summ[k] for k in ("p50_ms", "p99_ms", "mean_ms", "makespan_s", "dofs_per_s",
                                                     "failed", "created_contexts")}
    del bufs
    res["small_requests"] = small_res
    return res


def distorted_section(p, torch, dev, stream, flush):
    """Randomly distorted 3D 64^3 Q3 mesh (7,189,057 DoFs; every interior
    vertex moved by 0.25 h in a random direction, seed 2512), mixed
    precision: additive and multiplicative smoothers, each with the full
    local cycle under CG and with the half cycle under GMRES; median of 3
    solves (L2 flushed before each), plus the stored-G_q FP32 apply."""
    from paper_2512_02577_gb300.inputs import vertex_displacements
    n, k, delta = 64, 3, 0.25
    disp = vertex_displacements(3, n, delta, 2512)
    res = {"delta": delta}
    for sm, half, outer, name in ((p.ADDITIVE, 0, p.OUTER_CG, "full_cg"), (p.ADDITIVE, 1, p.OUTER_GMRES, "half_gmres"),
                                  (p.MULTIPLICATIVE, 0, p.OUTER_CG, "mult_full_cg"),
                                  (p.MULTIPLICATIVE, 1, p.OUTER_GMRES, "mult_half_gmres")):
        ctx = p.Context(p.make_config(dim=3, n_cells=n, degree=k, geometry=p.DISTORTED, vertex_disp=disp,
                                      mg_precision=p.FP32, local_half=half, outer_solver=outer, smoother=sm),
                        stream=stream, device=dev)
        b = torch.empty(ctx.num_dofs(), dtype=torch.float64, device=dev)
        ctx.rhs_manufactured(b)
        x = torch.zeros_like(b)
        ctx.solve(b, x)
        infos = []
        for _ in range(3):
            flush.zero_()
            torch.cuda.synchronize()
            infos.append(ctx.solve(b, x))
        res[name] = {"solve_ms_p50": pct([i.time_ms for i in infos], 50), "iterations": infos[-1].iterations,
                     "rel_residual": infos[-1].rel_residual, "l2_error": ctx.l2_error_manufactured(x),
                     "smoother_phases_ms": dict(zip(("residual", "patch", "gather"),
                                                    ctx.smoother_phase_times(reps=3)))}
        if name == "full_cg":
            b32, y32 = b.float(), torch.empty(ctx.num_dofs(), dtype=torch.float32, device=dev)
            res["dofs"] = ctx.num_dofs()
            res["apply_fp32_ms"] = _timed_ms(torch, stream, flush, lambda: ctx.apply(b32, y32, prec=p.FP32))
            del b32, y32
        ctx.close()
        del b, x
    return res


def outer_solver_section(p, torch, dev, stream, flush):
    """3D 32^3 Q4 manufactured problem: additive smoother with the full
    local V-cycle under CG and GMRES and with the half local V-cycle (§3.2.2)
    under GMRES; multiplicative smoother (Algorithm 1, colour by colour) with
    the full cycle under CG and the half cycle under GMRES (the paper's
    configuration); FP64 and mixed; median of 3 solves (L2 flushed before
    each) and the smoother's patch launch time (all patches)."""
    res = {}
    for prec, pname in ((p.FP64, "fp64"), (p.FP32, "mixed")):
        for sm, half, outer, name in ((p.ADDITIVE, 0, p.OUTER_CG, "full_cg"),
                                      (p.ADDITIVE, 0, p.OUTER_GMRES, "full_gmres"),
                                      (p.ADDITIVE, 1, p.OUTER_GMRES, "half_gmres"),
                                      (p.MULTIPLICATIVE, 0, p.OUTER_CG, "mult_full_cg"),
                                      (p.MULTIPLICATIVE, 1, p.OUTER_GMRES, "mult_half_gmres")):
            ctx = p.Context(p.make_config(dim=3, n_cells=32, degree=4, mg_precision=prec, local_half=half,
                                          outer_solver=outer, smoother=sm, coarse_dofs=COARSE_DOFS),
                            stream=stream, device=dev)
            b = torch.empty(ctx.num_dofs(), dtype=torch.float64, device=dev)
            ctx.rhs_manufactured(b)
            x = torch.zeros_like(b)
            ctx.solve(b, x)
            infos = []
            for _ in range(3):
                flush.zero_()
                torch.cuda.synchronize()
                infos.append(ctx.solve(b, x))
            res["%s_%s" % (pname, name)] = {
                "solve_ms_p50": pct([i.time_ms for i in infos], 50), "iterations": infos[-1].iterations,
                "rel_residual": infos[-1].rel_residual, "l2_error": ctx.l2_error_manufactured(x),
                "patch_launch_ms": ctx.smoother_phase_times(reps=3)[1]}
            ctx.close()
    return res


def degree_sweep():
    """k = 1..8 on the unit cube: apply and smoother step at n = round(200/k)
    (~8M DoFs; odd n: single-level contexts, the step on that level), FP64,
    mixed and mixed with the float-float outer operator solves on the
    nearest power-of-two mesh whose coarse level stays small; N(0,1)
    right-hand side (seed 20251202 + k)."""
    import torch
    import paper_2512_02577_gb300 as p
    from paper_2512_02577_gb300.inputs import random_vector
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    rows = []
    with torch.cuda.stream(stream):
        for k in range(1, 9):
            n = int(round(200.0 / k))
            row = {"k": k, "n": n}
            for prec in (p.FP64, p.FP32):
                ctx = p.Context(p.make_config(dim=3, n_cells=n, degree=k, n_levels=1 if n % 2 else 2,
                                              mg_precision=prec), stream=stream, device=dev)
                N = ctx.num_dofs()
                dt = torch.float64 if prec == p.FP64 else torch.float32
                xv = torch.randn(N, dtype=dt, device=dev)
                yv = torch.empty_like(xv)
                ta = _timed_ms(torch, stream, flush, lambda: ctx.apply(xv, yv, prec=prec))
                tag = "fp64" if prec == p.FP64 else "fp32"
                row["dofs_apply"] = N
                row["apply_%s_ms" % tag] = ta
                row["apply_%s_gdofs" % tag] = N / ta / 1e6
                ph = ctx.smoother_phase_times(reps=2)   # finest level (odd n: the single level)
                row["sweep_%s_ms" % tag] = sum(ph)
                row["sweep_%s_gdofs" % tag] = N / sum(ph) / 1e6
                ctx.close()
            ns = 2 ** int(round(__import__("math").log2(200.0 / k)))
            row["n_solve"] = ns
            for prec, apply, tag in ((p.FP64, p.APPLY_FP64, "fp64"), (p.FP32, p.APPLY_FP64, "mixed"),
                                     (p.FP32, p.APPLY_FLOAT_FLOAT, "mixed_ff")):
                ctx = p.Context(p.make_config(dim=3, n_cells=ns, degree=k, mg_precision=prec, outer_apply=apply),
                                stream=stream, device=dev)
                b = torch.tensor(random_vector(3, ns, k, seed=20251202 + k), device=dev)
                x = torch.zeros_like(b)
                ctx.solve(b, x)
                infos = [ctx.solve(b, x) for _ in range(2)]
                row["dofs_solve"] = ctx.num_dofs()
                row["solve_%s_ms" % tag] = min(i.time_ms for i in infos)
                row["iterations_%s" % tag] = infos[-1].iterations
                row["rel_residual_%s" % tag] = infos[-1].rel_residual
                ctx.close()
            row["mixed_speedup"] = row["solve_fp64_ms"] / row["solve_mixed_ms"]
            row["mixed_ff_speedup"] = row["solve_fp64_ms"] / row["solve_mixed_ff_ms"]
            print(json.dumps(row), flush=True)
            rows.append(row)
    print(json.dumps({"degree_sweep": rows}))


# ----------------------------------------------------------------- profiling
def profile_region(region, n_def, k_prof=0):
    """One NVTX range named 'profile' after warm-up, for
    ncu --nvtx --nvtx-include "profile/": one mixed-precision solve of the
    32^3 Q4 problem (degree k_prof instead of 4 if given; with the FP64 or
    the float-float outer operator), one
    FP32 apply and one FP32 sweep of the deformed Q3 problem on n_def^3 cells,
    one FP32 apply of the Cartesian Q3 problem on n_def^3 cells, or one
    grouped solve of 16 Q3 systems on 4^3, 8^3, 16^3 and 8^3 cells
    (four of each, FP32 V-cycle)."""
    import torch
    import paper_2512_02577_gb300 as p
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        if region in ("mixed_solve", "mixed_solve_ff"):
            apply = p.APPLY_FLOAT_FLOAT if region == "mixed_solve_ff" else p.APPLY_FP64
            k = k_prof or K
            ctx = p.Context(p.make_config(dim=D, n_cells=NCELL, degree=k, mg_precision=p.FP32, outer_apply=apply,
                                          coarse_dofs=COARSE_DOFS),
                            stream=stream, device=dev)
            b = torch.empty(ctx.num_dofs(), dtype=torch.float64, device=dev)
            ctx.rhs_manufactured(b)
            x = torch.zeros_like(b)
            for _ in range(3):
                ctx.solve(b, x)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push("profile")
            ctx.solve(b, x)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
        elif region == "cart_apply32":
            ctx = p.Context(p.make_config(dim=3, n_cells=n_def, degree=3, mg_precision=p.FP32), stream=stream,
                            device=dev)
            x = torch.randn(ctx.num_dofs(), dtype=torch.float32, device=dev)
            y = torch.empty_like(x)
            for _ in range(3):
                ctx.apply(x, y, prec=p.FP32)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push("profile")
            ctx.apply(x, y, prec=p.FP32)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
        elif region == "grouped":
            from paper_2512_02577_gb300.inputs import random_vector
            ns = [4, 8, 16, 8] * 4
            ctxs = [p.Context(p.make_config(dim=3, n_cells=n, degree=3, mg_precision=p.FP32), stream=stream,
                              device=dev) for n in ns]
            bs = [torch.from_numpy(random_vector(3, n, 3, seed=i)).to(dev) for i, n in enumerate(ns)]
            xs = [torch.zeros_like(b) for b in bs]
            for _ in range(3):
                p.solve_group(ctxs, bs, xs)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push("profile")
            p.solve_group(ctxs, bs, xs)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
        else:
            ctx = p.Context(p.make_config(dim=3, n_cells=n_def, degree=3, geometry=p.DEFORMED,
                                          mg_precision=p.FP32), stream=stream, device=dev)
            N = ctx.num_dofs()
            x = torch.randn(N, dtype=torch.float32, device=dev)
            y = torch.empty_like(x)
            for _ in range(3):
                ctx.apply(x, y, prec=p.FP32)
                ctx.smooth(x, y)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push("profile")
            ctx.apply(x, y, prec=p.FP32)
            ctx.smooth(x, y)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()


# ----------------------------------------------------------------- ranks
def reduce_over_ranks(local_ms, local_dofs, device=None):
    """Replicas: the job's time is the slowest rank's, its work the sum of
    all ranks' DoFs.  Single process: unchanged."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_ms), float(local_dofs)
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    w = torch.tensor([float(local_dofs)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


# ----------------------------------------------------------------- main
def pct(xs, q):
    xs = sorted(xs)
    i = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[i]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--oracle-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-child", type=float, default=None)
    ap.add_argument("--oracle-steps", type=int, default=0)
    ap.add_argument("--oracle-case", default="sample", choices=["sample", "cfg1"])
    ap.add_argument("--profile-region", default=None, choices=["mixed_solve", "mixed_solve_ff", "deformed", "grouped", "cart_apply32"],
                    help="warm up, then run one NVTX-marked region 'profile' for ncu and exit")
    ap.add_argument("--profile-k", type=int, default=0, help="degree of the mixed-solve profile case (0: 4)")
    ap.add_argument("--profile-n", type=int, default=48, help="cells per side of the deformed and Cartesian-apply profile cases")
    ap.add_argument("--no-extras", action="store_true", help="skip the deformed and serving sections")
    ap.add_argument("--sweep", action="store_true", help="degree sweep k = 1..8 at ~8M DoFs (separate JSON)")
    args = ap.parse_args()
    if args.oracle_child is not None:
        oracle_child(args.oracle_child, args.oracle_steps, args.oracle_case)
        return
    if args.profile_region:
        profile_region(args.profile_region, args.profile_n, args.profile_k)
        return
    if args.sweep:
        degree_sweep()
        return
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        # exactly W untimed + K timed oracle steps, each on the bounded sample
        res = run_oracle(0.0, n_steps=args.warmup + max(args.steps, 1))
        times = res["times"][args.warmup:]
        t = statistics.median(times)
        value = res["dofs"] / t
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DoFs/s", "n_gpus": args.gpus,
                "steps": len(times), "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "sample": "4^3 cells of the same workload (%d DoFs)" % res["dofs"]},
                "cpu_baseline": dict(cpu_baseline_entry(res), value=value),
                "e2e": {"value": value, "unit": "DoFs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    import paper_2512_02577_gb300 as p

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    # CPU baseline before any GPU work of this process's children
    cpu = cpu1 = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_entry(run_oracle(args.oracle_seconds))
        r1 = run_oracle(min(args.oracle_seconds, 5.0), case="cfg1")
        t1 = statistics.median(r1["times"])
        cpu1 = {"workload": "2D unit square, 16x16 Q2, 3 levels (1,089 DoFs), manufactured RHS, in full",
                "step_ms": t1 * 1e3, "dofs_per_s": r1["dofs"] / t1, "cg_iterations": r1["iterations"],
                "cores": 1, "host_cores": os.cpu_count(), "steps": len(r1["times"])}

    stream = torch.cuda.Stream(device=dev)
    cfg = p.make_config(dim=D, n_cells=NCELL, degree=K, mg_precision=p.FP64, coarse_dofs=COARSE_DOFS)
    cfg32 = p.make_config(dim=D, n_cells=NCELL, degree=K, mg_precision=p.FP32, coarse_dofs=COARSE_DOFS)
    with torch.cuda.stream(stream):
        ctx = p.Context(cfg, stream=stream, device=dev)
        ctx32 = p.Context(cfg32, stream=stream, device=dev)
        N = ctx.num_dofs()
        b = torch.empty(N, dtype=torch.float64, device=dev)
        ctx.rhs_manufactured(b)
        xa = torch.empty_like(b)
        ctx.rhs_manufactured(xa)
        ya = torch.empty_like(b)
        u = torch.empty_like(b)
        xs = torch.empty_like(b)
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

        def step(info_out=None):
            ctx.apply(xa, ya)
            u.zero_()
            ctx.smooth(b, u)
            info = ctx.solve(b, xs, rtol=1e-8)
            if info_out is not None:
                info_out.append(info)

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        infos = []
        clocks = ClockSampler()
        clocks.start()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        l0 = p.launch_count()
        torch.cuda.nvtx.range_push("timed_step")
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step(infos)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        launches = p.launch_count() - l0
        if world > 1:
            torch.distributed.barrier()
        clocks.stop()
        step_ms = [a.elapsed_time(z) for a, z in ev]
        total_ms, total_dofs = reduce_over_ranks(sum(step_ms), N * args.steps, dev)
        ms_per_step = total_ms / args.steps
        value = total_dofs / (total_ms * 1e-3)

        # ---- component timings (not part of value): apply, sweep, residual, solves
        def timed(fn, reps):
            for _ in range(2):
                fn()
            ts = []
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return ts

        t_apply = timed(lambda: ctx.apply(xa, ya), 20)
        t_res = timed(lambda: ctx.residual(b, xa, ya), 20)
        t_sweep = timed(lambda: ctx.smooth(b, u), 10)
        solve64 = [i.time_ms for i in infos]
        it64 = infos[-1].iterations
        res64 = infos[-1].rel_residual
        info32 = []
        for _ in range(2):
            ctx32.solve(b, xs)
        for _ in range(max(args.steps, 5)):
            flush.zero_()
            torch.cuda.synchronize()
            info32.append(ctx32.solve(b, xs, rtol=1e-8))
        l2err = ctx32.l2_error_manufactured(xs)
        ctx.solve(b, xs)
        l2err64 = ctx.l2_error_manufactured(xs)
        solve32 = [i.time_ms for i in info32]
        # mixed precision with the float-float outer operator
        ctxff = p.Context(p.make_config(dim=D, n_cells=NCELL, degree=K, mg_precision=p.FP32,
                                        outer_apply=p.APPLY_FLOAT_FLOAT, coarse_dofs=COARSE_DOFS),
                          stream=stream, device=dev)
        infoff = []
        for _ in range(2):
            ctxff.solve(b, xs)
        for _ in range(max(args.steps, 5)):
            flush.zero_()
            torch.cuda.synchronize()
            infoff.append(ctxff.solve(b, xs, rtol=1e-8))
        Axs = torch.empty_like(xs)
        ctx.apply(xs, Axs)                        # true residual with the FP64 operator
        true_res_ff = float(torch.linalg.norm(b - Axs) / torch.linalg.norm(b))
        l2err_ff = ctxff.l2_error_manufactured(xs)
        t_apply_ff = timed(lambda: ctxff.apply(xa, ya), 20)
        solveff = [i.time_ms for i in infoff]
        ctxff.close()

        # roofline of the dominant kernel: the FP64 patch launch (every local
        # solve of the finest level), timed live on the library's stream
        sweep_ms = statistics.median(t_sweep)
        phases = ctx.smoother_phase_times(reps=10)
        patch_launch_ms = phases[1]
        n_patches = (NCELL - 1) ** D
        flops_launch = patch_flops(D, K) * n_patches
        achieved = flops_launch / (patch_launch_ms * 1e-3) / 1e12
        phases32 = ctx32.smoother_phase_times(reps=10)

        # ---- end-to-end through the host-buffer C-ABI path
        pin_b = b.cpu().pin_memory()
        pin_x = torch.empty(N, dtype=torch.float64).pin_memory()
        pin_xa = xa.cpu().pin_memory()
        pin_ya = torch.empty(N, dtype=torch.float64).pin_memory()
        pin_u = torch.empty(N, dtype=torch.float64).pin_memory()
        db = torch.empty_like(b)

        def e2e_step():
            xa.copy_(pin_xa, non_blocking=True)
            db.copy_(pin_b, non_blocking=True)
            ctx.apply(xa, ya)
            u.zero_()
            ctx.smooth(db, u)
            ctx.solve_host(pin_b, pin_x, rtol=1e-8)
            pin_ya.copy_(ya, non_blocking=True)
            pin_u.copy_(u, non_blocking=True)
            torch.cuda.synchronize()

        for _ in range(2):
            e2e_step()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        # whole job: every rank's DoFs over the slowest rank's wall time
        e2e_ms, e2e_dofs = reduce_over_ranks((time.perf_counter() - t0) * 1e3, N * args.steps, dev)
        e2e_value = e2e_dofs / (e2e_ms * 1e-3)
        extra = {} if args.no_extras else extra_sections(p, torch, dev, stream, flush)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": "DoFs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "dofs": N, "l2_flush": "512 MB write between timed steps",
                   "parallelism": "replicas" if world > 1 else "single GPU", "smoother": "additive vertex patch",
                   "local_solver": "full p-multigrid V-cycle", "levels": ctx.n_levels,
                   "coarsest": "%d^3 cells, dense inverse (coarse_dofs %d)" % (NCELL >> (ctx.n_levels - 1), COARSE_DOFS)},
        "gpu_launches": launches,
        "apply_dofs_per_s": N / (statistics.median(t_apply) * 1e-3),
        "sweep_dofs_per_s": N / (sweep_ms * 1e-3),
        "solve_fp64_ms": {"p50": pct(solve64, 50), "p99": pct(solve64, 99), "iterations": it64,
                          "rel_residual": res64, "l2_error": l2err64},
        "solve_mixed_ms": {"p50": pct(solve32, 50), "p99": pct(solve32, 99), "iterations": info32[-1].iterations,
                           "rel_residual": info32[-1].rel_residual, "l2_error": l2err},
        "mixed_speedup_vs_fp64": pct(solve64, 50) / pct(solve32, 50),
        "solve_mixed_float_float_operator_ms": {
            "p50": pct(solveff, 50), "p99": pct(solveff, 99), "iterations": infoff[-1].iterations,
            "rel_residual": infoff[-1].rel_residual, "true_rel_residual_fp64_operator": true_res_ff,
            "l2_error": l2err_ff, "apply_ms": statistics.median(t_apply_ff),
            "speedup_vs_fp64": pct(solve64, 50) / pct(solveff, 50)},
        "roofline": {"kernel": "patch_cart_kernel<3,double> (all 29,791 patches of the finest level)",
                     "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS, "traffic": PATCH64_TRAFFIC_BYTES,
                     "flops_per_launch": flops_launch, "launch_ms": patch_launch_ms,
                     "peak_note": "nominal FP64 (measured FMA probe 1.255 TFLOP/s)"},
        "smoother_phases_ms": {"fp64": {"residual": phases[0], "patch": phases[1], "gather": phases[2]},
                               "fp32": {"residual": phases32[0], "patch": phases32[1], "gather": phases32[2],
                                        "patch_tflops": flops_launch / (phases32[1] * 1e-3) / 1e12,
                                        "patch_frac_of_fp32_peak":
                                            flops_launch / (phases32[1] * 1e-3) / 1e12 / FP32_PEAK_TFLOPS}},
        "e2e": {"value": e2e_value, "unit": "DoFs/s", "h2d_bytes_per_step": 3 * 8 * N * world,
                "d2h_bytes_per_step": 3 * 8 * N * world},
        "clocks": clocks.summary(),
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
        line["cpu_oracle_2d_16_q2"] = cpu1
    line.update(extra)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
