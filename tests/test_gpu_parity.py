"""CUDA path vs the CPU oracle, through the C ABI.

Tolerances (each check bounds both the relative 2-norm ||a - b|| / ||b|| and
the element-wise max|a - b| / max|b|, see tests/parity.py):
  FP64 operator apply / residual       1e-12
  FP64 smoother sweep / V-cycle        1e-11  (summation order differs)
  FP32 apply / sweep / V-cycle         2e-5 vs the oracle's FP64
  FP64 solve: ||r||/||b|| <= 1e-8, CG iterations within +-1 of the oracle's
  mixed solve: ||r||/||b|| <= 1e-8, solution within 1e-6 of the oracle's
"""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2512_02577_gb300 as p
from oracle import constants, fem, solver
from paper_2512_02577_gb300.inputs import random_vector

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


from tests.parity import rel  # noqa: E402  (max of norm-relative and element-wise error)


def make_ctx(d, n, k, L=0, geom="cartesian", prec=p.FP64, **kw):
    cfg = p.make_config(dim=d, n_cells=n, degree=k, n_levels=L,
                        geometry=p.DEFORMED if geom == "deformed" else p.CARTESIAN,
                        deform_amp=0.05, mg_precision=prec,
                        omega_jacobi=constants.omega_jacobi(d, k), omega_patch=constants.omega_patch(d), **kw)
    return p.Context(cfg, device=DEV)


@functools.lru_cache(maxsize=None)
def oracle_level(d, n, k, geom, n_iter=1):
    m = fem.Mesh(d, n, k, geom, 0.05, geom_fp32=True)
    return solver.Level(m, constants.omega_jacobi(d, k), constants.omega_patch(d), n_iter=n_iter)


@functools.lru_cache(maxsize=None)
def oracle_operator(d, n, k, geom):
    """Assembled level operator only (no patch solvers): apply tests."""
    m = fem.Mesh(d, n, k, geom, 0.05, geom_fp32=True)
    return solver.Level(m, constants.omega_jacobi(d, k), constants.omega_patch(d), with_patches=False)


@functools.lru_cache(maxsize=None)
def oracle_hier(d, n, k, L, geom):
    m = fem.Mesh(d, n, k, geom, 0.05, geom_fp32=True)
    return solver.Hierarchy(m, L, constants.omega_jacobi(d, k), constants.omega_patch(d))


def n_levels_auto(n):
    L = 1
    while n % 2 == 0:
        n //= 2
        L += 1
    return L


def to_dev(v, dtype=torch.float64):
    return torch.tensor(v, dtype=dtype, device=DEV)


def full(lev, v_int):
    out = np.zeros(lev.mesh.n_dofs)
    out[lev.I] = v_int
    return out


APPLY_CASES = [(2, 16, 2, "cartesian"), (2, 5, 3, "cartesian"), (2, 3, 8, "cartesian"), (3, 4, 1, "cartesian"),
               (3, 3, 2, "cartesian"), (3, 4, 3, "cartesian"), (3, 3, 4, "cartesian"), (3, 2, 5, "cartesian"),
               (3, 2, 6, "cartesian"), (3, 2, 7, "cartesian"), (3, 2, 8, "cartesian"), (2, 6, 3, "deformed"),
               (3, 3, 2, "deformed"), (3, 4, 3, "deformed"), (3, 2, 4, "deformed")]


@pytest.mark.parametrize("d,n,k,geom", APPLY_CASES)
def test_apply_and_residual_fp64(d, n, k, geom):
    ctx = make_ctx(d, n, k, L=1, geom=geom)
    lev = oracle_operator(d, n, k, geom)
    x = random_vector(d, n, k, seed=10 + n + k)
    x_noisy = x.copy()
    x_noisy[~lev.mesh.interior_mask()] = 7.0       # boundary inputs are ignored
    y = torch.empty(lev.mesh.n_dofs, dtype=torch.float64, device=DEV)
    ctx.apply(to_dev(x_noisy), y)
    y_ref = fem.apply_full(lev.mesh, lev.A, x)
    yh = y.cpu().numpy()
    assert rel(yh, y_ref) < 1e-12
    assert np.all(yh[~lev.mesh.interior_mask()] == 0)
    b = random_vector(d, n, k, seed=99)
    r = torch.empty_like(y)
    ctx.residual(to_dev(b), to_dev(x), r)
    assert rel(r.cpu().numpy(), b - y_ref) < 1e-12


@pytest.mark.parametrize("d,n,k,geom", [(2, 16, 2, "cartesian"), (3, 4, 3, "cartesian"), (3, 2, 8, "cartesian"),
                                        (3, 4, 3, "deformed")])
def test_apply_fp32(d, n, k, geom):
    ctx = make_ctx(d, n, k, L=1, geom=geom, prec=p.FP32)
    lev = oracle_operator(d, n, k, geom)
    x = random_vector(d, n, k, seed=3)
    y = torch.empty(lev.mesh.n_dofs, dtype=torch.float32, device=DEV)
    ctx.apply(to_dev(x, torch.float32), y, prec=p.FP32)
    assert rel(y.cpu().double().numpy(), fem.apply_full(lev.mesh, lev.A, x)) < 2e-5


SMOOTH_CASES = [(2, 8, 2, "cartesian"), (2, 6, 3, "cartesian"), (2, 4, 4, "cartesian"), (2, 6, 1, "cartesian"),
                (3, 4, 2, "cartesian"), (3, 6, 3, "cartesian"), (3, 4, 4, "cartesian"), (3, 2, 5, "cartesian"),
                (3, 4, 1, "cartesian"), (2, 4, 8, "cartesian"), (2, 6, 2, "deformed"), (3, 4, 2, "deformed"),
                (3, 4, 3, "deformed")]


@pytest.mark.parametrize("d,n,k,geom", SMOOTH_CASES)
def test_smoother_sweep_fp64(d, n, k, geom):
    ctx = make_ctx(d, n, k, L=2, geom=geom)
    lev = oracle_level(d, n, k, geom)
    b = random_vector(d, n, k, seed=21)
    u0 = random_vector(d, n, k, seed=22)
    u = to_dev(u0)
    ctx.smooth(to_dev(b), u, sweeps=2)
    ref = lev.smooth(b[lev.I], u0[lev.I], sweeps=2)
    assert rel(u.cpu().numpy(), full(lev, ref)) < 1e-11


@pytest.mark.parametrize("d,n,k,geom", [(2, 8, 3, "cartesian"), (3, 4, 3, "cartesian"), (3, 4, 2, "deformed")])
def test_smoother_sweep_fp32(d, n, k, geom):
    ctx = make_ctx(d, n, k, L=2, geom=geom, prec=p.FP32)
    lev = oracle_level(d, n, k, geom)
    b = random_vector(d, n, k, seed=31)
    u = torch.zeros(lev.mesh.n_dofs, dtype=torch.float32, device=DEV)
    ctx.smooth(to_dev(b, torch.float32), u, sweeps=1)
    ref = lev.smooth(b[lev.I], np.zeros(len(lev.I)), sweeps=1)
    assert rel(u.cpu().double().numpy(), full(lev, ref)) < 2e-5


def test_smoother_local_richardson_cycles():
    d, n, k = 3, 4, 3
    cfg_kw = dict(local_cycles=3)
    ctx = make_ctx(d, n, k, L=2, **cfg_kw)
    lev = oracle_level(d, n, k, "cartesian", n_iter=3)
    b = random_vector(d, n, k, seed=41)
    u = torch.zeros(lev.mesh.n_dofs, dtype=torch.float64, device=DEV)
    ctx.smooth(to_dev(b), u)
    ref = lev.smooth(b[lev.I], np.zeros(len(lev.I)))
    assert rel(u.cpu().numpy(), full(lev, ref)) < 1e-11


VCYCLE_CASES = [(2, 16, 2, 3, "cartesian"), (2, 8, 4, 0, "cartesian"), (3, 4, 2, 0, "cartesian"),
                (3, 4, 3, 0, "cartesian"), (3, 8, 1, 0, "cartesian"), (3, 6, 2, 2, "cartesian"),
                (2, 8, 3, 0, "deformed"), (3, 4, 2, 0, "deformed")]


@pytest.mark.parametrize("d,n,k,L,geom", VCYCLE_CASES)
def test_vcycle_fp64(d, n, k, L, geom):
    ctx = make_ctx(d, n, k, L=L, geom=geom)
    Lo = L if L else n_levels_auto(n)
    h = oracle_hier(d, n, k, Lo, geom)
    fine = h.levels[-1]
    r = random_vector(d, n, k, seed=51)
    z = torch.empty(fine.mesh.n_dofs, dtype=torch.float64, device=DEV)
    ctx.vcycle(to_dev(r), z)
    ref = h.vcycle(r[fine.I])
    assert rel(z.cpu().numpy(), full(fine, ref)) < 1e-11
    # the graph replay gives the same result
    z2 = torch.empty_like(z)
    ctx.vcycle(to_dev(r), z2)
    assert torch.equal(z, z2)


@pytest.mark.parametrize("d,n,k,L,geom", [(2, 16, 2, 3, "cartesian"), (3, 4, 3, 0, "cartesian"),
                                          (3, 4, 2, 0, "deformed")])
def test_vcycle_fp32(d, n, k, L, geom):
    ctx = make_ctx(d, n, k, L=L, geom=geom, prec=p.FP32)
    h = oracle_hier(d, n, k, L if L else n_levels_auto(n), geom)
    fine = h.levels[-1]
    r = random_vector(d, n, k, seed=52)
    z = torch.empty(fine.mesh.n_dofs, dtype=torch.float64, device=DEV)
    ctx.vcycle(to_dev(r), z)
    assert rel(z.cpu().numpy(), full(fine, h.vcycle(r[fine.I]))) < 2e-5


SOLVE_CASES = [(2, 16, 2, 3, "cartesian"), (2, 16, 4, 0, "cartesian"), (3, 8, 2, 0, "cartesian"),
               (3, 4, 4, 0, "cartesian"), (2, 8, 3, 0, "deformed"), (3, 4, 3, 0, "deformed")]


@pytest.mark.parametrize("d,n,k,L,geom", SOLVE_CASES)
@pytest.mark.parametrize("prec", [p.FP64, p.FP32])
def test_solve(d, n, k, L, geom, prec):
    ctx = make_ctx(d, n, k, L=L, geom=geom, prec=prec)
    h = oracle_hier(d, n, k, L if L else n_levels_auto(n), geom)
    fine = h.levels[-1]
    m = fine.mesh
    b_ref = fem.rhs_manufactured(m)
    b = torch.empty(m.n_dofs, dtype=torch.float64, device=DEV)
    ctx.rhs_manufactured(b)
    assert rel(b.cpu().numpy(), b_ref) < 1e-13
    x = torch.zeros_like(b)
    info = ctx.solve(b, x, rtol=1e-8)
    x_ref, it_ref, _ = solver.solve(h, b_ref[fine.I], rtol=1e-8)
    assert info.status == 0 and info.rel_residual <= 1e-8
    xh = x.cpu().numpy()
    true_res = np.linalg.norm(b_ref[fine.I] - fine.A @ xh[fine.I]) / np.linalg.norm(b_ref[fine.I])
    assert true_res <= 2e-8
    if prec == p.FP64:
        assert abs(info.iterations - it_ref) <= 1, (info.iterations, it_ref)
    else:
        assert info.iterations <= it_ref + 3, (info.iterations, it_ref)
    assert rel(xh, full(fine, x_ref)) < (1e-6 if prec == p.FP64 else 1e-5)
    # discretisation error through the library equals the oracle's
    e_lib = ctx.l2_error_manufactured(x)
    e_ref = fem.l2_error_manufactured(m, full(fine, x_ref))
    assert abs(e_lib - e_ref) <= 1e-4 * e_ref + 1e-12


def test_solve_host_buffers_match_device():
    ctx = make_ctx(3, 4, 3)
    n = ctx.num_dofs()
    b = torch.empty(n, dtype=torch.float64, device=DEV)
    ctx.rhs_manufactured(b)
    x = torch.zeros_like(b)
    info = ctx.solve(b, x)
    bh = b.cpu().pin_memory()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()
    info_h = ctx.solve_host(bh, xh)
    assert info_h.iterations == info.iterations
    assert torch.equal(xh, x.cpu())


def test_l2_convergence_rate_through_library():
    for k, ns in ((2, (4, 8, 16)), (3, (4, 8, 16))):
        errs = []
        for n in ns:
            ctx = make_ctx(3, n, k)
            b = torch.empty(ctx.num_dofs(), dtype=torch.float64, device=DEV)
            ctx.rhs_manufactured(b)
            x = torch.zeros_like(b)
            ctx.solve(b, x, rtol=1e-12, maxit=200)
            errs.append(ctx.l2_error_manufactured(x))
        rate = np.log2(errs[-2] / errs[-1])
        assert abs(rate - (k + 1)) < 0.25, (k, errs)


# ------------------------------------------------------------------ edge cases
def test_single_cell_mesh_is_a_coarse_solve():
    # n = 1: no patches; the V-cycle is the exact coarse solve, CG takes 1 step
    ctx = make_ctx(3, 1, 4)
    b = to_dev(random_vector(3, 1, 4, seed=5))
    x = torch.zeros_like(b)
    info = ctx.solve(b, x, rtol=1e-10)
    assert info.iterations == 1 and info.rel_residual < 1e-12


def test_zero_rhs_gives_zero_solution():
    ctx = make_ctx(2, 8, 2)
    b = torch.zeros(ctx.num_dofs(), dtype=torch.float64, device=DEV)
    x = torch.ones_like(b)
    info = ctx.solve(b, x)
    assert info.iterations == 0 and torch.count_nonzero(x) == 0


def test_not_converged_is_reported():
    ctx = make_ctx(3, 8, 2)
    b = to_dev(random_vector(3, 8, 2, seed=6))
    x = torch.zeros_like(b)
    info = ctx.solve(b, x, rtol=1e-14, maxit=2)
    assert info.status == p.PMG_NOT_CONVERGED and info.iterations == 2


def test_bad_arguments_raise_not_crash():
    ctx = make_ctx(2, 8, 2)
    n = ctx.num_dofs()
    with pytest.raises(ValueError):
        ctx.apply(torch.zeros(n - 1, dtype=torch.float64, device=DEV), torch.zeros(n, dtype=torch.float64, device=DEV))
    with pytest.raises(p.PmgError):
        ctx.apply(torch.zeros(n, dtype=torch.float64, device=DEV), torch.zeros(n, dtype=torch.float64, device=DEV),
                  level=7)
    with pytest.raises(p.PmgError):  # FP32 on an FP64 context
        ctx.apply(torch.zeros(n, dtype=torch.float32, device=DEV), torch.zeros(n, dtype=torch.float32, device=DEV),
                  prec=p.FP32)
    with pytest.raises(p.PmgError):  # smoothing on the coarsest level
        ctx.smooth(torch.zeros(ctx.num_dofs(0), dtype=torch.float64, device=DEV),
                   torch.zeros(ctx.num_dofs(0), dtype=torch.float64, device=DEV), level=0)


def test_caller_workspace_too_small_is_oom():
    import ctypes
    lib = p.load_library()
    cfg = p.make_config(dim=2, n_cells=8, degree=2)
    need = p.bytes_required(cfg)
    ws = torch.empty(need // 2, dtype=torch.uint8, device=DEV)
    h = ctypes.c_void_p()
    rc = lib.pmg_create(ctypes.byref(cfg), None, ctypes.c_void_p(ws.data_ptr()), need // 2, ctypes.byref(h))
    assert rc == p.PMG_ERR_OOM


def test_determinism_bitwise():
    ctx = make_ctx(3, 8, 3)
    b = to_dev(random_vector(3, 8, 3, seed=8))
    x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
    ctx.solve(b, x1)
    ctx.solve(b, x2)
    assert torch.equal(x1, x2)


# ------------------------------------------------------------------ full size
def _sampled_apply_rows(m, x, rows):
    """(A x)_i for selected full-grid rows i, from the oracle's element
    matrices of the cells touching i (computed one by one)."""
    k, n, d, n1 = m.k, m.n, m.d, m.n1
    out = []
    cache = {}
    for g in rows:
        coords = [(g // n1 ** j) % n1 for j in range(d)]
        if any(c == 0 or c == n1 - 1 for c in coords):
            out.append(0.0)
            continue
        cells_per_dim = []
        for c in coords:
            cc = {min(c // k, n - 1)}
            if c % k == 0:
                cc.add(c // k - 1)
            cells_per_dim.append(sorted(x for x in cc if 0 <= x < n))
        s = 0.0
        import itertools
        for cell in itertools.product(*cells_per_dim):
            if cell not in cache:
                cache[cell] = fem.element_stiffness(m, cell)
            Ke = cache[cell]
            dofs = m.cell_dofs(cell)
            a = int(np.nonzero(dofs == g)[0][0])
            xv = x[dofs].copy()
            bnd = np.zeros(len(dofs), bool)
            for j in range(d):
                cj = (dofs // n1 ** j) % n1
                bnd |= (cj == 0) | (cj == n1 - 1)
            xv[bnd] = 0.0
            s += Ke[a] @ xv
        out.append(s)
    return np.array(out)


@pytest.mark.parametrize("prec", [p.FP64, p.FP32])
def test_full_size_3d_q4_apply_samples_and_symmetry(prec):
    # 3D, 32^3 cells, Q4 (2,146,689 DoFs), the benchmark's apply configuration
    d, n, k = 3, 32, 4
    ctx = make_ctx(d, n, k, prec=prec)
    m = fem.Mesh(d, n, k)
    N = m.n_dofs
    assert N == 2146689
    dt = torch.float64 if prec == p.FP64 else torch.float32
    x = random_vector(d, n, k, seed=61)
    y = torch.empty(N, dtype=torch.float64, device=DEV)
    ctx.apply(to_dev(x), y)                         # outer CG operator: FP64
    rows = np.random.default_rng(62).integers(0, N, 300)
    ref = _sampled_apply_rows(m, x, rows)
    got = y.cpu().numpy()[rows]
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-12 * scale * 10
    # symmetry <A u, v> = <u, A v> and positivity, in the MG precision
    u = to_dev(random_vector(d, n, k, seed=63), dt)
    v = to_dev(random_vector(d, n, k, seed=64), dt)
    Au, Av = torch.empty_like(u), torch.empty_like(v)
    ctx.apply(u, Au, prec=prec)
    ctx.apply(v, Av, prec=prec)
    a, b = float(torch.dot(Au.double(), v.double())), float(torch.dot(u.double(), Av.double()))
    tol = 1e-12 if prec == p.FP64 else 1e-5
    assert abs(a - b) <= tol * abs(a)
    assert float(torch.dot(Au.double(), u.double())) > 0


def test_full_size_3d_q4_smoother_and_vcycle_symmetry_and_solve():
    d, n, k = 3, 32, 4
    ctx = make_ctx(d, n, k)
    N = ctx.num_dofs()
    r1 = to_dev(random_vector(d, n, k, seed=71))
    r2 = to_dev(random_vector(d, n, k, seed=72))
    # smoother from a zero guess: u = S b; S is symmetric
    s1, s2 = torch.zeros_like(r1), torch.zeros_like(r2)
    ctx.smooth(r1, s1)
    ctx.smooth(r2, s2)
    a, b = float(torch.dot(s1, r2)), float(torch.dot(r1, s2))
    assert abs(a - b) <= 1e-12 * abs(a)
    z1, z2 = torch.empty_like(r1), torch.empty_like(r2)
    ctx.vcycle(r1, z1)
    ctx.vcycle(r2, z2)
    a, b = float(torch.dot(z1, r2)), float(torch.dot(r1, z2))
    assert abs(a - b) <= 1e-11 * abs(a)
    assert float(torch.dot(z1, r1)) > 0
    bm = torch.empty_like(r1)
    ctx.rhs_manufactured(bm)
    x = torch.zeros_like(bm)
    info = ctx.solve(bm, x, rtol=1e-8)
    assert info.status == 0 and info.rel_residual <= 1e-8
    Ax = torch.empty_like(x)
    ctx.apply(x, Ax)
    true_res = float(torch.linalg.norm(bm - Ax) / torch.linalg.norm(bm))
    assert true_res <= 2e-8
    err = ctx.l2_error_manufactured(x)
    assert err < 1e-6        # O(h^5) with h = 1/32


# ------------------------------------------------------------------ autotuner
@pytest.mark.parametrize("geom,prec", [("cartesian", p.FP64), ("cartesian", p.FP32), ("deformed", p.FP32)])
def test_patches_per_block_does_not_change_results(geom, prec):
    # each patch is computed by the same code whatever the block packing, so
    # every admissible value gives bitwise the same sweep
    d, n, k = 3, 8, 3
    dt = torch.float64 if prec == p.FP64 else torch.float32
    b = to_dev(random_vector(d, n, k, seed=81), dt)
    outs = []
    for ppc in (1, 3, 7):
        ctx = make_ctx(d, n, k, L=2, geom=geom, prec=prec, patches_per_block=ppc)
        assert ctx.patches_per_block() == ppc
        u = torch.zeros_like(b)
        ctx.smooth(b, u)
        outs.append(u)
        ctx.close()
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


def test_autotuned_patches_per_block_is_admissible():
    ctx = make_ctx(3, 32, 2)            # 29,791 patches: the tuner times candidates
    ppc = ctx.patches_per_block()
    assert 1 <= ppc <= 64
    b = to_dev(random_vector(3, 32, 2, seed=82))
    u = torch.zeros_like(b)
    ctx.smooth(b, u)
    ref = make_ctx(3, 32, 2, patches_per_block=1)
    u1 = torch.zeros_like(b)
    ref.smooth(b, u1)
    assert torch.equal(u, u1)


def test_vcycle_refused_above_dense_coarse_limit():
    ctx = make_ctx(3, 5, 8)                  # single level, (39)^3 coarse DoFs
    n = ctx.num_dofs()
    x = to_dev(random_vector(3, 5, 8, seed=90))
    y = torch.empty_like(x)
    ctx.apply(x, y)                          # apply works
    with pytest.raises(p.PmgError) as e:
        ctx.vcycle(x, y)
    assert e.value.code == p.PMG_ERR_UNSUPPORTED


def test_full_size_deformed_96_q3_apply_samples_and_mixed_solve():
    # 3D deformed, 96^3 cells, Q3 (24,137,569 DoFs): the deformed benchmark
    # configuration, FP32 V-cycle, FP64 CG and FP64 operator
    d, n, k = 3, 96, 3
    ctx = make_ctx(d, n, k, geom="deformed", prec=p.FP32)
    m = fem.Mesh(d, n, k, "deformed", 0.05, geom_fp32=True)
    N = m.n_dofs
    assert N == 24137569
    x = random_vector(d, n, k, seed=91)
    y = torch.empty(N, dtype=torch.float64, device=DEV)
    ctx.apply(to_dev(x), y)
    rows = np.random.default_rng(92).integers(0, N, 60)
    ref = _sampled_apply_rows(m, x, rows)
    got = y.cpu().numpy()[rows]
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()
    b = torch.empty_like(y)
    ctx.rhs_manufactured(b)
    xs = torch.zeros_like(b)
    info = ctx.solve(b, xs)
    assert info.status == 0 and info.rel_residual <= 1e-8
    Ax = torch.empty_like(xs)
    ctx.apply(xs, Ax)
    assert float(torch.linalg.norm(b - Ax) / torch.linalg.norm(b)) <= 2e-8
    assert ctx.l2_error_manufactured(xs) < 1e-7


def test_full_size_k8_apply_samples():
    # degree 8 at 25^3 cells (8,120,601 DoFs), FP64 and FP32 operators
    d, n, k = 3, 25, 8
    ctx = make_ctx(d, n, k, L=1, prec=p.FP32)
    m = fem.Mesh(d, n, k)
    x = random_vector(d, n, k, seed=93)
    rows = np.random.default_rng(94).integers(0, m.n_dofs, 40)
    ref = _sampled_apply_rows(m, x, rows)
    y = torch.empty(m.n_dofs, dtype=torch.float64, device=DEV)
    ctx.apply(to_dev(x), y)
    assert np.abs(y.cpu().numpy()[rows] - ref).max() <= 1e-11 * np.abs(ref).max()
    y32 = torch.empty(m.n_dofs, dtype=torch.float32, device=DEV)
    ctx.apply(to_dev(x, torch.float32), y32, prec=p.FP32)
    assert np.abs(y32.cpu().double().numpy()[rows] - ref).max() <= 2e-5 * np.abs(ref).max()


@pytest.mark.parametrize("n,k", [(23, 3), (13, 5), (9, 8)])
def test_fp32_apply_across_tiles_and_ragged_tail(n, k):
    # The FP32 3D apply forms its x and y passes on tiles of 32 / k cells per
    # side of one z plane: these meshes span several tiles with a partial last
    # one.  Rows on the tile seams (every 32 / k cells), on the last partial
    # tile and random rows, against the oracle's element matrices.
    d = 3
    ctx = make_ctx(d, n, k, prec=p.FP32)
    m = fem.Mesh(d, n, k)
    N = m.n_dofs
    x = random_vector(d, n, k, seed=91)
    y = torch.empty(N, dtype=torch.float32, device=DEV)
    ctx.apply(to_dev(x, torch.float32), y, prec=p.FP32)
    n1, cx = m.n1, max(1, 32 // k)
    seams = sorted({min(n1 - 1, max(0, k * c + a)) for c in range(0, n + 1, cx) for a in (-1, 0, 1)} | {n1 - 2, n1 - 1})
    rng = np.random.default_rng(92)
    rows = [int(xx + n1 * (yy + n1 * zz)) for xx in seams for yy in seams for zz in rng.choice(n1, 2)]
    rows += list(rng.integers(0, N, 200))
    ref = _sampled_apply_rows(m, x.astype(np.float32).astype(np.float64), rows)
    got = y.cpu().numpy().astype(np.float64)[rows]
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 2e-5 * scale


@pytest.mark.parametrize("n", [49, 52])
def test_deformed_fast_apply_whole_lines(n):
    # The FP32 and the float-float deformed apply (half-warp per cell, eight
    # parity launches adding into y) on odd and even n: whole x-lines of a
    # few (y, z) -- every node of a line, shared or not -- and random rows,
    # against the oracle's element matrices on the same FP32-stored geometry.
    d, k = 3, 3
    m = fem.Mesh(d, n, k, "deformed", 0.05, geom_fp32=True)
    N, n1 = m.n_dofs, m.n1
    x = random_vector(d, n, k, seed=93)
    rng = np.random.default_rng(94)
    rows = [int(xx + n1 * (yy + n1 * zz)) for yy, zz in ((1, 1), (3, 4), (n1 // 2, n1 - 2), (6, 3 * (n // 2)))
            for xx in range(n1)]
    rows += list(rng.integers(0, N, 100))
    ref = _sampled_apply_rows(m, x, rows)
    scale = np.abs(ref).max()
    ctx = make_ctx(d, n, k, geom="deformed", prec=p.FP32)
    y32 = torch.empty(N, dtype=torch.float32, device=DEV)
    ctx.apply(to_dev(x, torch.float32), y32, prec=p.FP32)
    ref32 = _sampled_apply_rows(m, x.astype(np.float32).astype(np.float64), rows)
    assert np.abs(y32.cpu().numpy().astype(np.float64)[rows] - ref32).max() <= 2e-5 * scale
    ctx.close()
    ctx = make_ctx(d, n, k, geom="deformed", prec=p.FP32, outer_apply=p.APPLY_FLOAT_FLOAT)
    y = torch.empty(N, dtype=torch.float64, device=DEV)
    ctx.apply(to_dev(x), y)
    assert np.abs(y.cpu().numpy()[rows] - ref).max() <= 1e-11 * scale
