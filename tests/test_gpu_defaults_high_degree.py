"""Parity of what the benchmark and the server actually run, through the C ABI.

1. Default damping.  The benchmark, the server and the Table 1 runs build
   their contexts without damping values, so the library resolves omega_J
   (Lanczos on the Cartesian patch) and omega_AS itself.  These tests build
   contexts that way and compare (a) the resolved values with the oracle's
   readings and (b) sweeps and V-cycles with the oracle built from its own
   constants (§2.2, §3.2 leave omega open; the reading is the same on both
   sides, the computation of lambda_max is not).
2. High degrees in 3D on overlapping patches.  The served stream draws k up
   to 7 and the degree sweep runs k = 8; their patch kernels are separate
   template instances (no launch bounds above k = 4, larger shared-memory
   layouts).  Sweeps and V-cycles at k = 6, 7 on n = 4 (27 patches, every
   parity colour, overlapping) and k = 8 on n = 3 (8 patches), FP64 and FP32,
   plus FP32 at the mixed headline degree k = 4 (Algorithm 2/3, §3.2).

Tolerances as in test_gpu_parity: FP64 sweep / V-cycle 1e-11, FP32 2e-5 of
the oracle's FP64 (norm-relative and element-wise, tests/parity.py).
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
from tests.parity import rel
from tests.test_gpu_parity import DEV, full, n_levels_auto, oracle_level, to_dev

pytestmark = pytest.mark.gpu


def ctx_default(d, n, k, L=0, prec=p.FP64, **kw):
    """A context with the library's own damping (no omega in the config)."""
    return p.Context(p.make_config(dim=d, n_cells=n, degree=k, n_levels=L, mg_precision=prec, **kw), device=DEV)


@functools.lru_cache(maxsize=None)
def hier(d, n, k):
    """Oracle hierarchy with automatic coarsening and the oracle's damping."""
    m = fem.Mesh(d, n, k)
    return solver.Hierarchy(m, n_levels_auto(n), constants.omega_jacobi(d, k), constants.omega_patch(d))


def _tol(prec):
    return 1e-11 if prec == p.FP64 else 2e-5


# ------------------------------------------------------------ default damping
@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("k", range(1, 9))
def test_context_default_damping_is_the_oracle_reading(d, k):
    ctx = ctx_default(d, 2, k, L=1)
    wp, wj = ctx.damping()
    assert wp == constants.omega_patch(d)
    ref = constants.omega_jacobi(d, k)
    for l, w in enumerate(ref):
        assert abs(wj[l] - w) <= 1e-12 * w, (l, wj[l], w)
    # values given in the config are used as given
    cfg = p.make_config(dim=d, n_cells=2, degree=k, n_levels=1, omega_patch=0.3, omega_jacobi=[1.0, 0.7, 0.6, 0.5])
    wp2, wj2 = p.Context(cfg, device=DEV).damping()
    assert wp2 == 0.3 and wj2[1:len(ref)] == [0.7, 0.6, 0.5][:len(ref) - 1]


@pytest.mark.parametrize("d,n,k,prec", [(3, 4, 2, p.FP64), (3, 4, 4, p.FP64), (3, 4, 4, p.FP32), (3, 4, 7, p.FP64),
                                        (2, 8, 3, p.FP64), (2, 8, 3, p.FP32)])
def test_default_damping_sweep_and_vcycle_match_oracle(d, n, k, prec):
    ctx = ctx_default(d, n, k, prec=prec)
    h = hier(d, n, k)
    fine = h.levels[-1]
    dt = torch.float64 if prec == p.FP64 else torch.float32
    b = random_vector(d, n, k, seed=301)
    u0 = random_vector(d, n, k, seed=302)
    u = to_dev(u0, dt)
    ctx.smooth(to_dev(b, dt), u, sweeps=1)
    assert rel(u, full(fine, fine.smooth(b[fine.I], u0[fine.I], sweeps=1))) < _tol(prec)
    z = torch.empty(fine.mesh.n_dofs, dtype=torch.float64, device=DEV)
    ctx.vcycle(to_dev(b), z)
    assert rel(z, full(fine, h.vcycle(b[fine.I]))) < _tol(prec)


def test_default_damping_solve_matches_oracle_iterations():
    # the headline configuration's method at a size the oracle solves quickly:
    # 3D Q4, additive smoother, library damping, FP64 CG to 1e-8
    d, n, k = 3, 4, 4
    ctx = ctx_default(d, n, k)
    h = hier(d, n, k)
    fine = h.levels[-1]
    b_ref = fem.rhs_manufactured(fine.mesh)
    b = torch.empty(fine.mesh.n_dofs, dtype=torch.float64, device=DEV)
    ctx.rhs_manufactured(b)
    x = torch.zeros_like(b)
    info = ctx.solve(b, x, rtol=1e-8)
    x_ref, it_ref, _ = solver.solve(h, b_ref[fine.I], rtol=1e-8)
    assert info.status == 0 and abs(info.iterations - it_ref) <= 1, (info.iterations, it_ref)
    assert rel(x, full(fine, x_ref)) < 1e-6


# ------------------------------------------------------------ high degrees, 3D
@pytest.mark.parametrize("k", [6, 7])
@pytest.mark.parametrize("prec", [p.FP64, p.FP32])
def test_high_degree_sweep_on_overlapping_patches(k, prec):
    d, n = 3, 4                     # 27 patches, all eight parity colours
    fine = hier(d, n, k).levels[-1]
    dt = torch.float64 if prec == p.FP64 else torch.float32
    ctx = ctx_default(d, n, k, prec=prec)
    b = random_vector(d, n, k, seed=311 + k)
    u0 = random_vector(d, n, k, seed=312 + k)
    u = to_dev(u0, dt)
    ctx.smooth(to_dev(b, dt), u, sweeps=2)
    assert rel(u, full(fine, fine.smooth(b[fine.I], u0[fine.I], sweeps=2))) < _tol(prec)


@pytest.mark.parametrize("k", [6, 7])
@pytest.mark.parametrize("prec", [p.FP64, p.FP32])
def test_high_degree_vcycle(k, prec):
    d, n = 3, 4
    h = hier(d, n, k)
    fine = h.levels[-1]
    ctx = ctx_default(d, n, k, prec=prec)
    r = random_vector(d, n, k, seed=321 + k)
    z = torch.empty(fine.mesh.n_dofs, dtype=torch.float64, device=DEV)
    ctx.vcycle(to_dev(r), z)
    assert rel(z, full(fine, h.vcycle(r[fine.I]))) < _tol(prec)


@pytest.mark.parametrize("prec", [p.FP64, p.FP32])
def test_degree_8_sweep_on_overlapping_patches(prec):
    # n = 3 cannot be coarsened: the single level is smoothed (8 patches)
    d, n, k = 3, 3, 8
    lev = oracle_level(d, n, k, "cartesian")
    dt = torch.float64 if prec == p.FP64 else torch.float32
    ctx = ctx_default(d, n, k, L=1, prec=prec)
    b = random_vector(d, n, k, seed=331)
    u0 = random_vector(d, n, k, seed=332)
    u = to_dev(u0, dt)
    ctx.smooth(to_dev(b, dt), u, level=0, sweeps=1)
    assert rel(u, full(lev, lev.smooth(b[lev.I], u0[lev.I], sweeps=1))) < _tol(prec)


def test_fp32_sweep_at_the_mixed_headline_degree():
    d, n, k = 3, 4, 4
    fine = hier(d, n, k).levels[-1]
    ctx = ctx_default(d, n, k, prec=p.FP32)
    b = random_vector(d, n, k, seed=341)
    u = torch.zeros(fine.mesh.n_dofs, dtype=torch.float32, device=DEV)
    ctx.smooth(to_dev(b, torch.float32), u, sweeps=1)
    assert rel(u, full(fine, fine.smooth(b[fine.I], np.zeros(len(fine.I)), sweeps=1))) < 2e-5


# ------------------------------------------------------------ single-level smoothing
@pytest.mark.parametrize("d,n,k,geom", [(2, 5, 2, "deformed"), (3, 3, 3, "cartesian"), (3, 3, 2, "deformed")])
def test_single_level_context_smooths_its_level(d, n, k, geom):
    # odd n gives one level; its patches are smoothed (degree sweep at odd n)
    cfg = p.make_config(dim=d, n_cells=n, degree=k, n_levels=1,
                        geometry=p.DEFORMED if geom == "deformed" else p.CARTESIAN)
    ctx = p.Context(cfg, device=DEV)
    lev = oracle_level(d, n, k, geom)
    b = random_vector(d, n, k, seed=351)
    u = torch.zeros(lev.mesh.n_dofs, dtype=torch.float64, device=DEV)
    ctx.smooth(to_dev(b), u, level=0)
    assert rel(u, full(lev, lev.smooth(b[lev.I], np.zeros(len(lev.I))))) < 1e-11
    assert all(t > 0 for t in ctx.smoother_phase_times(level=0, reps=1))


def test_coarsest_level_smoothing_rules():
    # Cartesian coarsest level with patches: smoothable; deformed: no data
    ctx = p.Context(p.make_config(dim=3, n_cells=6, degree=2), device=DEV)      # levels n = 3, 6
    b = to_dev(random_vector(3, 3, 2, seed=361))
    u = torch.zeros_like(b)
    ctx.smooth(b, u, level=0)
    assert float(torch.linalg.norm(u)) > 0
    dctx = p.Context(p.make_config(dim=3, n_cells=6, degree=2, geometry=p.DEFORMED), device=DEV)
    with pytest.raises(p.PmgError):
        dctx.smooth(b, u, level=0)


# ------------------------------------------------------------ interleaved patch layout
@pytest.mark.parametrize("d,n,k,prec", [(3, 4, 2, p.FP32), (3, 4, 4, p.FP32), (3, 4, 4, p.FP64), (3, 4, 6, p.FP32),
                                        (3, 4, 7, p.FP32), (3, 3, 8, p.FP32), (2, 8, 3, p.FP32), (2, 8, 5, p.FP64)])
def test_interleaved_layout_sweep_and_vcycle_match_oracle(d, n, k, prec):
    # the interleaved shared-memory layout forced on every level
    L = 1 if n % 2 else 0
    ctx = ctx_default(d, n, k, L=L, prec=prec, patch_layout=p.PATCH_INTERLEAVED, patch_threads=256)
    lay, ppc, thr = ctx.patch_layout()
    assert lay == p.PATCH_INTERLEAVED and thr == 256 and ppc in (2, 4, 8, 16)
    dt = torch.float64 if prec == p.FP64 else torch.float32
    if L == 1:
        fine, h = oracle_level(d, n, k, "cartesian"), None
    else:
        h = hier(d, n, k)
        fine = h.levels[-1]
    b = random_vector(d, n, k, seed=371 + k)
    u0 = random_vector(d, n, k, seed=372 + k)
    u = to_dev(u0, dt)
    ctx.smooth(to_dev(b, dt), u, level=-1, sweeps=1)
    assert rel(u, full(fine, fine.smooth(b[fine.I], u0[fine.I], sweeps=1))) < _tol(prec)
    if h is not None:
        z = torch.empty(fine.mesh.n_dofs, dtype=torch.float64, device=DEV)
        ctx.vcycle(to_dev(b), z)
        assert rel(z, full(fine, h.vcycle(b[fine.I]))) < _tol(prec)


@pytest.mark.parametrize("k,prec", [(2, p.FP32), (3, p.FP32), (4, p.FP32), (4, p.FP64), (5, p.FP32), (7, p.FP32)])
def test_interleaved_and_patch_major_layouts_are_bitwise_equal(k, prec):
    # same per-patch arithmetic in both layouts: identical sweeps, V-cycles
    # and multiplicative colour sweeps, at every admissible block shape
    d, n = 3, 16 if k <= 4 else 8
    dt = torch.float64 if prec == p.FP64 else torch.float32
    b = to_dev(random_vector(d, n, k, seed=381), dt)
    r = to_dev(random_vector(d, n, k, seed=382))
    outs = []
    for lay, ppc, thr in ((p.PATCH_MAJOR, 1, 0), (p.PATCH_MAJOR, 3, 0), (p.PATCH_INTERLEAVED, 0, 128),
                          (p.PATCH_INTERLEAVED, 0, 416), (p.PATCH_INTERLEAVED, 0, 768)):
        for sm in (p.ADDITIVE, p.MULTIPLICATIVE):
            try:
                ctx = ctx_default(d, n, k, prec=prec, patch_layout=lay, patches_per_block=ppc, patch_threads=thr,
                                  smoother=sm)
            except p.PmgError as e:             # block shape above the kernel's limit
                assert e.code == p.PMG_ERR_ARG and thr > 0
                continue
            u = torch.zeros_like(b)
            ctx.smooth(b, u)
            z = torch.empty_like(r)
            ctx.vcycle(r, z)
            outs.append((sm, u, z))
            ctx.close()
    for sm in (p.ADDITIVE, p.MULTIPLICATIVE):
        got = [(u, z) for s, u, z in outs if s == sm]
        assert len(got) >= 3
        for u, z in got[1:]:
            assert torch.equal(u, got[0][0]) and torch.equal(z, got[0][1])


def test_autotuner_considers_the_interleaved_layout():
    ctx = ctx_default(3, 32, 4, prec=p.FP32)       # 29,791 patches: timed
    lay, ppc, thr = ctx.patch_layout()
    assert lay in (p.PATCH_MAJOR, p.PATCH_INTERLEAVED) and ppc >= 1 and thr % 32 == 0
    with pytest.raises(p.PmgError):                 # no interleaved layout for deformed meshes
        ctx_default(3, 4, 2, geometry=p.DEFORMED, patch_layout=p.PATCH_INTERLEAVED)


# ------------------------------------------------------------ deformed apply block shape
@pytest.mark.parametrize("k,prec,cands", [(3, p.FP32, (4, 8, 16)), (2, p.FP32, (4, 16)), (3, p.FP64, (1, 4, 16)),
                                          (4, p.FP32, (1, 2, 8))])
def test_deformed_apply_block_shapes_are_bitwise_equal(k, prec, cands):
    # cells per block change the packing of cells into blocks, not the
    # arithmetic of a cell: every admissible value gives the same bits
    d, n = 3, 6
    dt = torch.float64 if prec == p.FP64 else torch.float32
    x = to_dev(random_vector(d, n, k, seed=391), dt)
    outs = []
    for cpb in cands:
        ctx = p.Context(p.make_config(dim=d, n_cells=n, degree=k, n_levels=1, geometry=p.DEFORMED, mg_precision=prec,
                                      apply_cells_per_block=cpb), device=DEV)
        assert ctx.apply_cells_per_block() == cpb
        y = torch.empty_like(x)
        ctx.apply(x, y, prec=prec)
        outs.append(y)
        ctx.close()
    assert all(torch.equal(o, outs[0]) for o in outs[1:])


def test_deformed_apply_block_shape_is_tuned():
    ctx = p.Context(p.make_config(dim=3, n_cells=32, degree=3, geometry=p.DEFORMED, mg_precision=p.FP32),
                    device=DEV)
    assert ctx.apply_cells_per_block() in (4, 8, 16)
    with pytest.raises(p.PmgError):
        p.Context(p.make_config(dim=3, n_cells=4, degree=3, geometry=p.DEFORMED, mg_precision=p.FP32,
                                apply_cells_per_block=5), device=DEV)


def test_cached_coarse_inverse_serves_a_second_hierarchy():
    # n = 6 and n = 12 at k = 2 share the coarse mesh n_0 = 3: the second
    # context takes the first one's coarse inverse from the process cache;
    # both V-cycles match the oracle
    d, k = 3, 2
    for n in (6, 12):
        ctx = ctx_default(d, n, k)
        h = hier(d, n, k)
        fine = h.levels[-1]
        r = random_vector(d, n, k, seed=400 + n)
        z = torch.empty(fine.mesh.n_dofs, dtype=torch.float64, device=DEV)
        ctx.vcycle(to_dev(r), z)
        assert rel(z, full(fine, h.vcycle(r[fine.I]))) < 1e-11
        ctx.close()


@pytest.mark.parametrize("k,prec,lay", [(4, p.FP32, p.PATCH_MAJOR), (4, p.FP64, p.PATCH_MAJOR),
                                        (7, p.FP32, p.PATCH_MAJOR), (3, p.FP32, p.PATCH_INTERLEAVED)])
def test_persistent_patch_launches_are_bitwise_equal(k, prec, lay):
    # persistent grids take batches of patches from a counter; every patch is
    # computed by the same code and written to the same place
    d, n = 3, 32 if k <= 4 else 16
    dt = torch.float64 if prec == p.FP64 else torch.float32
    b = to_dev(random_vector(d, n, k, seed=395), dt)
    outs = []
    for pers in (-1, 1):
        for sm in (p.ADDITIVE, p.MULTIPLICATIVE):
            kw = dict(patches_per_block=2) if lay == p.PATCH_MAJOR else dict(patch_threads=256)
            ctx = ctx_default(d, n, k, prec=prec, patch_layout=lay, patch_persistent=pers, smoother=sm, **kw)
            assert ctx.patch_persistent() == (pers > 0)
            u = torch.zeros_like(b)
            ctx.smooth(b, u, sweeps=2)
            outs.append((sm, u))
            ctx.close()
    for sm in (p.ADDITIVE, p.MULTIPLICATIVE):
        got = [u for s_, u in outs if s_ == sm]
        assert torch.equal(got[0], got[1])


@pytest.mark.parametrize("cd,levels", [(0, 6), (4096, 4), (3375, 4), (3374, 5), (343, 5), (27, 6)])
def test_coarse_dofs_levels(cd, levels):
    ctx = ctx_default(3, 32, 4, prec=p.FP32, coarse_dofs=cd)
    assert ctx.n_levels == levels
    ctx.close()


def test_coarse_dofs_solve_matches_the_oracle_hierarchy():
    # 2D 32^2 Q3 stopped at 4^2 cells (11^2 = 121 free DoFs <= 128): the same
    # solve as the oracle's 4-level hierarchy with the same damping
    d, n, k = 2, 32, 3
    wj, wp = constants.omega_jacobi(d, k), constants.omega_patch(d)
    ctx = p.Context(p.make_config(dim=d, n_cells=n, degree=k, coarse_dofs=128, omega_jacobi=wj, omega_patch=wp),
                    device=DEV)
    assert ctx.n_levels == 4
    m = fem.Mesh(d, n, k)
    h = solver.Hierarchy(m, 4, wj, wp)
    fine = h.levels[-1]
    b_ref = fem.rhs_manufactured(m)
    b = torch.empty(m.n_dofs, dtype=torch.float64, device=DEV)
    ctx.rhs_manufactured(b)
    x = torch.zeros_like(b)
    info = ctx.solve(b, x, rtol=1e-8)
    x_ref, it_ref, _ = solver.solve(h, b_ref[fine.I], rtol=1e-8)
    assert abs(info.iterations - it_ref) <= 1
    xf = np.zeros(m.n_dofs)
    xf[fine.I] = x_ref
    assert np.abs(x.cpu().numpy() - xf).max() <= 1e-6 * np.abs(xf).max()
