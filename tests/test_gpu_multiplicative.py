"""Multiplicative vertex-patch smoother (Algorithm 1, colour by colour over
the 2^d vertex-parity colours): CUDA path vs the CPU oracle, through the C
ABI.  Tolerances as in test_gpu_parity (FP64 sweep / V-cycle 1e-11
relative, FP32 2e-5; solves to ||b - A x|| / ||b|| <= 2e-8 with iteration
counts within +-1 of the oracle's)."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2512_02577_gb300 as p
from oracle import constants, fem, solver
from paper_2512_02577_gb300.inputs import random_vector
from tests.test_gpu_parity import DEV, full, make_ctx, n_levels_auto, rel, to_dev

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def mult_level(d, n, k, geom, half=False):
    m = fem.Mesh(d, n, k, geom, 0.05, geom_fp32=True)
    return solver.Level(m, constants.omega_jacobi(d, k), constants.omega_patch(d), full_vcycle=not half,
                        multiplicative=True)


@functools.lru_cache(maxsize=None)
def mult_hier(d, n, k, L, geom, half=False):
    m = fem.Mesh(d, n, k, geom, 0.05, geom_fp32=True)
    return solver.Hierarchy(m, L, constants.omega_jacobi(d, k), constants.omega_patch(d), full_vcycle=not half,
                            multiplicative=True)


# n = 6, 10: the parity colours hold different numbers of patches (3 odd and
# 2 even vertex indices per direction at n = 6); n = 2: a single patch
SWEEP_CASES = [(2, 8, 3, "cartesian"), (2, 10, 2, "cartesian"), (2, 2, 5, "cartesian"), (3, 4, 3, "cartesian"),
               (3, 6, 2, "cartesian"), (3, 2, 4, "cartesian"), (3, 4, 1, "cartesian"), (2, 6, 3, "deformed"),
               (3, 4, 2, "deformed"), (3, 6, 2, "deformed")]


@pytest.mark.parametrize("d,n,k,geom", SWEEP_CASES)
def test_multiplicative_sweep_fp64(d, n, k, geom):
    ctx = make_ctx(d, n, k, L=2, geom=geom, smoother=p.MULTIPLICATIVE)
    lev = mult_level(d, n, k, geom)
    b = random_vector(d, n, k, seed=71)
    u0 = random_vector(d, n, k, seed=72)
    u = to_dev(u0)
    ctx.smooth(to_dev(b), u, sweeps=2)
    ref = lev.smooth(b[lev.I], u0[lev.I], sweeps=2)
    assert rel(u.cpu().numpy(), full(lev, ref)) < 1e-11


@pytest.mark.parametrize("d,n,k,geom", [(3, 4, 3, "cartesian"), (3, 4, 2, "deformed")])
def test_multiplicative_sweep_fp32_and_half_cycle(d, n, k, geom):
    ctx = make_ctx(d, n, k, L=2, geom=geom, prec=p.FP32, smoother=p.MULTIPLICATIVE)
    lev = mult_level(d, n, k, geom)
    b = random_vector(d, n, k, seed=73)
    u = torch.zeros(lev.mesh.n_dofs, dtype=torch.float32, device=DEV)
    ctx.smooth(to_dev(b, torch.float32), u, sweeps=1)
    ref = lev.smooth(b[lev.I], np.zeros(len(lev.I)), sweeps=1)
    assert rel(u.cpu().double().numpy(), full(lev, ref)) < 2e-5
    ctx_h = make_ctx(d, n, k, L=2, geom=geom, smoother=p.MULTIPLICATIVE, local_half=1)
    lev_h = mult_level(d, n, k, geom, half=True)
    uh = torch.zeros(lev.mesh.n_dofs, dtype=torch.float64, device=DEV)
    ctx_h.smooth(to_dev(b), uh)
    ref_h = lev_h.smooth(b[lev_h.I], np.zeros(len(lev_h.I)))
    assert rel(uh.cpu().numpy(), full(lev_h, ref_h)) < 1e-11


@pytest.mark.parametrize("d,n,k,L,geom", [(2, 16, 2, 3, "cartesian"), (3, 4, 3, 0, "cartesian"),
                                          (3, 6, 2, 2, "cartesian"), (3, 4, 2, 0, "deformed")])
def test_multiplicative_vcycle_and_symmetry(d, n, k, L, geom):
    ctx = make_ctx(d, n, k, L=L, geom=geom, smoother=p.MULTIPLICATIVE)
    h = mult_hier(d, n, k, L if L else n_levels_auto(n), geom)
    fine = h.levels[-1]
    r = random_vector(d, n, k, seed=74)
    s = random_vector(d, n, k, seed=75)
    z = torch.empty(fine.mesh.n_dofs, dtype=torch.float64, device=DEV)
    w = torch.empty_like(z)
    ctx.vcycle(to_dev(r), z)
    ctx.vcycle(to_dev(s), w)
    assert rel(z.cpu().numpy(), full(fine, h.vcycle(r[fine.I]))) < 1e-11
    # forward pre- and backward post-smoothing: <B r, s> = <r, B s>
    a, b = float(z.cpu().numpy() @ s), float(r @ w.cpu().numpy())
    assert abs(a - b) <= 1e-11 * max(abs(a), abs(b))


@pytest.mark.parametrize("d,n,k,L,geom,half", [(2, 16, 3, 3, "cartesian", 0), (3, 8, 2, 0, "cartesian", 0),
                                               (3, 8, 2, 0, "cartesian", 1), (3, 4, 3, 0, "deformed", 0),
                                               (3, 4, 3, 0, "deformed", 1)])
@pytest.mark.parametrize("prec", [p.FP64, p.FP32])
def test_multiplicative_solve(d, n, k, L, geom, half, prec):
    outer = p.OUTER_GMRES if half else p.OUTER_CG
    ctx = make_ctx(d, n, k, L=L, geom=geom, prec=prec, smoother=p.MULTIPLICATIVE, local_half=half,
                   outer_solver=outer)
    h = mult_hier(d, n, k, L if L else n_levels_auto(n), geom, half=bool(half))
    fine = h.levels[-1]
    b_ref = fem.rhs_manufactured(fine.mesh)
    x = torch.zeros(fine.mesh.n_dofs, dtype=torch.float64, device=DEV)
    info = ctx.solve(to_dev(b_ref), x, rtol=1e-8)
    x_ref, it_ref, _ = solver.solve(h, b_ref[fine.I], rtol=1e-8, outer="gmres" if half else "cg")
    assert info.status == 0 and info.rel_residual <= 1e-8
    xh = x.cpu().numpy()
    assert np.linalg.norm(b_ref[fine.I] - fine.A @ xh[fine.I]) <= 2e-8 * np.linalg.norm(b_ref[fine.I])
    if prec == p.FP64:
        assert abs(info.iterations - it_ref) <= 1, (info.iterations, it_ref)
        assert rel(xh, full(fine, x_ref)) < 1e-6
    else:
        assert info.iterations <= it_ref + 3, (info.iterations, it_ref)


def test_multiplicative_needs_fewer_iterations_than_additive():
    its = {}
    for sm in (p.ADDITIVE, p.MULTIPLICATIVE):
        ctx = make_ctx(3, 16, 3, smoother=sm)
        b = torch.empty(ctx.num_dofs(), dtype=torch.float64, device=DEV)
        ctx.rhs_manufactured(b)
        x = torch.zeros_like(b)
        its[sm] = ctx.solve(b, x).iterations
    assert its[p.MULTIPLICATIVE] < its[p.ADDITIVE], its


def test_multiplicative_two_half_cycles_and_deformed_2d_vcycle():
    # N_iter = 2 around the half local cycle inside the multiplicative sweep
    d, n, k = 3, 4, 3
    ctx = make_ctx(d, n, k, L=2, smoother=p.MULTIPLICATIVE, local_half=1, local_cycles=2)
    m = fem.Mesh(d, n, k, "cartesian", 0.05, geom_fp32=True)
    lev = solver.Level(m, constants.omega_jacobi(d, k), constants.omega_patch(d), n_iter=2, full_vcycle=False,
                       multiplicative=True)
    b = random_vector(d, n, k, seed=76)
    u = torch.zeros(m.n_dofs, dtype=torch.float64, device=DEV)
    ctx.smooth(to_dev(b), u)
    assert rel(u.cpu().numpy(), full(lev, lev.smooth(b[lev.I], np.zeros(len(lev.I))))) < 1e-11
    # 2D deformed V-cycle
    ctx2 = make_ctx(2, 8, 3, L=0, geom="deformed", smoother=p.MULTIPLICATIVE)
    h = mult_hier(2, 8, 3, n_levels_auto(8), "deformed")
    fine = h.levels[-1]
    r = random_vector(2, 8, 3, seed=77)
    z = torch.empty(fine.mesh.n_dofs, dtype=torch.float64, device=DEV)
    ctx2.vcycle(to_dev(r), z)
    assert rel(z.cpu().numpy(), full(fine, h.vcycle(r[fine.I]))) < 1e-11
