"""Half local V-cycle (§3.2.2) and the flexible GMRES outer solver: CUDA
path vs the CPU oracle, through the C ABI.

Tolerances as in test_gpu_parity: FP64 sweep / V-cycle 1e-11 relative,
FP32 2e-5; solves reach ||b - A x|| / ||b|| <= 2e-8 with GMRES iteration
counts within +-1 of the oracle's (FP64; the GPU orthogonalises with two
classical Gram-Schmidt passes, the oracle with modified Gram-Schmidt).
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
from tests.test_gpu_parity import DEV, full, make_ctx, n_levels_auto, rel, to_dev

pytestmark = pytest.mark.gpu


@functools.lru_cache(maxsize=None)
def half_level(d, n, k, geom, n_iter=1):
    m = fem.Mesh(d, n, k, geom, 0.05, geom_fp32=True)
    return solver.Level(m, constants.omega_jacobi(d, k), constants.omega_patch(d), n_iter=n_iter,
                        full_vcycle=False)


@functools.lru_cache(maxsize=None)
def hier(d, n, k, L, geom, full_vcycle):
    m = fem.Mesh(d, n, k, geom, 0.05, geom_fp32=True)
    return solver.Hierarchy(m, L, constants.omega_jacobi(d, k), constants.omega_patch(d),
                            full_vcycle=full_vcycle)


@pytest.mark.parametrize("d,n,k,geom", [(2, 8, 3, "cartesian"), (2, 4, 7, "cartesian"), (3, 4, 3, "cartesian"),
                                        (3, 2, 8, "cartesian"), (2, 6, 3, "deformed"), (3, 4, 3, "deformed")])
def test_half_vcycle_smoother_sweep_fp64(d, n, k, geom):
    ctx = make_ctx(d, n, k, L=2 if n % 2 == 0 else 1, geom=geom, local_half=1)
    lev = half_level(d, n, k, geom)
    b = random_vector(d, n, k, seed=61)
    u0 = random_vector(d, n, k, seed=62)
    u = to_dev(u0)
    ctx.smooth(to_dev(b), u, sweeps=2)
    ref = lev.smooth(b[lev.I], u0[lev.I], sweeps=2)
    assert rel(u.cpu().numpy(), full(lev, ref)) < 1e-11


@pytest.mark.parametrize("d,n,k,geom", [(3, 4, 3, "cartesian"), (3, 4, 2, "deformed")])
def test_half_vcycle_smoother_sweep_fp32_and_two_cycles(d, n, k, geom):
    ctx = make_ctx(d, n, k, L=2, geom=geom, prec=p.FP32, local_half=1)
    lev = half_level(d, n, k, geom)
    b = random_vector(d, n, k, seed=63)
    u = torch.zeros(lev.mesh.n_dofs, dtype=torch.float32, device=DEV)
    ctx.smooth(to_dev(b, torch.float32), u, sweeps=1)
    ref = lev.smooth(b[lev.I], np.zeros(len(lev.I)), sweeps=1)
    assert rel(u.cpu().double().numpy(), full(lev, ref)) < 2e-5
    # "2 half V-cycles" (Algorithm 2 with N_iter = 2 around the half cycle)
    ctx2 = make_ctx(d, n, k, L=2, geom=geom, local_half=1, local_cycles=2)
    lev2 = half_level(d, n, k, geom, n_iter=2)
    u2 = torch.zeros(lev.mesh.n_dofs, dtype=torch.float64, device=DEV)
    ctx2.smooth(to_dev(b), u2)
    ref2 = lev2.smooth(b[lev2.I], np.zeros(len(lev2.I)))
    assert rel(u2.cpu().numpy(), full(lev2, ref2)) < 1e-11


@pytest.mark.parametrize("d,n,k,L,geom", [(2, 16, 2, 3, "cartesian"), (3, 4, 3, 0, "cartesian"),
                                          (3, 4, 2, 0, "deformed")])
def test_half_vcycle_preconditioner(d, n, k, L, geom):
    ctx = make_ctx(d, n, k, L=L, geom=geom, local_half=1)
    h = hier(d, n, k, L if L else n_levels_auto(n), geom, False)
    fine = h.levels[-1]
    r = random_vector(d, n, k, seed=64)
    z = torch.empty(fine.mesh.n_dofs, dtype=torch.float64, device=DEV)
    ctx.vcycle(to_dev(r), z)
    assert rel(z.cpu().numpy(), full(fine, h.vcycle(r[fine.I]))) < 1e-11


GMRES_CASES = [(2, 16, 3, 3, "cartesian", 0), (2, 16, 3, 3, "cartesian", 1), (3, 8, 2, 0, "cartesian", 1),
               (3, 4, 4, 0, "cartesian", 0), (3, 4, 4, 0, "cartesian", 1), (2, 8, 3, 0, "deformed", 1),
               (3, 4, 3, 0, "deformed", 1)]


@pytest.mark.parametrize("d,n,k,L,geom,half", GMRES_CASES)
@pytest.mark.parametrize("prec", [p.FP64, p.FP32])
def test_gmres_solve(d, n, k, L, geom, half, prec):
    ctx = make_ctx(d, n, k, L=L, geom=geom, prec=prec, local_half=half, outer_solver=p.OUTER_GMRES)
    h = hier(d, n, k, L if L else n_levels_auto(n), geom, not half)
    fine = h.levels[-1]
    b_ref = fem.rhs_manufactured(fine.mesh)
    b = to_dev(b_ref)
    x = torch.zeros_like(b)
    info = ctx.solve(b, x, rtol=1e-8)
    x_ref, it_ref, _ = solver.solve(h, b_ref[fine.I], rtol=1e-8, outer="gmres")
    assert info.status == 0 and info.rel_residual <= 1e-8
    xh = x.cpu().numpy()
    true_res = np.linalg.norm(b_ref[fine.I] - fine.A @ xh[fine.I]) / np.linalg.norm(b_ref[fine.I])
    assert true_res <= 2e-8
    if prec == p.FP64:
        assert abs(info.iterations - it_ref) <= 1, (info.iterations, it_ref)
        assert rel(xh, full(fine, x_ref)) < 1e-6
    else:
        assert info.iterations <= it_ref + 3, (info.iterations, it_ref)
        assert rel(xh, full(fine, x_ref)) < 1e-5


def test_gmres_restarts_match_oracle():
    # restart length 2 forces several cycles, each restarted from b - A x
    d, n, k, L = 2, 16, 3, 3
    ctx = make_ctx(d, n, k, L=L, local_half=1, outer_solver=p.OUTER_GMRES, gmres_restart=2)
    h = hier(d, n, k, L, "cartesian", False)
    fine = h.levels[-1]
    b_ref = random_vector(d, n, k, seed=65)
    x = torch.zeros(fine.mesh.n_dofs, dtype=torch.float64, device=DEV)
    info = ctx.solve(to_dev(b_ref), x, rtol=1e-8, maxit=200)
    x_ref, it_ref, _ = solver.gmres(fine.A, b_ref[fine.I], h.vcycle, rtol=1e-8, maxit=200, restart=2)
    assert info.status == 0
    assert abs(info.iterations - it_ref) <= 1, (info.iterations, it_ref)
    xh = x.cpu().numpy()
    assert np.linalg.norm(b_ref[fine.I] - fine.A @ xh[fine.I]) <= 2e-8 * np.linalg.norm(b_ref[fine.I])


def test_half_vcycle_costs_a_few_more_iterations_than_full():
    # §3.2.2 / Table 1 (soft): the half cycle needs at most a few more outer
    # GMRES iterations than the full cycle
    its = {}
    for half in (0, 1):
        ctx = make_ctx(3, 8, 3, local_half=half, outer_solver=p.OUTER_GMRES)
        b = torch.empty(ctx.num_dofs(), dtype=torch.float64, device=DEV)
        ctx.rhs_manufactured(b)
        x = torch.zeros_like(b)
        its[half] = ctx.solve(b, x, rtol=1e-8).iterations
    assert its[0] <= its[1] <= its[0] + 4, its


def test_gmres_deterministic_zero_rhs_and_maxit():
    ctx = make_ctx(3, 4, 3, local_half=1, outer_solver=p.OUTER_GMRES)
    b = torch.empty(ctx.num_dofs(), dtype=torch.float64, device=DEV)
    ctx.rhs_manufactured(b)
    x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
    i1, i2 = ctx.solve(b, x1), ctx.solve(b, x2)
    assert i1.iterations == i2.iterations and torch.equal(x1, x2)
    z = torch.zeros_like(b)
    x = torch.ones_like(b)
    info = ctx.solve(z, x)
    assert info.iterations == 0 and float(x.abs().max()) == 0.0
    info = ctx.solve(b, x, rtol=1e-14, maxit=2)
    assert info.status == p.PMG_NOT_CONVERGED and info.iterations == 2


def test_gmres_through_the_server_matches_direct_solve():
    cfg = p.make_config(dim=3, n_cells=8, degree=3, mg_precision=p.FP32, local_half=1)
    ctx = p.Context(cfg, device=DEV)
    b = torch.empty(ctx.num_dofs(), dtype=torch.float64, device=DEV)
    ctx.rhs_manufactured(b)
    x = torch.zeros_like(b)
    info = ctx.solve(b, x)
    srv = p.Server(0, 2)
    bh = b.cpu().pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    rid = srv.submit(cfg, bh, xh)
    while srv.result(rid)["state"] < 2:
        srv.poll()
    res = srv.result(rid)
    assert res["state"] == 2 and res["iterations"] == info.iterations
    assert torch.equal(xh, x.cpu())
    srv.close()


def test_gmres_restart_one_matches_oracle():
    # GMRES(1): one minimal-residual step per cycle, restarted from b - A x
    d, n, k, L = 2, 8, 2, 3
    ctx = make_ctx(d, n, k, L=L, outer_solver=p.OUTER_GMRES, gmres_restart=1)
    h = hier(d, n, k, L, "cartesian", True)
    fine = h.levels[-1]
    b_ref = random_vector(d, n, k, seed=66)
    x = torch.zeros(fine.mesh.n_dofs, dtype=torch.float64, device=DEV)
    info = ctx.solve(to_dev(b_ref), x, rtol=1e-8, maxit=300)
    x_ref, it_ref, _ = solver.gmres(fine.A, b_ref[fine.I], h.vcycle, rtol=1e-8, maxit=300, restart=1)
    assert info.status == 0
    assert abs(info.iterations - it_ref) <= 1, (info.iterations, it_ref)
    assert rel(x.cpu().numpy(), full(fine, x_ref)) < 1e-6
