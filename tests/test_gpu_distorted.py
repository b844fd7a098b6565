"""Randomly distorted meshes (§3.2.2, §4): every interior vertex of the
finest mesh moved by delta h in a random direction, trilinear cells, the
general stored-G_q operator.  CUDA path vs the CPU oracle through the C ABI;
tolerances as in test_gpu_parity (the FP32-stored G_q is the discrete
operator on both sides)."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2512_02577_gb300 as p
from oracle import constants, fem, solver
from paper_2512_02577_gb300.inputs import random_vector, vertex_displacements
from tests.test_gpu_parity import DEV, full, n_levels_auto, rel, to_dev

pytestmark = pytest.mark.gpu
DELTA = 0.25


@functools.lru_cache(maxsize=None)
def disp(d, n, delta=DELTA, seed=2512):
    return vertex_displacements(d, n, delta, seed)


def ctx_for(d, n, k, L=0, prec=p.FP64, delta=DELTA, **kw):
    cfg = p.make_config(dim=d, n_cells=n, degree=k, n_levels=L, geometry=p.DISTORTED, mg_precision=prec,
                        vertex_disp=disp(d, n, delta), omega_jacobi=constants.omega_jacobi(d, k),
                        omega_patch=constants.omega_patch(d), **kw)
    return p.Context(cfg, device=DEV)


def mesh_for(d, n, k, delta=DELTA):
    return fem.Mesh(d, n, k, "distorted", geom_fp32=True, disp=disp(d, n, delta))


@functools.lru_cache(maxsize=None)
def hier_for(d, n, k, L, half=False, mult=False, delta=DELTA):
    return solver.Hierarchy(mesh_for(d, n, k, delta), L, constants.omega_jacobi(d, k), constants.omega_patch(d),
                            full_vcycle=not half, multiplicative=mult)


@pytest.mark.parametrize("d,n,k", [(2, 6, 2), (2, 4, 5), (3, 3, 2), (3, 4, 3), (3, 2, 6)])
def test_distorted_apply_and_rhs(d, n, k):
    ctx = ctx_for(d, n, k, L=1)
    m = mesh_for(d, n, k)
    A = fem.assemble(m)
    I = m.interior_index()
    x = random_vector(d, n, k, seed=91)
    y = torch.empty(m.n_dofs, dtype=torch.float64, device=DEV)
    ctx.apply(to_dev(x), y)
    yh = y.cpu().numpy()
    assert rel(yh[I], A @ x[I]) < 1e-12
    b = torch.empty_like(y)
    ctx.rhs_manufactured(b)
    assert rel(b.cpu().numpy(), fem.rhs_manufactured(m)) < 1e-13


@pytest.mark.parametrize("d,n,k,mult", [(2, 8, 3, False), (3, 4, 2, False), (3, 4, 3, True)])
def test_distorted_sweep_and_vcycle(d, n, k, mult):
    sm = p.MULTIPLICATIVE if mult else p.ADDITIVE
    ctx = ctx_for(d, n, k, L=2, smoother=sm)
    h = hier_for(d, n, k, 2, mult=mult)
    lev = h.levels[-1]
    b = random_vector(d, n, k, seed=92)
    u0 = random_vector(d, n, k, seed=93)
    u = to_dev(u0)
    ctx.smooth(to_dev(b), u, sweeps=2)
    assert rel(u.cpu().numpy(), full(lev, lev.smooth(b[lev.I], u0[lev.I], sweeps=2))) < 1e-11
    z = torch.empty_like(u)
    ctx.vcycle(to_dev(b), z)
    assert rel(z.cpu().numpy(), full(lev, h.vcycle(b[lev.I]))) < 1e-11


@pytest.mark.parametrize("d,n,k,half", [(2, 16, 3, 0), (2, 16, 3, 1), (3, 4, 3, 0), (3, 4, 3, 1)])
@pytest.mark.parametrize("prec", [p.FP64, p.FP32])
def test_distorted_solve_and_l2_error(d, n, k, half, prec):
    L = n_levels_auto(n)
    ctx = ctx_for(d, n, k, prec=prec, local_half=half)
    h = hier_for(d, n, k, L, half=bool(half))
    fine = h.levels[-1]
    m = fine.mesh
    b_ref = fem.rhs_manufactured(m)
    b = to_dev(b_ref)
    x = torch.zeros_like(b)
    info = ctx.solve(b, x, rtol=1e-8)
    x_ref, it_ref, _ = solver.solve(h, b_ref[fine.I], rtol=1e-8, outer="gmres" if half else "cg")
    assert info.status == 0
    xh = x.cpu().numpy()
    assert np.linalg.norm(b_ref[fine.I] - fine.A @ xh[fine.I]) <= 2e-8 * np.linalg.norm(b_ref[fine.I])
    if prec == p.FP64:
        assert abs(info.iterations - it_ref) <= 1, (info.iterations, it_ref)
    else:
        assert info.iterations <= it_ref + 3, (info.iterations, it_ref)
    e_lib = ctx.l2_error_manufactured(x)
    e_ref = fem.l2_error_manufactured(m, full(fine, x_ref))
    assert abs(e_lib - e_ref) <= 1e-4 * e_ref + 1e-12


def test_distortion_costs_a_few_iterations():
    # Table 1 (soft): distortion raises the outer iteration count modestly
    its = []
    for delta in (0.0, 0.1, 0.25):
        ctx = ctx_for(3, 8, 3, delta=delta)
        b = torch.empty(ctx.num_dofs(), dtype=torch.float64, device=DEV)
        ctx.rhs_manufactured(b)
        x = torch.zeros_like(b)
        its.append(ctx.solve(b, x).iterations)
    assert its[0] <= its[2] <= its[0] + 8, its
    # zero distortion is the Cartesian mesh
    cart = p.Context(p.make_config(dim=3, n_cells=8, degree=3), device=DEV)
    b = torch.empty(cart.num_dofs(), dtype=torch.float64, device=DEV)
    cart.rhs_manufactured(b)
    x = torch.zeros_like(b)
    assert abs(cart.solve(b, x).iterations - its[0]) <= 1



def test_distorted_fp32_apply_and_block_packing():
    d, n, k = 3, 4, 3
    m = mesh_for(d, n, k)
    A = fem.assemble(m)
    x = random_vector(d, n, k, seed=94)
    ctx = ctx_for(d, n, k, L=2, prec=p.FP32)
    y = torch.empty(m.n_dofs, dtype=torch.float32, device=DEV)
    ctx.apply(to_dev(x, torch.float32), y, prec=p.FP32)
    assert rel(y.cpu().double().numpy()[m.interior_index()], A @ x[m.interior_index()]) < 2e-5
    # every admissible block packing gives bitwise the same sweep
    b = to_dev(random_vector(d, n, k, seed=95), torch.float32)
    outs = []
    for ppc in (1, 2, 5):
        c = ctx_for(d, n, k, L=2, prec=p.FP32, patches_per_block=ppc)
        u = torch.zeros_like(b)
        c.smooth(b, u)
        outs.append(u)
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


def test_inverted_cell_is_rejected():
    # vertex (1, 1) of a 4 x 4 mesh pushed 1.5 h past its neighbour: the
    # cells around it fold over (det J < 0), and pmg_create says so
    n = 4
    d = np.zeros(((n + 1) ** 2, 2))
    d[1 + (n + 1) * 1] = [1.5 / n, 1.5 / n]
    cfg = p.make_config(dim=2, n_cells=n, degree=2, geometry=p.DISTORTED, vertex_disp=d)
    with pytest.raises(p.PmgError) as e:
        p.Context(cfg, device=DEV)
    assert e.value.code == p.PMG_ERR_ARG and "inverted" in str(e.value)
