"""The float-float FP64 operator (outer_apply = PMG_OUTER_APPLY_FLOAT_FLOAT)
against the oracle, through the C ABI.

The operator of Eq. (4) applied to FP64 vectors with every product and sum
carried as a pair of floats (about 48 significant bits).  Bound used here:
the same 1e-12 relative (norm and element-wise) as the FP64 apply, which
float-float meets with room to spare on these sizes (its rounding is a few
1e-14 of |A||x| per entry); the mixed-precision solve with it must reach
||r|| <= 1e-8 ||b|| with the true residual (recomputed by the oracle's
assembled matrix) below 2e-8, in the iterations of the FP64-apply solve +-1.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2512_02577_gb300 as p
from oracle import fem, solver
from paper_2512_02577_gb300.inputs import random_vector
from tests.parity import rel
from tests.test_gpu_parity import (DEV, _sampled_apply_rows, full, make_ctx, n_levels_auto, oracle_hier,
                                   oracle_operator, to_dev)

pytestmark = pytest.mark.gpu
FF = dict(outer_apply=p.APPLY_FLOAT_FLOAT)


@pytest.mark.parametrize("d,n,k", [(2, 16, 2), (2, 5, 3), (2, 3, 8), (3, 4, 1), (3, 3, 2), (3, 4, 3), (3, 3, 4),
                                   (3, 2, 5), (3, 2, 6), (3, 2, 7), (3, 2, 8)])
def test_float_float_apply_and_residual(d, n, k):
    ctx = make_ctx(d, n, k, L=1, **FF)
    lev = oracle_operator(d, n, k, "cartesian")
    x = random_vector(d, n, k, seed=20 + n + k)
    x_noisy = x.copy()
    x_noisy[~lev.mesh.interior_mask()] = 3.0          # boundary inputs are ignored
    y = torch.empty(lev.mesh.n_dofs, dtype=torch.float64, device=DEV)
    ctx.apply(to_dev(x_noisy), y)
    y_ref = fem.apply_full(lev.mesh, lev.A, x)
    assert rel(y, y_ref) < 1e-12
    assert torch.count_nonzero(y.cpu()[torch.tensor(~lev.mesh.interior_mask())]) == 0
    b = random_vector(d, n, k, seed=98)
    r = torch.empty_like(y)
    ctx.residual(to_dev(b), to_dev(x), r)
    assert rel(r, b - y_ref) < 1e-12


def test_float_float_full_size_sampled_rows():
    d, n, k = 3, 32, 4
    ctx = make_ctx(d, n, k, prec=p.FP32, **FF)
    m = fem.Mesh(d, n, k)
    x = random_vector(d, n, k, seed=61)
    y = torch.empty(m.n_dofs, dtype=torch.float64, device=DEV)
    ctx.apply(to_dev(x), y)
    rows = np.random.default_rng(62).integers(0, m.n_dofs, 300)
    ref = _sampled_apply_rows(m, x, rows)
    assert np.abs(y.cpu().numpy()[rows] - ref).max() <= 1e-12 * np.abs(ref).max()
    # against the FP64 apply on every entry
    ctx64 = make_ctx(d, n, k, prec=p.FP32)
    y64 = torch.empty_like(y)
    ctx64.apply(to_dev(x), y64)
    assert rel(y, y64) < 1e-12


@pytest.mark.parametrize("d,n,k,L", [(2, 16, 2, 3), (3, 8, 2, 0), (3, 4, 4, 0)])
def test_mixed_solve_with_float_float_operator(d, n, k, L):
    h = oracle_hier(d, n, k, L if L else n_levels_auto(n), "cartesian")
    fine = h.levels[-1]
    b_ref = fem.rhs_manufactured(fine.mesh)
    its = {}
    for apply in (p.APPLY_FP64, p.APPLY_FLOAT_FLOAT):
        ctx = make_ctx(d, n, k, L=L, prec=p.FP32, outer_apply=apply)
        b = torch.empty(fine.mesh.n_dofs, dtype=torch.float64, device=DEV)
        ctx.rhs_manufactured(b)
        x = torch.zeros_like(b)
        info = ctx.solve(b, x, rtol=1e-8)
        assert info.status == 0 and info.rel_residual <= 1e-8
        xh = x.cpu().numpy()
        true_res = np.linalg.norm(b_ref[fine.I] - fine.A @ xh[fine.I]) / np.linalg.norm(b_ref[fine.I])
        assert true_res <= 2e-8, (apply, true_res)
        x_ref, _, _ = solver.solve(h, b_ref[fine.I], rtol=1e-8)
        assert rel(xh, full(fine, x_ref)) < 1e-5
        its[apply] = info.iterations
    assert abs(its[p.APPLY_FP64] - its[p.APPLY_FLOAT_FLOAT]) <= 1, its


@pytest.mark.parametrize("d,n,k", [(3, 4, 3), (3, 3, 2), (3, 4, 1)])
def test_float_float_deformed_apply_and_residual(d, n, k):
    # the half-warp cell kernel in float-float arithmetic on the FP32-stored
    # G_q (the same discrete operator as the FP64 apply and the oracle's)
    ctx = make_ctx(d, n, k, L=1, geom="deformed", **FF)
    lev = oracle_operator(d, n, k, "deformed")
    x = random_vector(d, n, k, seed=40 + n + k)
    y = torch.empty(lev.mesh.n_dofs, dtype=torch.float64, device=DEV)
    ctx.apply(to_dev(x), y)
    y_ref = fem.apply_full(lev.mesh, lev.A, x)
    assert rel(y, y_ref) < 1e-12
    b = random_vector(d, n, k, seed=97)
    r = torch.empty_like(y)
    ctx.residual(to_dev(b), to_dev(x), r)
    assert rel(r, b - y_ref) < 1e-12


def test_float_float_distorted_mixed_solve():
    from paper_2512_02577_gb300.inputs import vertex_displacements
    d, n, k = 3, 8, 3
    disp = vertex_displacements(d, n, 0.2, 31)
    its = {}
    for apply in (p.APPLY_FP64, p.APPLY_FLOAT_FLOAT):
        ctx = p.Context(p.make_config(dim=d, n_cells=n, degree=k, geometry=p.DISTORTED, vertex_disp=disp,
                                      mg_precision=p.FP32, outer_apply=apply), device=DEV)
        b = torch.empty(ctx.num_dofs(), dtype=torch.float64, device=DEV)
        ctx.rhs_manufactured(b)
        x = torch.zeros_like(b)
        info = ctx.solve(b, x, rtol=1e-8)
        assert info.status == 0 and info.rel_residual <= 1e-8
        its[apply] = (info.iterations, x)
    assert abs(its[p.APPLY_FP64][0] - its[p.APPLY_FLOAT_FLOAT][0]) <= 1
    assert rel(its[p.APPLY_FLOAT_FLOAT][1], its[p.APPLY_FP64][1]) < 1e-7


@pytest.mark.parametrize("kw", [dict(dim=2, n_cells=4, degree=2, geometry=p.DEFORMED),
                                dict(dim=3, n_cells=4, degree=4, geometry=p.DEFORMED),
                                dict(dim=3, n_cells=4, degree=2, geometry=p.DEFORMED, geom_precision=p.FP64)])
def test_float_float_operator_limits(kw):
    with pytest.raises(p.PmgError) as e:
        p.Context(p.make_config(**kw, **FF), device=DEV)
    assert e.value.code == p.PMG_ERR_UNSUPPORTED
