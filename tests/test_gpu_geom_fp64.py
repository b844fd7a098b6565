"""FP64 storage of the quadrature-point tensors G_q (pmg_config.geom_precision
= PMG_FP64) on deformed and distorted meshes, against the oracle's operator
built from the unrounded G_q (Eq. (3) at the Gauss points, geom_fp32=False).

Same bounds as the FP32-geometry parity tests: FP64 apply 1e-12, sweeps and
V-cycles 1e-11, FP32 multigrid 2e-5, norm-relative and element-wise.  The
FP32-geometry operator differs from the FP64-geometry one by the rounding of
G_q (about 1e-7 relative), which the last tests check is visible, so that the
option is known to take effect.
"""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2512_02577_gb300 as p
from oracle import constants, fem, solver
from paper_2512_02577_gb300.inputs import random_vector, vertex_displacements
from tests.parity import rel
from tests.test_gpu_parity import DEV, full, n_levels_auto, to_dev

pytestmark = pytest.mark.gpu


def _disp(d, n):
    return vertex_displacements(d, n, 0.2, 77)


def make(d, n, k, geom, L=0, prec=p.FP64, gprec=p.FP64):
    kw = dict(vertex_disp=_disp(d, n)) if geom == "distorted" else {}
    cfg = p.make_config(dim=d, n_cells=n, degree=k, n_levels=L, mg_precision=prec, geom_precision=gprec,
                        geometry=p.DISTORTED if geom == "distorted" else p.DEFORMED, deform_amp=0.05,
                        omega_jacobi=constants.omega_jacobi(d, k), omega_patch=constants.omega_patch(d), **kw)
    return p.Context(cfg, device=DEV)


def mesh(d, n, k, geom):
    if geom == "distorted":
        return fem.Mesh(d, n, k, "distorted", geom_fp32=False, disp=_disp(d, n))
    return fem.Mesh(d, n, k, "deformed", 0.05, geom_fp32=False)


@functools.lru_cache(maxsize=None)
def level(d, n, k, geom):
    return solver.Level(mesh(d, n, k, geom), constants.omega_jacobi(d, k), constants.omega_patch(d))


@functools.lru_cache(maxsize=None)
def hier(d, n, k, geom):
    return solver.Hierarchy(mesh(d, n, k, geom), n_levels_auto(n), constants.omega_jacobi(d, k),
                            constants.omega_patch(d))


@pytest.mark.parametrize("d,n,k,geom", [(3, 4, 3, "deformed"), (3, 3, 2, "deformed"), (2, 6, 3, "deformed"),
                                        (3, 4, 2, "distorted"), (3, 2, 5, "deformed")])
def test_fp64_geometry_apply(d, n, k, geom):
    ctx = make(d, n, k, geom, L=1)
    m = mesh(d, n, k, geom)
    A = fem.assemble(m)
    I = m.interior_index()
    x = random_vector(d, n, k, seed=501)
    y = torch.empty(m.n_dofs, dtype=torch.float64, device=DEV)
    ctx.apply(to_dev(x), y)
    ref = np.zeros(m.n_dofs)
    ref[I] = A @ x[I]
    assert rel(y, ref) < 1e-12
    # the FP32-geometry operator is a different (rounded) one
    ctx32 = make(d, n, k, geom, L=1, gprec=p.FP32)
    y32 = torch.empty_like(y)
    ctx32.apply(to_dev(x), y32)
    assert 1e-10 < rel(y32, ref) < 1e-6


@pytest.mark.parametrize("d,n,k,geom", [(3, 4, 2, "deformed"), (3, 4, 3, "deformed"), (2, 8, 3, "distorted")])
def test_fp64_geometry_sweep_and_vcycle(d, n, k, geom):
    ctx = make(d, n, k, geom)
    h = hier(d, n, k, geom)
    fine = h.levels[-1]
    b = random_vector(d, n, k, seed=511)
    u0 = random_vector(d, n, k, seed=512)
    u = to_dev(u0)
    ctx.smooth(to_dev(b), u, sweeps=1)
    assert rel(u, full(fine, fine.smooth(b[fine.I], u0[fine.I], sweeps=1))) < 1e-11
    z = torch.empty(fine.mesh.n_dofs, dtype=torch.float64, device=DEV)
    ctx.vcycle(to_dev(b), z)
    assert rel(z, full(fine, h.vcycle(b[fine.I]))) < 1e-11


def test_fp64_geometry_mixed_solve_and_geometry_rounding_effect():
    # FP32 V-cycle on FP64-stored G_q, FP64 CG: converges to the oracle's
    # solution of the unrounded operator; the FP32-geometry solve differs
    # from it by the rounding of G_q
    d, n, k = 3, 4, 3
    h = hier(d, n, k, "deformed")
    fine = h.levels[-1]
    b_ref = fem.rhs_manufactured(fine.mesh)
    xs = {}
    for gprec in (p.FP64, p.FP32):
        ctx = make(d, n, k, "deformed", prec=p.FP32, gprec=gprec)
        b = torch.empty(fine.mesh.n_dofs, dtype=torch.float64, device=DEV)
        ctx.rhs_manufactured(b)
        assert rel(b, b_ref) < 1e-13
        x = torch.zeros_like(b)
        info = ctx.solve(b, x, rtol=1e-10)
        assert info.status == 0
        xs[gprec] = x.cpu().numpy()
    x_ref, _, _ = solver.solve(h, b_ref[fine.I], rtol=1e-10)
    assert rel(xs[p.FP64], full(fine, x_ref)) < 1e-8
    assert 1e-10 < rel(xs[p.FP32], xs[p.FP64]) < 1e-5
