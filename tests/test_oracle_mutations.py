"""Planted mistakes in the oracle (CPU only) must be caught by its pins.

Each test swaps one oracle routine for a plausibly wrong variant and checks
that the property the pin suite relies on fails for it, so the pins are
known to be sensitive to that class of mistake.
"""
import numpy as np

from oracle import constants, fem, patch, solver


def _vcycle_matrix(ps):
    n = ps.A[-1].shape[0]
    return np.column_stack([ps.local_solve(e) for e in np.eye(n)])


def _ps(d=2, k=3):
    m = fem.Mesh(d, 2, k)
    return patch.PatchSolver(m, (1,) * d, constants.omega_jacobi(d, k))


def test_dropped_post_smoothing_breaks_symmetry():
    ps = _ps()
    V = _vcycle_matrix(ps)
    assert np.abs(V - V.T).max() < 1e-12 * np.abs(V).max()
    Vh = np.column_stack([ps.local_solve(e, full=False) for e in np.eye(ps.A[-1].shape[0])])
    assert np.abs(Vh - Vh.T).max() > 1e-6 * np.abs(Vh).max()


def test_residual_sign_error_breaks_contraction(monkeypatch):
    ps = _ps()
    orig = patch.PatchSolver.vcycle

    def wrong(self, l, r, full=True):
        if l == 0:
            return r / self.A[0][0, 0]
        om = self.omega[l]
        d = om * self.Dinv[l] * r
        res = r + self.A[l] @ d                       # planted: wrong sign
        e = wrong(self, l - 1, self.T[l].T @ res, full)
        d = d + self.T[l] @ e
        res = r - self.A[l] @ d
        return d + om * self.Dinv[l] * res

    monkeypatch.setattr(patch.PatchSolver, "vcycle", wrong)
    V = _vcycle_matrix(ps)
    rho = np.max(np.abs(np.linalg.eigvals(np.eye(V.shape[0]) - V @ ps.A[-1])))
    monkeypatch.setattr(patch.PatchSolver, "vcycle", orig)
    assert rho >= 1 or np.abs(V - V.T).max() > 1e-8


def test_transposed_geometry_tensor_breaks_convergence(monkeypatch):
    # planted: G = w det J J^{-T} J^{-1} instead of J^{-1} J^{-T}
    def wrong_geometry(self, c, nq):
        _, X, w = self.cell_quadrature(c, nq)
        _, DF = self.map_and_jacobian(X)
        J = DF * self.h
        Jinv = np.linalg.inv(J)
        return w[:, None, None] * np.linalg.det(J)[:, None, None] * np.einsum("qji,qjk->qik", Jinv, Jinv)

    def err(n):
        m = fem.Mesh(2, n, 2, "deformed", 0.05)
        A = fem.assemble(m)
        b = fem.rhs_manufactured(m)
        I = m.interior_index()
        u = np.zeros(m.n_dofs)
        u[I] = solver.direct_solve(A, b[I])
        return fem.l2_error_manufactured(m, u)

    good = err(16)
    monkeypatch.setattr(fem.Mesh, "cell_geometry", wrong_geometry)
    bad = err(16)
    assert bad > 20 * good


def test_wrong_transfer_breaks_galerkin_identity(monkeypatch):
    d, q, p = 2, 1, 3
    m = fem.Mesh(d, 2, p)
    T = patch.transfer(q, p, d)
    Ap = patch.patch_matrix(m, (1,) * d, p)
    Aq = patch.patch_matrix(m, (1,) * d, q)
    Tbad = T[::-1]                                    # planted: reversed node order
    Tbad = Tbad * 0.9
    assert np.abs(T.T @ Ap @ T - Aq).max() < 1e-12 * np.abs(Aq).max()
    assert np.abs(Tbad.T @ Ap @ Tbad - Aq).max() > 1e-3 * np.abs(Aq).max()
