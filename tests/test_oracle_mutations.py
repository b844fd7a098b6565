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


def _nonsymmetric(n=20, seed=4):
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.5
    M = np.eye(n) + 0.1 * rng.standard_normal((n, n))
    return A, M, rng.standard_normal(n)


def test_wrong_givens_sign_breaks_minimal_residual():
    # planted: g_{j+1} = +sn g_j (the rotated right-hand side with the wrong
    # sign); the least-squares optimality pin must notice
    A, M, b = _nonsymmetric()
    j = 4
    K = np.column_stack([np.linalg.matrix_power(A @ M, i) @ b for i in range(j)])
    y = np.linalg.lstsq(A @ M @ K, b, rcond=None)[0]
    best = np.linalg.norm(b - A @ M @ K @ y)
    x, _, _ = solver.gmres(A, b, lambda v: M @ v, rtol=0.0, maxit=j, restart=30)
    assert abs(np.linalg.norm(b - A @ x) - best) < 1e-9 * best

    def wrong_gmres(A, b, precond, rtol=1e-8, maxit=500, restart=30):
        # the oracle's loop with one planted sign, written out for the test
        x = np.zeros_like(b)
        r = b.copy()
        beta = np.linalg.norm(r)
        V, Z = [r / beta], []
        H = np.zeros((restart + 1, restart))
        g = np.zeros(restart + 1)
        g[0] = beta
        cs, sn = np.zeros(restart), np.zeros(restart)
        for jj in range(maxit):
            Z.append(precond(V[jj]))
            w = A @ Z[jj]
            for i in range(jj + 1):
                H[i, jj] = w @ V[i]
                w = w - H[i, jj] * V[i]
            H[jj + 1, jj] = np.linalg.norm(w)
            V.append(w / H[jj + 1, jj])
            for i in range(jj):
                hi, hn = H[i, jj], H[i + 1, jj]
                H[i, jj] = cs[i] * hi + sn[i] * hn
                H[i + 1, jj] = -sn[i] * hi + cs[i] * hn
            rho = np.hypot(H[jj, jj], H[jj + 1, jj])
            cs[jj], sn[jj] = H[jj, jj] / rho, H[jj + 1, jj] / rho
            H[jj, jj], H[jj + 1, jj] = rho, 0.0
            g[jj + 1] = +sn[jj] * g[jj]                 # planted: sign
            g[jj] = cs[jj] * g[jj]
        yy = np.linalg.solve(np.triu(H[:maxit, :maxit]), g[:maxit])
        return x + sum(yy[i] * Z[i] for i in range(maxit)), maxit, None

    xw, _, _ = wrong_gmres(A, b, lambda v: M @ v, maxit=j)
    assert np.linalg.norm(b - A @ xw) > best * (1 + 1e-6)


def test_missing_residual_update_breaks_sequential_equivalence():
    # planted: every colour reuses the residual of the first one (no update
    # between colours); the pin against the patch-by-patch loop must notice
    m = fem.Mesh(2, 6, 2)
    lev = solver.Level(m, constants.omega_jacobi(2, 2), constants.omega_patch(2), multiplicative=True)
    rng = np.random.default_rng(1)
    b, u = rng.standard_normal(len(lev.I)), rng.standard_normal(len(lev.I))
    ref = lev.mult_sweep_sequential(b, u)
    r = b - lev.A @ u
    wrong = u.copy()
    for c in range(4):
        for v, idx, ps in lev.patches:
            if solver.colour_of(v) == c:
                wrong[idx] += ps.local_solve(r[idx])
    np.testing.assert_allclose(lev.mult_sweep(b, u), ref, atol=1e-12 * np.abs(u).max())
    assert np.abs(wrong - ref).max() > 1e-3 * np.abs(ref).max()


def test_swapped_trilinear_shape_functions_break_volume(monkeypatch):
    # planted: N_0 and N_1 exchanged in the trilinear map; the exact-volume
    # and linear-energy pins must notice
    from paper_2512_02577_gb300.inputs import vertex_displacements
    m = fem.Mesh(2, 3, 2, "distorted", disp=vertex_displacements(2, 3, 0.25, 17))
    orig = fem.Mesh._trilinear_map

    def swapped(self, X):
        Xs = X.copy()
        c = np.minimum(np.floor(Xs * self.n), self.n - 1)
        Xs = (c + 1.0 - (Xs * self.n - c)) / self.n    # xi -> 1 - xi in every cell
        return orig(self, Xs)

    def energy():
        Af = fem.assemble_full(m)
        u = fem.dof_coordinates(m)[:, 0]
        return u @ (Af @ u)

    assert abs(energy() - 1) < 1e-12
    monkeypatch.setattr(fem.Mesh, "_trilinear_map", swapped)
    assert abs(energy() - 1) > 1e-6


def test_eigenvalues_of_a_instead_of_the_jacobi_scaled_patch_break_the_damping_pins():
    # planted: lambda_max of A_{j,p} itself instead of D^{-1/2} A_{j,p} D^{-1/2}
    from tests.test_oracle_pins import lambda_bounds_hold

    def wrong(d, p):
        A = patch.patch_matrix(fem.Mesh(d, 2, p), (1,) * d, p)
        return float(np.linalg.eigvalsh(A)[-1])

    cases = [(2, 2), (2, 5), (3, 2), (3, 3), (3, 4)]
    assert all(lambda_bounds_hold(constants.lambda_max_jacobi(d, p), d, p) for d, p in cases)
    assert not any(lambda_bounds_hold(wrong(d, p), d, p) for d, p in cases)


def test_patch_closure_instead_of_interior_breaks_the_damping_pins():
    # planted: all (2p+1)^d nodes of the 2^d patch cells (Neumann patch
    # matrix with the patch boundary kept) instead of the (2p-1)^d interior
    import itertools
    from tests.test_oracle_pins import lambda_bounds_hold

    def wrong(d, p):
        m = fem.Mesh(d, 2, p)
        nf = 2 * p + 1
        A = np.zeros((nf ** d, nf ** d))
        for off in itertools.product(*([range(2)] * d)):
            Ke = fem.element_stiffness(m, off, p)
            loc = np.zeros(1, dtype=np.int64)
            for dd in range(d):
                g = p * off[dd] + np.arange(p + 1)
                loc = (loc[None, :] + nf ** dd * g[:, None]).reshape(-1)
            A[np.ix_(loc, loc)] += Ke
        s = 1.0 / np.sqrt(np.diag(A))
        return float(np.linalg.eigvalsh(s[:, None] * A * s[None, :])[-1])

    assert not any(lambda_bounds_hold(wrong(d, p), d, p) for d, p in [(2, 3), (3, 2), (3, 3)])
