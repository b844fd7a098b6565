"""Pins of the CPU oracle against facts other than itself.

Each test checks one piece of the oracle against a closed form, an
independent construction, an invariant of the mathematics, or a number the
paper prints (golden fixtures under tests/golden/), chosen so that a dropped
term, a wrong sign or index, or a transposed operand fails at least one.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import constants, fem, patch, quadrature, solver
from tests.conftest import golden_rows


# ---------------------------------------------------------------- quadrature
def test_gll_closed_forms():
    np.testing.assert_allclose(quadrature.gauss_lobatto_nodes(1), [0, 1], atol=1e-15)
    np.testing.assert_allclose(quadrature.gauss_lobatto_nodes(2), [0, 0.5, 1], atol=1e-15)
    s5 = 1 / math.sqrt(5)
    np.testing.assert_allclose(quadrature.gauss_lobatto_nodes(3),
                               [0, (1 - s5) / 2, (1 + s5) / 2, 1], atol=1e-15)
    s37 = math.sqrt(3 / 7)
    np.testing.assert_allclose(quadrature.gauss_lobatto_nodes(4),
                               [0, (1 - s37) / 2, 0.5, (1 + s37) / 2, 1], atol=1e-15)


def test_gauss_closed_form_and_library():
    x, w = quadrature.gauss_legendre(2)
    np.testing.assert_allclose(x, [0.5 - 0.5 / math.sqrt(3), 0.5 + 0.5 / math.sqrt(3)], atol=1e-15)
    np.testing.assert_allclose(w, [0.5, 0.5], atol=1e-15)
    for n in range(1, 12):
        x, w = quadrature.gauss_legendre(n)
        xl, wl = np.polynomial.legendre.leggauss(n)
        np.testing.assert_allclose(x, (xl + 1) / 2, atol=1e-14)
        np.testing.assert_allclose(w, wl / 2, atol=1e-14)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 9])
def test_gauss_exactness(n):
    x, w = quadrature.gauss_legendre(n)
    assert abs(w.sum() - 1) < 1e-14
    for m in range(2 * n):
        assert abs(w @ x ** m - 1 / (m + 1)) < 1e-14, m
    assert abs(w @ x ** (2 * n) - 1 / (2 * n + 1)) > 1e-12  # not exact beyond 2n-1


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_lagrange_basis(k):
    nodes = quadrature.gauss_lobatto_nodes(k)
    np.testing.assert_allclose(quadrature.lagrange_values(nodes, nodes), np.eye(k + 1), atol=1e-13)
    x = np.linspace(0, 1, 13)
    V = quadrature.lagrange_values(nodes, x)
    D = quadrature.lagrange_derivatives(nodes, x)
    np.testing.assert_allclose(V.sum(1), 1, atol=1e-13)
    np.testing.assert_allclose(D.sum(1), 0, atol=1e-11)
    for m in range(k + 1):   # interpolation reproduces x^m and its derivative
        np.testing.assert_allclose(V @ nodes ** m, x ** m, atol=1e-12)
        np.testing.assert_allclose(D @ nodes ** m, m * x ** max(m - 1, 0) * (m > 0), atol=1e-10)


def test_q1_reference_matrices():
    M, K = quadrature.reference_matrices_1d(1)
    np.testing.assert_allclose(M, [[1 / 3, 1 / 6], [1 / 6, 1 / 3]], atol=1e-15)
    np.testing.assert_allclose(K, [[1, -1], [-1, 1]], atol=1e-15)
    for k in range(1, 9):
        M, K = quadrature.reference_matrices_1d(k)
        assert abs(M.sum() - 1) < 1e-13          # int 1 = 1
        np.testing.assert_allclose(K.sum(1), 0, atol=1e-11)


# ---------------------------------------------------------------- mesh / DoFs
def test_paper_dof_counts():
    for table, r, patches, p, dofs in golden_rows("dof_counts.txt"):
        r, patches, p, dofs = int(r), int(patches), int(p), int(dofs)
        m = fem.Mesh(3, 2 ** (r + 1), p)
        assert m.n_dofs == dofs, (table, r, p)
        assert (m.n - 1) ** 3 == patches
    # enumerate the smallest case's patches explicitly
    assert len(patch.interior_vertices(fem.Mesh(3, 8, 2))) == 343


def test_p_hierarchy_golden():
    for row in golden_rows("p_hierarchy.txt"):
        k, levels = int(row[0]), [int(v) for v in row[1:]]
        assert patch.p_hierarchy(k) == levels
    assert patch.p_hierarchy(8) == [1, 3, 7, 8]
    assert patch.p_hierarchy(2) == [1, 2]


# ---------------------------------------------------------------- geometry
def test_deformation_jacobian_vs_finite_differences():
    for d in (2, 3):
        m = fem.Mesh(d, 4, 2, "deformed", 0.05)
        X = np.random.default_rng(0).random((7, d))
        _, J = m.map_and_jacobian(X)
        eps = 1e-6
        for j in range(d):
            e = np.zeros(d)
            e[j] = eps
            xp, _ = m.map_and_jacobian(X + e)
            xm, _ = m.map_and_jacobian(X - e)
            np.testing.assert_allclose(J[:, :, j], (xp - xm) / (2 * eps), atol=1e-8)


def test_deformation_keeps_boundary_and_orientation():
    m = fem.Mesh(3, 4, 2, "deformed", 0.05)
    g = np.linspace(0, 1, 9)
    for face in range(3):
        for val in (0.0, 1.0):
            P = np.random.default_rng(1).random((20, 3))
            P[:, face] = val
            x, _ = m.map_and_jacobian(P)
            np.testing.assert_allclose(x, P, atol=1e-15)
    X = np.random.default_rng(2).random((1000, 3))
    _, J = m.map_and_jacobian(X)
    assert np.linalg.det(J).min() > 0


def test_deformed_volume_by_quadrature():
    # sum_q w_q det J_q approximates |Omega| = 1 (F maps the cube onto itself)
    for d in (2, 3):
        m = fem.Mesh(d, 4, 3, "deformed", 0.05)
        vol = 0.0
        for c in m.cells():
            G = m.cell_geometry(c, 4)
            _, X, w = m.cell_quadrature(c, 4)
            _, DF = m.map_and_jacobian(X)
            vol += np.sum(w * np.linalg.det(DF * m.h))
        assert abs(vol - 1) < 1e-6


# ---------------------------------------------------------------- assembly
@pytest.mark.parametrize("d,n,k", [(2, 3, 1), (2, 2, 4), (3, 2, 2), (3, 3, 1), (3, 2, 3)])
def test_assembled_equals_kronecker_sum(d, n, k):
    m = fem.Mesh(d, n, k)
    A = fem.assemble(m)
    B = fem.kron_stiffness_cartesian(m)
    assert abs(A - B).max() < 1e-13 * abs(B).max()


@pytest.mark.parametrize("geom", ["cartesian", "deformed"])
@pytest.mark.parametrize("d,k", [(2, 3), (3, 2)])
def test_symmetry_and_neumann_nullspace(geom, d, k):
    m = fem.Mesh(d, 3, k, geom, 0.05)
    Af = fem.assemble_full(m)
    assert abs(Af - Af.T).max() < 1e-14 * abs(Af).max()
    ones = np.ones(Af.shape[0])
    assert np.abs(Af @ ones).max() < 1e-13 * abs(Af).max()
    A = fem.assemble(m)
    rng = np.random.default_rng(3)
    u, v = rng.standard_normal((2, A.shape[0]))
    assert abs(u @ (A @ v) - v @ (A @ u)) < 1e-12 * abs(u @ (A @ v))
    assert u @ (A @ u) > 0


def test_q1_patch_diagonal():
    # Q1 stiffness diagonal at an interior vertex: 8/3 (2D), 8h/3 (3D)
    for d, expect in ((2, 8 / 3), (3, 8 / 3 * 0.25)):
        m = fem.Mesh(d, 4, 1)
        A = fem.assemble(m)
        np.testing.assert_allclose(A.diagonal(), expect, rtol=1e-14)


@pytest.mark.parametrize("d,k", [(2, 1), (2, 3), (3, 2)])
def test_energy_of_linear_function(d, k):
    # u = x_1 lies in V_h on Cartesian meshes: a(u, u) = |Omega| = 1
    m = fem.Mesh(d, 3, k)
    Af = fem.assemble_full(m)
    u = fem.dof_coordinates(m)[:, 0]
    assert abs(u @ (Af @ u) - 1) < 1e-12


# ---------------------------------------------------------------- transfers
@pytest.mark.parametrize("d,k", [(2, 2), (2, 4), (3, 3)])
def test_prolongation_reproduces_polynomials(d, k):
    mc = fem.Mesh(d, 2, k)
    mf = mc.with_level(n=4)
    P = fem.prolongation(mc)
    f = lambda x: np.prod(x ** (k - 1) * (1 - x), axis=1)   # degree k, zero on the boundary
    uc = f(fem.dof_coordinates(mc))[mc.interior_index()]
    uf = f(fem.dof_coordinates(mf))[mf.interior_index()]
    np.testing.assert_allclose(P @ uc, uf, atol=1e-13)


@pytest.mark.parametrize("d,k", [(2, 1), (2, 3), (3, 2)])
def test_galerkin_identity_cartesian(d, k):
    # nested spaces + exact quadrature: P^T A_f P = A_c
    mc = fem.Mesh(d, 2, k)
    P = fem.prolongation(mc)
    Af = fem.assemble(mc.with_level(n=4))
    Ac = fem.assemble(mc)
    assert abs(P.T @ Af @ P - Ac).max() < 1e-12 * abs(Ac).max()


# ---------------------------------------------------------------- patches
def test_p1_patch_is_single_dof():
    for d in (2, 3):
        m = fem.Mesh(d, 3, 1)
        assert len(patch.patch_dofs(m, (1,) * d)) == 1
        assert patch.patch_matrix(m, (1,) * d, 1).shape == (1, 1)


@pytest.mark.parametrize("geom", ["cartesian", "deformed"])
@pytest.mark.parametrize("d,k", [(2, 3), (3, 2)])
def test_patch_matrix_is_submatrix(geom, d, k):
    m = fem.Mesh(d, 3, k, geom, 0.05)
    Af = fem.assemble_full(m).toarray()
    for v in [(1,) * d, (2,) + (1,) * (d - 1)]:
        idx = patch.patch_dofs(m, v)
        Aj = patch.patch_matrix(m, v, k)
        assert np.abs(Aj - Af[np.ix_(idx, idx)]).max() < 1e-15 * np.abs(Af).max() * 10


@pytest.mark.parametrize("q,p", [(1, 2), (1, 3), (3, 4), (3, 7), (7, 8)])
def test_p_transfer_reproduces_polynomials(q, p):
    T = patch.transfer_1d(q, p)
    nq, npn = quadrature.gauss_lobatto_nodes(q), quadrature.gauss_lobatto_nodes(p)
    sq = np.concatenate([nq[1:], 1 + nq[1:-1]])
    sp_ = np.concatenate([npn[1:], 1 + npn[1:-1]])
    f = lambda s: s * (2 - s) * s ** (q - 2) if q >= 2 else np.minimum(s, 2 - s)
    np.testing.assert_allclose(T @ f(sq), f(sp_), atol=1e-13)
    # zero blocks: coarse nodes strictly inside cell 0 do not reach cell 1
    assert np.all(T[p:, :q - 1] == 0) and np.all(T[:p - 1, q:] == 0)


@pytest.mark.parametrize("d,q,p", [(2, 1, 3), (2, 3, 4), (3, 1, 2), (3, 1, 3)])
def test_patch_galerkin_identity(d, q, p):
    m = fem.Mesh(d, 2, p)
    v = (1,) * d
    T = patch.transfer(q, p, d)
    Ap = patch.patch_matrix(m, v, p)
    Aq = patch.patch_matrix(m, v, q)
    assert np.abs(T.T @ Ap @ T - Aq).max() < 1e-12 * np.abs(Aq).max()


# ---------------------------------------------------------------- local p-MG
def _solver(d, k, geom="cartesian"):
    m = fem.Mesh(d, 2, k, geom, 0.05)
    return patch.PatchSolver(m, (1,) * d, constants.omega_jacobi(d, k))


@pytest.mark.parametrize("d,k", [(2, 2), (2, 7), (3, 3), (3, 4)])
def test_local_vcycle_symmetric_and_contracting(d, k):
    ps = _solver(d, k)
    A = ps.A[-1]
    n = A.shape[0]
    V = np.column_stack([ps.local_solve(e) for e in np.eye(n)])
    assert np.abs(V - V.T).max() < 1e-12 * np.abs(V).max()
    E = np.eye(n) - V @ A
    rho = np.max(np.abs(np.linalg.eigvals(E)))
    assert rho < 1
    # V A has spectrum in (0, 1]
    lam = np.linalg.eigvals(V @ A).real
    assert lam.min() > 0 and lam.max() <= 1 + 1e-10


def test_local_vcycle_k1_is_exact():
    for d in (2, 3):
        ps = _solver(d, 1)
        r = np.array([0.7])
        np.testing.assert_allclose(ps.local_solve(r), ps.exact_solve(r), rtol=1e-15)


@pytest.mark.parametrize("d,k,geom", [(2, 4, "cartesian"), (3, 3, "cartesian"), (3, 2, "deformed")])
def test_25_richardson_cycles_reach_cholesky(d, k, geom):
    ps = _solver(d, k, geom)
    r = np.random.default_rng(4).standard_normal(ps.A[-1].shape[0])
    x = ps.exact_solve(r)
    np.testing.assert_allclose(ps.A[-1] @ x, r, atol=1e-10)
    y = ps.local_solve(r, n_iter=25)
    assert np.linalg.norm(y - x) / np.linalg.norm(x) < 1e-6


def test_vmult_counts():
    # §2.2.1: with a zero initial guess the first full V-cycle costs two
    # fine-level vmults and a half V-cycle one; later cycles three and two.
    ps = _solver(2, 3)
    r = np.ones(ps.A[-1].shape[0])
    ps.local_solve(r, n_iter=1, full=True)
    assert ps.vmults[-1] == 2
    ps.vmults = [0] * len(ps.levels)
    ps.local_solve(r, n_iter=2, full=True)
    assert ps.vmults[-1] == 2 + 3
    ps.vmults = [0] * len(ps.levels)
    ps.local_solve(r, n_iter=1, full=False)
    assert ps.vmults[-1] == 1
    ps.vmults = [0] * len(ps.levels)
    ps.local_solve(r, n_iter=2, full=False)
    assert ps.vmults[-1] == 1 + 2


# ---------------------------------------------------------------- smoother
def test_k1_sweep_is_damped_jacobi():
    # k = 1: every patch is one vertex, so the additive sweep is point Jacobi
    for d in (2, 3):
        m = fem.Mesh(d, 4, 1)
        lev = solver.Level(m, constants.omega_jacobi(d, 1), 0.3)
        rng = np.random.default_rng(5)
        b, u = rng.standard_normal((2, lev.A.shape[0]))
        expect = u + 0.3 * (b - lev.A @ u) / lev.A.diagonal()
        np.testing.assert_allclose(lev.smooth(b, u), expect, rtol=1e-13)


def test_single_patch_sweep_with_exact_local_solves():
    # n = 2: one patch covers every free DoF; 25 local cycles ~ exact solve
    m = fem.Mesh(2, 2, 3)
    lev = solver.Level(m, constants.omega_jacobi(2, 3), 0.25, n_iter=25)
    b = np.random.default_rng(6).standard_normal(lev.A.shape[0])
    u = lev.smooth(b, np.zeros_like(b))
    x = solver.direct_solve(lev.A, b)
    np.testing.assert_allclose(u, 0.25 * x, rtol=1e-6, atol=1e-9 * np.abs(x).max())


# ---------------------------------------------------------------- V-cycle / PCG
def _hier(d, n, k, L, geom="cartesian"):
    m = fem.Mesh(d, n, k, geom, 0.05)
    return m, solver.Hierarchy(m, L, constants.omega_jacobi(d, k), constants.omega_patch(d))


@pytest.mark.parametrize("d,n,k,L", [(2, 4, 2, 2), (2, 8, 1, 3), (3, 2, 2, 2)])
def test_vcycle_symmetric_contraction(d, n, k, L):
    m, h = _hier(d, n, k, L)
    A = h.levels[-1].A.toarray()
    N = A.shape[0]
    B = np.column_stack([h.vcycle(e) for e in np.eye(N)])
    assert np.abs(B - B.T).max() < 1e-12 * np.abs(B).max()
    assert np.max(np.abs(np.linalg.eigvals(np.eye(N) - B @ A))) < 1


@pytest.mark.parametrize("d,n,k,L,geom", [(2, 16, 2, 3, "cartesian"), (2, 8, 3, 3, "deformed"),
                                           (3, 4, 2, 2, "cartesian")])
def test_pcg_matches_direct_solve(d, n, k, L, geom):
    m, h = _hier(d, n, k, L, geom)
    b = fem.rhs_manufactured(m)[m.interior_index()]
    x, it, hist = solver.solve(h, b, rtol=1e-8)
    assert hist[-1] <= 1e-8 and it < 40
    xs = solver.direct_solve(h.levels[-1].A, b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-6


# ---------------------------------------------------------------- convergence
def _l2_error(d, n, k, geom="cartesian"):
    m = fem.Mesh(d, n, k, geom, 0.05)
    A = fem.assemble(m)
    b = fem.rhs_manufactured(m)
    I = m.interior_index()
    u = np.zeros(m.n_dofs)
    u[I] = solver.direct_solve(A, b[I])
    return fem.l2_error_manufactured(m, u)


@pytest.mark.parametrize("d,k,ns,geom", [(2, 1, (8, 16, 32), "cartesian"), (2, 2, (4, 8, 16), "cartesian"),
                                         (2, 3, (4, 8, 16), "cartesian"), (2, 4, (4, 8, 16), "cartesian"),
                                         (2, 2, (4, 8, 16), "deformed"), (3, 1, (4, 8, 16), "cartesian"),
                                         (3, 2, (2, 4, 8), "cartesian")])
def test_l2_convergence_rate(d, k, ns, geom):
    e = [_l2_error(d, n, k, geom) for n in ns]
    rate = math.log(e[-2] / e[-1], 2)
    assert abs(rate - (k + 1)) < 0.2, (e, rate)


# ---------------------------------------------------------------- half V-cycle, GMRES
def _vcycle_closed_form(ps, full):
    """The local V-cycle as a matrix, by the recursion of Algorithm 3 written
    as products: with M = omega D^{-1} and C = T B_{l-1} T^T, pre-smoothing
    and coarse correction give X = M + C (I - A M); the full cycle adds
    post-smoothing, B = X + M (I - A X); the half cycle stops at X."""
    B = np.linalg.inv(ps.A[0])
    for l in range(1, len(ps.levels)):
        A = ps.A[l]
        M = np.diag(ps.omega[l] * ps.Dinv[l])
        C = ps.T[l] @ B @ ps.T[l].T
        I = np.eye(A.shape[0])
        X = M + C @ (I - A @ M)
        B = X + M @ (I - A @ X) if full else X
    return B


@pytest.mark.parametrize("d,k", [(2, 3), (2, 7), (3, 3), (3, 4)])
@pytest.mark.parametrize("full", [True, False])
def test_local_vcycle_equals_closed_form(d, k, full):
    ps = _solver(d, k)
    n = ps.A[-1].shape[0]
    V = np.column_stack([ps.local_solve(e, full=full) for e in np.eye(n)])
    B = _vcycle_closed_form(ps, full)
    np.testing.assert_allclose(V, B, atol=1e-12 * np.abs(B).max())
    if not full:
        # dropping post-smoothing makes the local solver nonsymmetric
        assert np.abs(V - V.T).max() > 1e-6 * np.abs(V).max()


@pytest.mark.parametrize("d,k", [(2, 3), (3, 4)])
def test_two_half_vcycles_are_richardson_on_the_half_cycle(d, k):
    # Algorithm 2 with N_iter = 2: d = B r + B (r - A B r) = (2B - B A B) r
    ps = _solver(d, k)
    n = ps.A[-1].shape[0]
    B = _vcycle_closed_form(ps, False)
    V2 = np.column_stack([ps.local_solve(e, n_iter=2, full=False) for e in np.eye(n)])
    np.testing.assert_allclose(V2, 2 * B - B @ ps.A[-1] @ B, atol=1e-12 * np.abs(V2).max())


def _nonsymmetric_system(n=24, seed=9):
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.5
    M = np.eye(n) + 0.1 * rng.standard_normal((n, n))     # a fixed nonsymmetric preconditioner
    b = rng.standard_normal(n)
    return A, M, b


def test_gmres_reaches_direct_solution():
    A, M, b = _nonsymmetric_system()
    x, it, hist = solver.gmres(A, b, lambda v: M @ v, rtol=1e-13, maxit=100, restart=50)
    assert it <= len(b)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10)
    assert np.linalg.norm(b - A @ x) <= 1e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("j", [1, 2, 3, 5])
def test_gmres_minimises_the_residual_over_the_krylov_space(j):
    # x_j = M K y with K = [b, (AM) b, ..., (AM)^{j-1} b] and y the least
    # squares minimiser of ||b - A M K y||: brute force with lstsq
    A, M, b = _nonsymmetric_system()
    x, it, hist = solver.gmres(A, b, lambda v: M @ v, rtol=0.0, maxit=j, restart=30)
    assert it == j
    K = np.column_stack([np.linalg.matrix_power(A @ M, i) @ b for i in range(j)])
    y = np.linalg.lstsq(A @ M @ K, b, rcond=None)[0]
    best = np.linalg.norm(b - A @ M @ K @ y)
    res = np.linalg.norm(b - A @ x)
    np.testing.assert_allclose(res, best, rtol=1e-9)
    # the Givens estimate is the true residual; the history never increases
    np.testing.assert_allclose(hist[-1] * np.linalg.norm(b), res, rtol=1e-9)
    assert all(h1 <= h0 * (1 + 1e-12) for h0, h1 in zip(hist, hist[1:]))


def test_gmres_restart_one_is_minimal_residual_step():
    # GMRES(1), one step: x = alpha M b with alpha = <AMb, b> / <AMb, AMb>
    A, M, b = _nonsymmetric_system()
    x, it, _ = solver.gmres(A, b, lambda v: M @ v, rtol=0.0, maxit=1, restart=1)
    w = A @ M @ b
    np.testing.assert_allclose(x, (w @ b) / (w @ w) * (M @ b), rtol=1e-12)
    # restarted cycles still converge on this well-conditioned system
    x, it, _ = solver.gmres(A, b, lambda v: M @ v, rtol=1e-10, maxit=400, restart=3)
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b) * 1.0001


@pytest.mark.parametrize("d,n,k,L", [(2, 8, 3, 3), (3, 4, 3, 2)])
def test_gmres_with_half_vcycle_matches_direct_solve(d, n, k, L):
    m = fem.Mesh(d, n, k)
    h = solver.Hierarchy(m, L, constants.omega_jacobi(d, k), constants.omega_patch(d), full_vcycle=False)
    fine = h.levels[-1]
    b = np.random.default_rng(2).standard_normal(fine.A.shape[0])
    x, it, hist = solver.solve(h, b, rtol=1e-10, outer="gmres")
    ref = solver.direct_solve(fine.A, b)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-8
    assert np.linalg.norm(b - fine.A @ x) <= 1.0001e-10 * np.linalg.norm(b)
    # §3.2.2: the half cycle costs a few more outer iterations than the full one
    hf = solver.Hierarchy(m, L, constants.omega_jacobi(d, k), constants.omega_patch(d))
    _, it_full, _ = solver.solve(hf, b, rtol=1e-10, outer="gmres")
    assert it_full <= it <= it_full + 6


# ---------------------------------------------------------------- multiplicative smoother
@pytest.mark.parametrize("d,n,k", [(2, 6, 2), (2, 5, 3), (3, 4, 2)])
@pytest.mark.parametrize("forward", [True, False])
def test_colour_sweep_equals_sequential_patch_loop(d, n, k, forward):
    # Algorithm 1 visited patch by patch (residual recomputed after every
    # patch) equals the colour-by-colour update
    m = fem.Mesh(d, n, k)
    lev = solver.Level(m, constants.omega_jacobi(d, k), constants.omega_patch(d), multiplicative=True)
    rng = np.random.default_rng(8)
    b, u = rng.standard_normal(len(lev.I)), rng.standard_normal(len(lev.I))
    np.testing.assert_allclose(lev.mult_sweep(b, u, forward), lev.mult_sweep_sequential(b, u, forward),
                               atol=1e-12 * np.abs(u).max())


def test_multiplicative_sweep_with_exact_solves_is_a_product_of_projections():
    # exact local solves: each patch step is u <- u + P_j (x - u) with the
    # A-orthogonal projection P_j = Pi_j^T A_j^{-1} Pi_j A, so the error
    # e = x - u never grows in the energy norm and the sweep equals the
    # product of (I - P_j) applied to e, patch by patch
    d, n, k = 2, 4, 3
    m = fem.Mesh(d, n, k)
    lev = solver.Level(m, constants.omega_jacobi(d, k), constants.omega_patch(d), multiplicative=True)
    A = lev.A.toarray()
    N = A.shape[0]
    for _, idx, ps in lev.patches:
        ps.local_solve = lambda r, n_iter=1, full=True, ps=ps: ps.exact_solve(r)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(N)
    b = A @ x
    u = lev.mult_sweep(b, np.zeros(N))
    e = x.copy()
    for _, idx, ps in lev.patches:
        Pj = np.zeros((N, N))
        Pj[np.ix_(idx, idx)] = np.linalg.inv(A[np.ix_(idx, idx)])
        e = e - Pj @ A @ e
    np.testing.assert_allclose(x - u, e, atol=1e-10 * np.abs(x).max())
    assert (x - u) @ A @ (x - u) < x @ A @ x


@pytest.mark.parametrize("d,n,k,L", [(2, 8, 3, 3), (3, 4, 2, 2)])
def test_multiplicative_vcycle_symmetric_and_cg_converges(d, n, k, L):
    m = fem.Mesh(d, n, k)
    h = solver.Hierarchy(m, L, constants.omega_jacobi(d, k), constants.omega_patch(d), multiplicative=True)
    fine = h.levels[-1]
    N = fine.A.shape[0]
    rng = np.random.default_rng(5)
    cols = rng.standard_normal((N, 6))
    Bc = np.column_stack([h.vcycle(c) for c in cols.T])
    # forward pre- and backward post-smoothing: <B x, y> = <x, B y>
    np.testing.assert_allclose(cols.T @ Bc, (cols.T @ Bc).T, atol=1e-11 * np.abs(Bc).max())
    b = rng.standard_normal(N)
    x, it, _ = solver.solve(h, b, rtol=1e-10)
    np.testing.assert_allclose(x, solver.direct_solve(fine.A, b), rtol=1e-7, atol=1e-9)
    # the multiplicative smoother needs no more iterations than the additive one
    ha = solver.Hierarchy(m, L, constants.omega_jacobi(d, k), constants.omega_patch(d))
    _, it_add, _ = solver.solve(ha, b, rtol=1e-10)
    assert it <= it_add


# ---------------------------------------------------------------- randomly distorted meshes
def _distorted(d, n, k, delta=0.25, seed=17):
    from paper_2512_02577_gb300.inputs import vertex_displacements
    return fem.Mesh(d, n, k, "distorted", disp=vertex_displacements(d, n, delta, seed))


def test_displacements_recipe():
    from paper_2512_02577_gb300.inputs import vertex_displacements
    D = vertex_displacements(3, 4, 0.3, 5)
    assert D.shape == (125, 3)
    norms = np.linalg.norm(D, axis=1)
    v = np.arange(125)
    inner = np.all([((v // 5 ** m) % 5 > 0) & ((v // 5 ** m) % 5 < 4) for m in range(3)], axis=0)
    np.testing.assert_allclose(norms[inner], 0.3 / 4, rtol=1e-14)
    assert np.all(norms[~inner] == 0)


@pytest.mark.parametrize("d,k", [(2, 1), (2, 3), (3, 1), (3, 2)])
def test_distorted_volume_and_linear_energy(d, k):
    # the trilinear cells tile the unit cube: sum w det J = 1 exactly (det J
    # is a polynomial the (k+1)-point rule integrates exactly), and u = x_1
    # lies in V_h (x is trilinear in the reference coordinates), so
    # a(u, u) = |Omega| = 1
    m = _distorted(d, 3, k)
    vol = 0.0
    for c in m.cells():
        _, X, w = m.cell_quadrature(c, k + 1)
        _, DF = m.map_and_jacobian(X)
        vol += np.sum(w * np.linalg.det(DF * m.h))
    assert abs(vol - 1) < 1e-13
    Af = fem.assemble_full(m)
    u = fem.dof_coordinates(m)[:, 0]
    assert abs(u @ (Af @ u) - 1) < 1e-12
    assert np.abs(Af @ np.ones(Af.shape[0])).max() < 1e-12 * abs(Af).max()
    assert abs(Af - Af.T).max() < 1e-14 * abs(Af).max()


def test_distorted_map_is_continuous_and_zero_distortion_is_cartesian():
    m = _distorted(3, 4, 2)
    # a point on the face x = 1/2 between two cells: both cells' maps agree
    X = np.array([0.5, 0.3, 0.6])
    left = m._trilinear_map(X[None, :] - [1e-15, 0, 0])[0][0]
    right = m._trilinear_map(X[None, :] + [1e-15, 0, 0])[0][0]
    np.testing.assert_allclose(left, right, atol=1e-12)
    # corners land on the displaced vertices
    x, _ = m.map_and_jacobian(np.array([[0.25, 0.5, 0.75]]))
    np.testing.assert_allclose(x[0], m.vertex_position((1, 2, 3)), atol=1e-15)
    m0 = fem.Mesh(3, 3, 2, "distorted", disp=np.zeros((64, 3)))
    A0, A = fem.assemble(m0), fem.assemble(fem.Mesh(3, 3, 2))
    assert abs(A0 - A).max() < 1e-13 * abs(A).max()


def test_distorted_coarse_levels_use_the_fine_vertices():
    m = _distorted(2, 8, 2)
    mc = m.with_level(n=2)
    # coarse vertex (1, 1) is fine vertex (4, 4)
    np.testing.assert_allclose(mc.vertex_position((1, 1)), m.vertex_position((4, 4)), atol=0)


@pytest.mark.parametrize("outer,half", [("cg", False), ("gmres", True)])
def test_distorted_solve_matches_direct(outer, half):
    m = _distorted(2, 8, 3, delta=0.3)
    h = solver.Hierarchy(m, 3, constants.omega_jacobi(2, 3), constants.omega_patch(2), full_vcycle=not half)
    fine = h.levels[-1]
    b = fem.rhs_manufactured(m)[m.interior_index()]
    x, it, hist = solver.solve(h, b, rtol=1e-10, outer=outer)
    assert it < 40
    xs = solver.direct_solve(fine.A, b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-8


def test_multiplicative_half_cycle_gmres_matches_direct_solve():
    # the paper's configuration (Algorithm 1 sweeps, half local V-cycle,
    # GMRES) on a distorted mesh reaches the sparse direct solution
    m = _distorted(2, 8, 3, delta=0.25)
    h = solver.Hierarchy(m, 3, constants.omega_jacobi(2, 3), constants.omega_patch(2), full_vcycle=False,
                         multiplicative=True)
    fine = h.levels[-1]
    b = fem.rhs_manufactured(m)[m.interior_index()]
    x, it, _ = solver.solve(h, b, rtol=1e-10, outer="gmres")
    xs = solver.direct_solve(fine.A, b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-8
    assert it < 20


def test_gmres_is_flexible():
    # a preconditioner that changes every step (M_0, M_1, M_0, ...): the
    # iterate still minimises ||b - A x|| over span{z_0..z_{j-1}}, the
    # stored preconditioned vectors (least squares on the explicit Z)
    A, M, b = _nonsymmetric_system()
    rng = np.random.default_rng(12)
    M2 = np.eye(len(b)) + 0.2 * rng.standard_normal(M.shape)
    calls, Z = [0], []

    def varying(v):
        z = (M if calls[0] % 2 == 0 else M2) @ v
        calls[0] += 1
        Z.append(z)
        return z

    j = 5
    x, it, _ = solver.gmres(A, b, varying, rtol=0.0, maxit=j, restart=30)
    assert it == j and len(Z) == j
    Zm = np.column_stack(Z)
    y = np.linalg.lstsq(A @ Zm, b, rcond=None)[0]
    np.testing.assert_allclose(np.linalg.norm(b - A @ x), np.linalg.norm(b - A @ Zm @ y), rtol=1e-9)
    np.testing.assert_allclose(x, Zm @ y, rtol=1e-8, atol=1e-12)


def test_table1_fixture_is_consistent():
    # the transcribed Table 1 has 16 rows (2 dims x 2 degrees x 4 local
    # solvers) of 4 counts, and the orderings the GPU test asserts hold for
    # the printed numbers themselves
    rows = golden_rows("table1_gmres_iterations.txt")
    assert len(rows) == 16 and all(len(r) == 7 for r in rows)
    t = {(int(r[0]), int(r[1]), r[2]): [int(v) for v in r[3:]] for r in rows}
    for dim in (2, 3):
        for k in (3, 7):
            for i in range(4):
                assert t[(dim, k, "25V")][i] <= t[(dim, k, "1V")][i] <= t[(dim, k, "1H")][i]
                assert t[(dim, k, "2H")][i] <= t[(dim, k, "1H")][i]
            for s in ("1V", "1H", "2H", "25V"):
                assert all(b >= a for a, b in zip(t[(dim, k, s)], t[(dim, k, s)][1:]))


# ------------------------------------------------------------ Jacobi damping
# lambda_max(D^{-1} A_{j,p}) on the unit Cartesian patch is what the omega_J
# reading (4 / (3 lambda_max)) rests on.  Pinned by bounds that the
# mathematics fixes and by a textbook construction, not by re-running the
# oracle's eigen-solve.
def _patch_and_diag(d, p):
    A = patch.patch_matrix(fem.Mesh(d, 2, p), (1,) * d, p)
    return A, np.diag(A).copy()


def _power_rayleigh(A, D, iters=3000):
    """Power iteration on D^{-1} A (own loop) and the generalised Rayleigh
    quotient v^T A v / v^T D v of its last iterate: a lower bound of
    lambda_max(D^{-1} A) for any v, equal to it once converged."""
    v = np.cos(2.1 * np.arange(A.shape[0])) + 0.3
    for _ in range(iters):
        w = (A @ v) / D
        v = w / np.linalg.norm(w)
    return float(v @ (A @ v)) / float(v @ (D * v))


def lambda_bounds_hold(lam, d, p):
    """Rayleigh lower bound <= lambda <= Gershgorin bound of D^{-1} A, and
    lambda within 1e-9 of the converged power-iteration quotient."""
    A, D = _patch_and_diag(d, p)
    R = _power_rayleigh(A, D)
    G = float(np.max(np.abs(A).sum(axis=1) / D))
    return R <= lam * (1 + 1e-12) and lam <= G and abs(lam - R) <= 1e-9 * lam


@pytest.mark.parametrize("d,p", [(2, 2), (2, 3), (2, 5), (2, 8), (3, 2), (3, 3), (3, 4), (3, 5)])
def test_lambda_max_jacobi_between_rayleigh_and_gershgorin(d, p):
    assert lambda_bounds_hold(constants.lambda_max_jacobi(d, p), d, p)


def _q2_patch_1d():
    """1D Q2 (nodes 0, 1/2, 1) element stiffness and exact mass on a unit
    cell, textbook values, assembled over two cells and restricted to the
    three patch-interior nodes (mid-point, centre vertex, mid-point)."""
    Ke = np.array([[7., -8., 1.], [-8., 16., -8.], [1., -8., 7.]]) / 3.0
    Me = np.array([[4., 2., -1.], [2., 16., 2.], [-1., 2., 4.]]) / 30.0
    K, M = np.zeros((5, 5)), np.zeros((5, 5))
    for c in (0, 2):
        K[c:c + 3, c:c + 3] += Ke
        M[c:c + 3, c:c + 3] += Me
    return K[1:4, 1:4], M[1:4, 1:4]


def test_q2_textbook_patch_matrices():
    # the typed element matrices: K annihilates constants, M integrates 1 to 1,
    # and the 1D patch has lambda_max(D^{-1} K) = 1 + 2/sqrt(7) in closed form
    Ke = np.array([[7., -8., 1.], [-8., 16., -8.], [1., -8., 7.]]) / 3.0
    Me = np.array([[4., 2., -1.], [2., 16., 2.], [-1., 2., 4.]]) / 30.0
    assert np.abs(Ke.sum(axis=1)).max() < 1e-15 and abs(Me.sum() - 1.0) < 1e-15
    K, _ = _q2_patch_1d()
    s = 1.0 / np.sqrt(np.diag(K))
    assert abs(np.linalg.eigvalsh(s[:, None] * K * s[None, :])[-1] - (1 + 2 / np.sqrt(7))) < 1e-14


@pytest.mark.parametrize("d", [2, 3])
def test_lambda_max_jacobi_q2_equals_textbook_kronecker_patch(d):
    # A_{j,2} = sum_dir (K on dir, M elsewhere) from the textbook 1D matrices
    # (the cell size scales A uniformly, so D^{-1} A does not depend on it)
    K, M = _q2_patch_1d()
    A = np.zeros((3 ** d, 3 ** d))
    for direction in range(d):
        term = np.ones((1, 1))
        for ax in reversed(range(d)):          # x fastest: the x factor is the last kron
            term = np.kron(term, K if ax == direction else M)
        A += term
    s = 1.0 / np.sqrt(np.diag(A))
    lam = np.linalg.eigvalsh(s[:, None] * A * s[None, :])[-1]
    assert abs(constants.lambda_max_jacobi(d, 2) - lam) <= 1e-12 * lam
