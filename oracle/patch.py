"""Vertex patches and the local p-multigrid solver, in dense form.

§2.1: a patch Omega_j is the set of 2^d cells around an interior vertex; Pi_j
extracts the DoFs strictly inside the patch.  §2.2 / §3.2: the local problem
on the patch interior is solved approximately by a p-multigrid V-cycle
(Algorithm 3) used as the preconditioner of a local Richardson iteration
(Algorithm 2), on the degree hierarchy p_l = 1, 3, 7, ... capped at the
target degree, with a damped Jacobi smoother on each level (inverse diagonal
stored), embedding prolongation between degrees and its transpose as
restriction, and an exact 1x1 solve on the p = 1 level (§3.2: the patch
interior at p = 1 is the centre vertex alone).

Readings (the paper is silent): each lower p-level operator A_{j,p} is the
rediscretised stiffness of degree p on the same cells and geometry with p+1
Gauss points per direction; the degree rule for targets outside 1, 3, 7, ...
keeps every 2^l - 1 below k and then k (so 4 -> 1, 3, 4 as in §2.2, 8 -> 1,
3, 7, 8, 2 -> 1, 2).  Patch-interior vectors are ordered lexicographically,
x fastest, over the (2p - 1)^d interior nodes of the patch.

Pinned by tests: p = 1 interior is 1 DoF; A_{j,k} equals the submatrix of the
assembled global matrix; the transfer reproduces degree-q polynomials; the
V-cycle is symmetric, a contraction, exact for k = 1, and 25 local Richardson
cycles reach the dense Cholesky solution; the fine level spends two patch
vmults for a zero initial guess (§2.2.1).
"""
import itertools

import numpy as np
import scipy.linalg as sla

from .fem import Mesh, element_stiffness
from .quadrature import gauss_lobatto_nodes, lagrange_values


def p_hierarchy(k):
    """Degrees of the local p-multigrid, coarsest first (§2.2)."""
    levels = []
    p = 1
    while p < k:
        levels.append(p)
        p = 2 * p + 1
    levels.append(k)
    return levels


def interior_vertices(mesh):
    """Interior vertices (v_x, v_y[, v_z]) in lexicographic order, x fastest."""
    rng = [range(1, mesh.n)] * mesh.d
    return [tuple(reversed(v)) for v in itertools.product(*rng[::-1])]


def patch_dofs(mesh, v, p=None):
    """Full-vector indices (on the degree-p grid of ``mesh``) of the
    (2p - 1)^d DoFs strictly inside the patch around vertex v."""
    p = mesh.k if p is None else p
    n1 = p * mesh.n + 1
    loc = np.arange(1, 2 * p)
    idx = np.zeros(1, dtype=np.int64)
    stride = 1
    for dd in range(mesh.d):
        g = p * (v[dd] - 1) + loc
        idx = (idx[None, :] + stride * g[:, None]).reshape(-1)
        stride *= n1
    return idx


def patch_matrix(mesh, v, p):
    """A_{j,p}: stiffness of degree p assembled over the 2^d cells of the
    patch (each cell's element matrix from ``element_stiffness`` with p+1
    Gauss points), restricted to the (2p - 1)^d interior nodes."""
    d = mesh.d
    m = 2 * p + 1
    A = np.zeros((m ** d, m ** d))
    for off in itertools.product(*([range(2)] * d)):
        c = tuple(v[dd] - 1 + off[dd] for dd in range(d))
        Ke = element_stiffness(mesh, c, p)
        loc = np.arange(p + 1)
        idx = np.zeros(1, dtype=np.int64)
        stride = 1
        for dd in range(d):
            g = p * off[dd] + loc
            idx = (idx[None, :] + stride * g[:, None]).reshape(-1)
            stride *= m
        A[np.ix_(idx, idx)] += Ke
    inner = np.arange(1, m - 1)
    idx = np.zeros(1, dtype=np.int64)
    stride = 1
    for dd in range(d):
        idx = (idx[None, :] + stride * inner[:, None]).reshape(-1)
        stride *= m
    return A[np.ix_(idx, idx)]


def transfer_1d(q, p):
    """T (2p-1) x (2q-1): the degree-q patch-interior basis (two cells of the
    patch at s in [0, 1] and [1, 2]) evaluated at the degree-p interior nodes.
    Prolongation from degree q to degree p (the embedding, §3.2)."""
    nq = gauss_lobatto_nodes(q)
    npn = gauss_lobatto_nodes(p)
    s_p = np.concatenate([npn[1:], 1.0 + npn[1:-1]])          # 2p - 1 fine nodes
    T = np.zeros((2 * p - 1, 2 * q - 1))
    for i, s in enumerate(s_p):
        for cell in (0, 1):
            if not (cell <= s <= cell + 1):
                continue
            vals = lagrange_values(nq, s - cell)[0]          # q + 1 local basis values
            for a in range(q + 1):
                node = q * cell + a - 1                       # interior index of local node a
                if 0 <= node < 2 * q - 1:
                    T[i, node] = vals[a]                      # same value from either cell at s = 1
    T[np.abs(T) < 1e-15] = 0.0
    return T


def transfer(q, p, d):
    """d-dimensional transfer T_{q->p} = T x ... x T (Kronecker), x fastest."""
    T1 = transfer_1d(q, p)
    T = T1
    for _ in range(d - 1):
        T = np.kron(T1, T)
    return T


class PatchSolver:
    """Dense local p-multigrid for one patch: matrices A_{j,p}, inverse
    diagonals, transfers, and the coarse 1x1 inverse."""

    def __init__(self, mesh, v, omega_jacobi):
        self.d = mesh.d
        self.levels = p_hierarchy(mesh.k)
        self.A = [patch_matrix(mesh, v, p) for p in self.levels]
        self.Dinv = [1.0 / np.diag(A) for A in self.A]
        self.T = [None] + [transfer(self.levels[l - 1], self.levels[l], mesh.d)
                           for l in range(1, len(self.levels))]
        self.omega = list(omega_jacobi)
        self.vmults = [0] * len(self.levels)

    def vcycle(self, l, r, full=True):
        """Algorithm 3 on level l (0 = p=1) for the residual r."""
        if l == 0:
            return r / self.A[0][0, 0]                         # 1x1 exact coarse solve
        om = self.omega[l]
        d = om * self.Dinv[l] * r                              # pre-smoothing, zero guess
        self.vmults[l] += 1
        res = r - self.A[l] @ d                                # residual
        e = self.vcycle(l - 1, self.T[l].T @ res, full)        # restrict, recurse
        d = d + self.T[l] @ e                                  # prolongate, correct
        if full:
            self.vmults[l] += 1
            res = r - self.A[l] @ d                            # residual for post-smoothing
            d = d + om * self.Dinv[l] * res                    # post-smoothing
        return d

    def local_solve(self, r, n_iter=1, full=True):
        """Algorithm 2: d = V(r); then n_iter - 1 Richardson steps."""
        top = len(self.levels) - 1
        d = self.vcycle(top, r, full)
        for _ in range(2, n_iter + 1):
            self.vmults[top] += 1
            res = r - self.A[top] @ d
            d = d + self.vcycle(top, res, full)
        return d

    def exact_solve(self, r):
        """Dense Cholesky solve with A_{j,k}: the exact patch inverse."""
        c = sla.cho_factor(self.A[-1])
        return sla.cho_solve(c, r)
