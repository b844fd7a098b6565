"""Additive vertex-patch smoother, geometric multigrid V-cycle and PCG.

Smoother (§2.1, Algorithm 1 with the sequential update replaced by a sum,
i.e. the additive Schwarz variant): with the global residual r = b - A u,

    u <- u + omega_AS * sum_j Pi_j^T LocalSolve_j(Pi_j r),

where LocalSolve is Algorithm 2 around Algorithm 3 (``patch.PatchSolver``).
The sum is accumulated colour by colour (the 2^d parities of the vertex
index), lexicographically within a colour; the order changes only rounding.

Multiplicative smoother (Algorithm 1 as printed): patches one after the
other, each computing its residual from the current u.  Patches of one
parity colour have disjoint interiors, and no patch's closure meets the
interior of another patch of its colour, so updating a whole colour from
one residual is the same as visiting its patches one by one: a sweep is
the sequential Algorithm 1 in colour-major order (colours 0..2^d-1 forward;
post-smoothing visits them backward, so the V-cycle stays symmetric).
The paper colours patches so that no two of a colour share any DoF; the
parity colouring is the weaker condition that suffices here, because a
patch writes only its interior.

V-cycle (§2, Eq. (1)-(4)): one pre- and one post-smoothing sweep, residual,
restriction R = P^T, recursion, prolongation P (the embedding), and an exact
dense Cholesky solve on the coarsest level.  Pre-smoothing starts from a zero
guess, so its residual is the right-hand side.

Outer solvers, x_0 = 0, stopping when ||r||_2 <= rtol ||b||_2 on the free
DoFs: preconditioned CG (the additive smoother with the full, symmetric
local V-cycle gives a symmetric preconditioner) and GMRES (the paper's outer
solver; needed once the local solver is the half V-cycle of §3.2.2, which
drops post-smoothing and makes the preconditioner nonsymmetric).  GMRES is
the flexible right-preconditioned form (restarted, Arnoldi with modified
Gram-Schmidt, Givens rotations on the Hessenberg matrix); with a fixed
preconditioner it is right-preconditioned GMRES.

Parity of the iteration counts of this additive variant is unpinned by the
paper (its Table 1 is for the multiplicative smoother with GMRES); the tests
pin the V-cycle's symmetry and contraction and the PCG solution against a
sparse direct solve.
"""
import itertools

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .fem import Mesh, assemble, prolongation
from .patch import PatchSolver, interior_vertices, patch_dofs


def colour_of(v):
    """Parity colour of a vertex: sum_i (v_i mod 2) 2^i."""
    return sum((vi % 2) << i for i, vi in enumerate(v))


class Level:
    """One mesh level: assembled A_l on the free DoFs and its patches."""

    def __init__(self, mesh, omega_jacobi, omega_patch, n_iter=1, full_vcycle=True,
                 with_patches=True, multiplicative=False):
        self.mesh = mesh
        self.A = assemble(mesh)
        self.I = mesh.interior_index()
        self.pos = -np.ones(mesh.n_dofs, dtype=np.int64)
        self.pos[self.I] = np.arange(len(self.I))
        self.omega_patch = omega_patch
        self.n_iter = n_iter
        self.full = full_vcycle
        self.multiplicative = multiplicative
        self.patches = []
        if with_patches:
            verts = interior_vertices(mesh)
            verts.sort(key=lambda v: colour_of(v))   # stable: lexicographic within a colour
            for v in verts:
                self.patches.append((v, self.pos[patch_dofs(mesh, v)],
                                     PatchSolver(mesh, v, omega_jacobi)))

    def smooth_correction(self, r):
        """omega_AS sum_j Pi_j^T LocalSolve_j(Pi_j r) for a residual r on the
        free DoFs."""
        c = np.zeros_like(r)
        for _, idx, ps in self.patches:
            c[idx] += ps.local_solve(r[idx], self.n_iter, self.full)
        return self.omega_patch * c

    def mult_sweep(self, b, u, forward=True):
        """One multiplicative sweep (Algorithm 1), colour by colour: per
        colour the residual b - A u, then every patch of the colour adds its
        local solve to its interior DoFs (no damping)."""
        u = u.copy()
        colours = range(1 << self.mesh.d)
        for c in (colours if forward else reversed(colours)):
            r = b - self.A @ u
            for v, idx, ps in self.patches:
                if colour_of(v) == c:
                    u[idx] += ps.local_solve(r[idx], self.n_iter, self.full)
        return u

    def mult_sweep_sequential(self, b, u, forward=True):
        """Algorithm 1 literally: patch after patch in colour-major order,
        each residual from the u its predecessor left (test reference for
        ``mult_sweep``)."""
        u = u.copy()
        order = self.patches if forward else self.patches[::-1]
        for v, idx, ps in order:
            r = b - self.A @ u
            u[idx] += ps.local_solve(r[idx], self.n_iter, self.full)
        return u

    def smooth(self, b, u, sweeps=1):
        """``sweeps`` sweeps: additive u <- u + S (b - A u), or forward
        multiplicative sweeps."""
        u = u.copy()
        for _ in range(sweeps):
            if self.multiplicative:
                u = self.mult_sweep(b, u)
            else:
                u = u + self.smooth_correction(b - self.A @ u)
        return u


class Hierarchy:
    """Geometric hierarchy n_l = n_0 2^l, l = 0..L (finest last)."""

    def __init__(self, mesh, n_levels, omega_jacobi, omega_patch, n_iter=1,
                 full_vcycle=True, smooth_steps=1, multiplicative=False):
        ns = [mesh.n]
        for _ in range(n_levels - 1):
            if ns[-1] % 2:
                raise ValueError("n must be divisible by 2^(levels-1)")
            ns.append(ns[-1] // 2)
        ns = ns[::-1]
        self.levels = []
        for l, n in enumerate(ns):
            self.levels.append(Level(mesh.with_level(n=n), omega_jacobi, omega_patch,
                                     n_iter, full_vcycle, with_patches=(l > 0),
                                     multiplicative=multiplicative))
        self.P = [None] + [prolongation(self.levels[l - 1].mesh) for l in range(1, len(ns))]
        A0 = self.levels[0].A.toarray()
        self.coarse = sla.cho_factor(A0) if A0.size else None
        self.smooth_steps = smooth_steps

    def coarse_solve(self, b):
        if self.coarse is None:
            return b.copy()
        return sla.cho_solve(self.coarse, b)

    def vcycle(self, b, l=None):
        """z = B_l b (zero initial guess)."""
        l = len(self.levels) - 1 if l is None else l
        if l == 0:
            return self.coarse_solve(b)
        lev = self.levels[l]
        u = np.zeros_like(b)
        for s in range(self.smooth_steps):
            if lev.multiplicative:
                u = lev.mult_sweep(b, u, forward=True)
            else:
                # the first pre-smoothing residual is b itself (zero guess)
                r = b if s == 0 else b - lev.A @ u
                u = u + lev.smooth_correction(r)
        r = b - lev.A @ u
        u = u + self.P[l] @ self.vcycle(self.P[l].T @ r, l - 1)
        for _ in range(self.smooth_steps):
            if lev.multiplicative:
                u = lev.mult_sweep(b, u, forward=False)
            else:
                u = u + lev.smooth_correction(b - lev.A @ u)
        return u


def pcg(A, b, precond, rtol=1e-8, maxit=500):
    """Preconditioned CG from x_0 = 0; returns (x, iterations, rel_residual
    history).  Stops when ||r|| <= rtol ||b||."""
    x = np.zeros_like(b)
    r = b.copy()
    nb = np.linalg.norm(b)
    hist = [1.0]
    if nb == 0:
        return x, 0, hist
    z = precond(r)
    p = z.copy()
    rz = r @ z
    it = 0
    while it < maxit:
        Ap = A @ p
        alpha = rz / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        it += 1
        hist.append(np.linalg.norm(r) / nb)
        if hist[-1] <= rtol:
            break
        z = precond(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, hist


def gmres(A, b, precond, rtol=1e-8, maxit=500, restart=30):
    """Flexible right-preconditioned GMRES(restart) from x_0 = 0; returns
    (x, iterations, rel_residual history).  Each Arnoldi step stores
    z_j = M^{-1} v_j, orthogonalises A z_j against v_0..v_j (modified
    Gram-Schmidt), and updates the QR factorisation of the Hessenberg matrix
    by one Givens rotation; |g_{j+1}| is then the residual norm of the
    minimiser over span{z_0..z_j}.  The step stops when that norm is below
    rtol ||b||, when maxit steps are done, or at the end of a cycle (then
    x += Z y and the cycle restarts from the true residual)."""
    x = np.zeros_like(b)
    nb = np.linalg.norm(b)
    hist = [1.0]
    if nb == 0:
        return x, 0, hist
    it = 0
    while True:
        r = b - A @ x
        beta = np.linalg.norm(r)
        if beta == 0 or it >= maxit:
            return x, it, hist
        V, Z = [r / beta], []
        H = np.zeros((restart + 1, restart))
        g = np.zeros(restart + 1)
        g[0] = beta
        cs, sn = np.zeros(restart), np.zeros(restart)
        j = 0
        while j < restart and it < maxit:
            Z.append(precond(V[j]))
            w = A @ Z[j]
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j] if H[j + 1, j] > 0 else w)
            for i in range(j):          # earlier rotations on the new column
                hi, hn = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * hi + sn[i] * hn
                H[i + 1, j] = -sn[i] * hi + cs[i] * hn
            rho = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / rho, H[j + 1, j] / rho
            H[j, j], H[j + 1, j] = rho, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            j += 1
            it += 1
            hist.append(abs(g[j]) / nb)
            if hist[-1] <= rtol:
                break
        y = sla.solve_triangular(H[:j, :j], g[:j])
        for i in range(j):
            x = x + y[i] * Z[i]
        if hist[-1] <= rtol or it >= maxit:
            return x, it, hist


def solve(h, b_int, rtol=1e-8, maxit=500, outer="cg", restart=30):
    """PCG (outer = "cg") or GMRES (outer = "gmres") on the finest level of
    hierarchy ``h`` with the V-cycle as preconditioner; b and x on the free
    DoFs."""
    fine = h.levels[-1]
    if outer == "gmres":
        return gmres(fine.A, b_int, h.vcycle, rtol, maxit, restart)
    return pcg(fine.A, b_int, h.vcycle, rtol, maxit)


def direct_solve(A, b):
    """Sparse direct reference solution."""
    return spla.spsolve(A.tocsc(), b)
