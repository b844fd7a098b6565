"""Structured Q_k finite elements on the unit square/cube, assembled.

Follows §2 of the paper: a hierarchy of nested meshes (Eq. (1)) with spaces
V_l, embedding prolongation and its l2-adjoint restriction (Eq. (2)), and the
level matrices A_l of Eq. (4) obtained by applying the bilinear form
a(u, v) = int grad u . grad v (Eq. (3)) to the basis functions of V_l.

Mesh: n cells per side, h = 1/n, DoFs on the (k n + 1)^d grid, lexicographic
with x fastest.  Dirichlet conditions: boundary DoFs are removed; a full-length
vector carries zeros there (the convention y_B = 0).

Geometry: Cartesian x = X, or the smooth deformation
F(X) = X + a prod_m sin(2 pi X_m) (1, ..., 1), evaluated analytically at the
quadrature points (§4 uses deformed meshes; this analytic map is the reading
for the smoothly deformed configuration).  F is the identity on the boundary,
so the domain stays the unit cube, and since F is one global map, coarse
spaces are exactly nested in fine ones (§2: topological nestedness).
Or a randomly distorted mesh (§3.2.2, §4): the vertices of the finest mesh
displaced (an input array), every cell of every level the trilinear
(bilinear in 2D) image of the reference cell spanned by its displaced
corners; a coarse vertex is the fine vertex at the same grid position, so
the levels are nested topologically but not geometrically (the transfers
stay the reference embedding, Eq. (2)).
"""
import functools
import itertools

import numpy as np
import scipy.sparse as sp

from .quadrature import (gauss_legendre, gauss_lobatto_nodes, lagrange_derivatives,
                         lagrange_values)


class Mesh:
    """Structured mesh description: dimension d, n cells per side, degree k,
    geometry ('cartesian' or 'deformed' with amplitude ``amp``), and whether
    the stored quadrature-point tensors are rounded to float32."""

    def __init__(self, d, n, k, geometry="cartesian", amp=0.05, geom_fp32=False, disp=None, n_fine=None):
        if d not in (2, 3):
            raise ValueError("d in {2, 3}")
        self.d, self.n, self.k = d, n, k
        self.geometry = geometry
        self.amp = amp
        # distorted: displacements of the finest mesh's (n_fine + 1)^d vertices
        self.disp = None if disp is None else np.asarray(disp, dtype=np.float64)
        self.n_fine = n if n_fine is None else n_fine
        if geometry == "distorted" and (self.disp is None or self.n_fine % n):
            raise ValueError("distorted geometry needs fine-vertex displacements and n | n_fine")
        self.geom_fp32 = bool(geom_fp32) and geometry != "cartesian"
        self.h = 1.0 / n
        self.n1 = k * n + 1

    def with_level(self, n=None, k=None):
        return Mesh(self.d, self.n if n is None else n, self.k if k is None else k,
                    self.geometry, self.amp, self.geom_fp32, self.disp, self.n_fine)

    @property
    def n_dofs(self):
        return self.n1 ** self.d

    def interior_mask(self):
        g = np.arange(self.n1)
        m1 = (g > 0) & (g < self.n1 - 1)
        m = m1
        for _ in range(self.d - 1):
            m = np.multiply.outer(m1, m)  # slowest index outermost
        return m.reshape(-1)

    def interior_index(self):
        """Full-vector indices of the free (interior) DoFs, ascending."""
        return np.nonzero(self.interior_mask())[0]

    def cells(self):
        """All cell multi-indices (c_x, c_y[, c_z]) in lexicographic order."""
        rng = [range(self.n)] * self.d
        for c in itertools.product(*rng[::-1]):
            yield tuple(reversed(c))

    def cell_dofs(self, c, k=None):
        """Global full-vector DoF indices of cell c at degree k, local order
        lexicographic x fastest."""
        k = self.k if k is None else k
        n1 = k * self.n + 1
        loc = np.arange(k + 1)
        idx = np.zeros(1, dtype=np.int64)
        stride = 1
        for dd in range(self.d):
            g = k * c[dd] + loc
            idx = (idx[None, :] + stride * g[:, None]).reshape(-1)
            stride *= n1
        return idx

    # ---- geometry -------------------------------------------------------
    def map_and_jacobian(self, X):
        """F(X) and dF/dX at points X (shape (..., d))."""
        X = np.asarray(X, dtype=np.float64)
        d = self.d
        if self.geometry == "cartesian":
            J = np.broadcast_to(np.eye(d), X.shape[:-1] + (d, d)).copy()
            return X.copy(), J
        if self.geometry == "distorted":
            return self._trilinear_map(X)
        s = np.sin(2 * np.pi * X)
        c = np.cos(2 * np.pi * X)
        prod = np.prod(s, axis=-1)
        x = X + self.amp * prod[..., None]
        J = np.broadcast_to(np.eye(d), X.shape[:-1] + (d, d)).copy()
        for j in range(d):
            others = np.ones(X.shape[:-1])
            for m in range(d):
                if m != j:
                    others = others * s[..., m]
            # dF_i / dX_j = delta_ij + a 2 pi cos(2 pi X_j) prod_{m != j} sin(2 pi X_m)
            J[..., :, j] += self.amp * 2 * np.pi * c[..., j][..., None] * others[..., None]
        return x, J

    def vertex_position(self, v):
        """Physical position of vertex v (integer index per direction) of this
        level: the reference position plus the displacement of the fine
        vertex at the same place."""
        stride = self.n_fine // self.n
        vf = [vi * stride for vi in v]
        flat = sum(vf[m] * (self.n_fine + 1) ** m for m in range(self.d))
        return np.asarray(v, dtype=np.float64) / self.n + self.disp[flat]

    def _trilinear_map(self, X):
        """x(X) and dx/dX for the trilinear cells: in cell c (the one holding
        X; the map is continuous across cells), xi = n X - c in [0, 1]^d and
        x = sum over the 2^d corners s of prod_m N_{s_m}(xi_m) P_{c+s} with
        N_0(t) = 1 - t, N_1(t) = t; dx/dX = n dx/dxi.  All points at once."""
        d = self.d
        shape = X.shape[:-1]
        Xf = X.reshape(-1, d)
        c = np.minimum(np.floor(Xf * self.n).astype(np.int64), self.n - 1)
        xi = Xf * self.n - c
        stride = self.n_fine // self.n
        x = np.zeros_like(Xf)
        J = np.zeros((Xf.shape[0], d, d))
        for s in itertools.product(*([(0, 1)] * d)):
            v = c + np.array(s)
            flat = sum(v[:, m] * stride * (self.n_fine + 1) ** m for m in range(d))
            P = v / self.n + self.disp[flat]                  # displaced corner positions
            N = [xi[:, m] if s[m] else 1.0 - xi[:, m] for m in range(d)]
            x += np.prod(N, axis=0)[:, None] * P
            for j in range(d):
                g = self.n * (1.0 if s[j] else -1.0) * np.prod([N[m] for m in range(d) if m != j], axis=0)
                J[:, :, j] += g[:, None] * P
        return x.reshape(shape + (d,)), J.reshape(shape + (d, d))

    def cell_quadrature(self, c, nq):
        """Reference tensor Gauss points of cell c: returns (X points (Q, d),
        weights (Q,)) with x fastest."""
        xq, wq = gauss_legendre(nq)
        pts = np.array(list(itertools.product(*([xq] * self.d)[::-1])))[:, ::-1]
        w = np.prod(np.array(list(itertools.product(*([wq] * self.d)[::-1]))), axis=1)
        X = self.h * (np.asarray(c, dtype=np.float64)[None, :] + pts)
        return pts, X, w

    def cell_geometry(self, c, nq):
        """Per quadrature point of cell c: G_q = w_q det(J) J^{-1} J^{-T} with
        J = dx/dxi = (dF/dX) h, the tensor of the transformed gradient form
        of Eq. (3).  Rounded to float32 (then read back as float64) when the
        mesh stores its geometry in float32."""
        _, X, w = self.cell_quadrature(c, nq)
        _, DF = self.map_and_jacobian(X)
        J = DF * self.h
        detJ = np.linalg.det(J)
        Jinv = np.linalg.inv(J)
        G = w[:, None, None] * detJ[:, None, None] * np.einsum("qij,qkj->qik", Jinv, Jinv)
        if self.geom_fp32:
            G = G.astype(np.float32).astype(np.float64)
        return G


@functools.lru_cache(maxsize=None)
def _tensor_basis(k, nq, d):
    """Values and reference gradients of the tensor Q_k basis at the tensor
    Gauss points: Phi (Q, n_loc) and Grad (d, Q, n_loc), x fastest."""
    xq, _ = gauss_legendre(nq)
    nodes = gauss_lobatto_nodes(k)
    V = lagrange_values(nodes, xq)
    D = lagrange_derivatives(nodes, xq)

    def kron_list(mats):  # mats[0] acts on x (fastest)
        out = mats[-1]
        for m in mats[-2::-1]:
            out = np.kron(out, m)
        return out

    Phi = kron_list([V] * d)
    Grad = []
    for i in range(d):
        mats = [V] * d
        mats = list(mats)
        mats[i] = D
        Grad.append(kron_list(mats))
    Grad = np.array(Grad)
    Phi.flags.writeable = False  # memoised: shared by every cell
    Grad.flags.writeable = False
    return Phi, Grad


def element_stiffness(mesh, c, k=None):
    """Element matrix K^c_ab = sum_q grad phi_a(xi_q)^T G_q grad phi_b(xi_q)
    (Eq. (3) mapped to the reference cell), k+1 Gauss points per direction."""
    k = mesh.k if k is None else k
    nq = k + 1
    _, Grad = _tensor_basis(k, nq, mesh.d)
    G = mesh.cell_geometry(c, nq)
    n_loc = Grad.shape[2]
    K = np.zeros((n_loc, n_loc))
    for i in range(mesh.d):
        for j in range(mesh.d):
            K += Grad[i].T @ (G[:, i, j][:, None] * Grad[j])
    return K


def assemble_full(mesh, k=None):
    """Assembled stiffness on ALL (k n + 1)^d DoFs (no boundary condition), CSR."""
    k = mesh.k if k is None else k
    rows, cols, vals = [], [], []
    for c in mesh.cells():
        idx = mesh.cell_dofs(c, k)
        Ke = element_stiffness(mesh, c, k)
        rows.append(np.repeat(idx, len(idx)))
        cols.append(np.tile(idx, len(idx)))
        vals.append(Ke.reshape(-1))
    n1 = k * mesh.n + 1
    N = n1 ** mesh.d
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N)).tocsr()
    A.sum_duplicates()
    return A


def assemble(mesh):
    """A_l of Eq. (4) restricted to the free DoFs (Dirichlet rows and columns
    dropped), CSR, indexed by ``mesh.interior_index()``."""
    A = assemble_full(mesh)
    I = mesh.interior_index()
    return A[I][:, I].tocsr()


def apply_full(mesh, A_int, x_full):
    """y = A x on full-length vectors with y_B = 0 (boundary inputs ignored)."""
    I = mesh.interior_index()
    y = np.zeros(mesh.n_dofs)
    y[I] = A_int @ np.asarray(x_full, dtype=np.float64)[I]
    return y


def kron_stiffness_cartesian(mesh):
    """Second, independent construction for Cartesian meshes:
    A = h^{d-2} sum_i (M x ... x K_i x ... x M) from the assembled 1D
    reference matrices.  Used only to pin ``assemble``."""
    from .quadrature import reference_matrices_1d
    k, n = mesh.k, mesh.n
    Me, Ke = reference_matrices_1d(k)
    n1 = k * n + 1
    M1 = np.zeros((n1, n1))
    K1 = np.zeros((n1, n1))
    for c in range(n):
        s = slice(k * c, k * c + k + 1)
        M1[s, s] += Me
        K1[s, s] += Ke
    # physical 1D: M scales with h, K with 1/h  -> product h^{d-2}
    terms = []
    for i in range(mesh.d):
        mats = [M1] * mesh.d
        mats = list(mats)
        mats[i] = K1
        out = mats[-1]
        for m in mats[-2::-1]:
            out = np.kron(out, m)
        terms.append(out)
    A = mesh.h ** (mesh.d - 2) * sum(terms)
    I = mesh.interior_index()
    return sp.csr_matrix(A[np.ix_(I, I)])


def dof_coordinates(mesh, k=None):
    """Physical coordinates of all DoF nodes (N, d), x fastest."""
    k = mesh.k if k is None else k
    nodes = gauss_lobatto_nodes(k)
    n1 = k * mesh.n + 1
    g = np.arange(n1)
    X1 = mesh.h * (np.minimum(g // k, mesh.n - 1) + nodes[g - k * np.minimum(g // k, mesh.n - 1)])
    grids = np.meshgrid(*([X1] * mesh.d), indexing="ij")  # grids[0] slowest
    X = np.stack([gr.reshape(-1) for gr in grids[::-1]], axis=1)  # column 0 = x
    x, _ = mesh.map_and_jacobian(X)
    return x


def manufactured_u(x):
    """u(x) = prod_i sin(pi x_i)."""
    return np.prod(np.sin(np.pi * x), axis=-1)


def manufactured_f(x):
    """f = -Laplace u = d pi^2 prod_i sin(pi x_i)."""
    d = x.shape[-1]
    return d * np.pi ** 2 * manufactured_u(x)


def rhs_manufactured(mesh):
    """b_a = sum_q f(F(X_q)) phi_a(xi_q) w_q det J_q on the full-length grid
    (boundary entries set to 0).  Geometry in float64 (no rounding)."""
    k = mesh.k
    nq = k + 1
    Phi, _ = _tensor_basis(k, nq, mesh.d)
    b = np.zeros(mesh.n_dofs)
    for c in mesh.cells():
        _, X, w = mesh.cell_quadrature(c, nq)
        x, DF = mesh.map_and_jacobian(X)
        detJ = np.linalg.det(DF * mesh.h)
        fq = manufactured_f(x) * w * detJ
        np.add.at(b, mesh.cell_dofs(c), Phi.T @ fq)
    b[~mesh.interior_mask()] = 0.0
    return b


def l2_error_manufactured(mesh, u_full):
    """|| u_h - u ||_{L2}, with (k+3) Gauss points per direction."""
    k = mesh.k
    nq = k + 3
    Phi, _ = _tensor_basis(k, nq, mesh.d)
    err2 = 0.0
    for c in mesh.cells():
        _, X, w = mesh.cell_quadrature(c, nq)
        x, DF = mesh.map_and_jacobian(X)
        detJ = np.linalg.det(DF * mesh.h)
        uh = Phi @ u_full[mesh.cell_dofs(c)]
        err2 += np.sum((uh - manufactured_u(x)) ** 2 * w * detJ)
    return float(np.sqrt(err2))


def prolongation_1d(k, n_coarse):
    """Global 1D embedding from n_coarse cells to 2 n_coarse cells, degree k:
    P[g_f, g_c] = coarse basis function g_c evaluated at fine node g_f
    (reference coordinates: child ch of coarse cell cc maps xi to (ch + xi)/2)."""
    nodes = gauss_lobatto_nodes(k)
    nf = 2 * n_coarse
    n1f, n1c = k * nf + 1, k * n_coarse + 1
    P = np.zeros((n1f, n1c))
    for gf in range(n1f):
        cf = min(gf // k, nf - 1)
        a = gf - k * cf
        cc = cf // 2
        eta = ((cf % 2) + nodes[a]) / 2.0
        vals = lagrange_values(nodes, eta)[0]
        for b in range(k + 1):
            P[gf, k * cc + b] = vals[b]
    P[np.abs(P) < 1e-15] = 0.0
    return P


def prolongation(mesh_coarse):
    """P_l: V_{l-1} -> V_l (Eq. (2), the embedding) as a sparse matrix on the
    free DoFs: Kronecker product of the 1D embeddings, boundary rows and
    columns dropped.  The restriction is its transpose."""
    d, k, nc = mesh_coarse.d, mesh_coarse.k, mesh_coarse.n
    P1 = sp.csr_matrix(prolongation_1d(k, nc))
    P = P1
    for _ in range(d - 1):
        P = sp.kron(P1, P, format="csr")
    fine = mesh_coarse.with_level(n=2 * nc)
    If = fine.interior_index()
    Ic = mesh_coarse.interior_index()
    return P[If][:, Ic].tocsr()
