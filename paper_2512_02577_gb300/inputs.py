"""Seeded synthetic inputs shared by the tests and the benchmark.

Holds none of the method's arithmetic: only random vectors on the nodal
grid (standard normal on the free nodes, zero on the boundary, the i.i.d.
N(0,1) right-hand sides of the degree-sweep and serving workloads) and the
serving workload recipe (Poisson arrivals, log-uniform mesh sizes, uniform
degrees).  The same vector is handed to the oracle and to the library.
"""
import numpy as np


def interior_mask(dim, n, k):
    n1 = k * n + 1
    g = np.arange(n1)
    m1 = (g > 0) & (g < n1 - 1)
    m = m1
    for _ in range(dim - 1):
        m = np.multiply.outer(m1, m)
    return m.reshape(-1)


def random_vector(dim, n, k, seed):
    """N(0,1) on the free nodes of the (k n + 1)^dim grid, 0 on the boundary
    (numpy default_rng(seed), PCG64)."""
    rng = np.random.default_rng(seed)
    m = interior_mask(dim, n, k)
    v = np.zeros(m.size)
    v[m] = rng.standard_normal(int(m.sum()))
    return v


# Mesh sizes a served request may have: n = n_0 2^L with a coarse level
# small enough for the dense coarse solve ((k n_0 - 1)^3 <= 4096), i.e.
# n_0 = 3 allowed up to degree 5, only n_0 = 1 (powers of two) above.
SIZES_LOW_DEGREE = (8, 12, 16, 24, 32, 48, 64)
SIZES_HIGH_DEGREE = (8, 16, 32, 64)


def serving_requests(n_requests=256, rate=50.0, arrival_seed=7, size_seed=11, rhs_seed0=1000,
                     n_lo=8, n_hi=64, k_lo=2, k_hi=7, snap="pow2"):
    """Serving workload: Poisson arrivals at ``rate`` per second; cells per
    side log-uniform in [n_lo, n_hi], snapped in log space to the nearest
    allowed size: ``snap="pow2"`` a power of two (every mesh coarsens to one
    cell), ``snap="coarse"`` the sizes above (with n_0 = 3 meshes for
    k <= 5); degree uniform in k_lo..k_hi; right-hand-side seed rhs_seed0 + i.
    The degree is drawn before the size is snapped."""
    ra = np.random.default_rng(arrival_seed)
    rs = np.random.default_rng(size_seed)
    gaps = ra.exponential(1.0 / rate, n_requests)
    t = np.cumsum(gaps) - gaps[0]
    logn = rs.uniform(np.log2(n_lo), np.log2(n_hi), n_requests)
    ks = rs.integers(k_lo, k_hi + 1, n_requests)
    ns = []
    for ln, k in zip(logn, ks):
        if snap == "pow2":
            ns.append(int(2 ** np.round(ln)))
        else:
            allowed = [n for n in (SIZES_LOW_DEGREE if k <= 5 else SIZES_HIGH_DEGREE) if n_lo <= n <= n_hi]
            ns.append(min(allowed, key=lambda n: (abs(np.log2(n) - ln), n)))
    return [dict(id=i, t_arrival=float(t[i]), n=int(ns[i]), k=int(ks[i]), rhs_seed=rhs_seed0 + i)
            for i in range(n_requests)]


def vertex_displacements(dim, n, delta, seed):
    """Random mesh distortion of §3.2.2 / §4: every interior vertex of the
    n^d mesh of the unit square/cube moves by delta h_v in a random direction
    (uniform on the sphere: a normalised N(0, I) draw), h_v = 1/n being the
    shortest edge at the vertex; boundary vertices stay.  Returns
    ((n+1)^d, dim) float64, vertices lexicographic with x fastest."""
    rng = np.random.default_rng(seed)
    nv = (n + 1) ** dim
    g = rng.standard_normal((nv, dim))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    idx = np.arange(nv)
    interior = np.ones(nv, dtype=bool)
    for d in range(dim):
        c = (idx // (n + 1) ** d) % (n + 1)
        interior &= (c > 0) & (c < n)
    return np.where(interior[:, None], g * (delta / n), 0.0)
