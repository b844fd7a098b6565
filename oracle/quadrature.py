"""1D nodes, quadrature rules and Lagrange bases on the unit interval [0, 1].

The paper uses a tensor-product nodal Q_k basis and Gaussian quadrature for
the matrix-free operator (§3, sum factorisation of Eq. (3)); it names neither
the node set nor the rule.  Reading taken: Lagrange polynomials on the k+1
Gauss-Lobatto (GLL) points, and the (k+1)-point Gauss-Legendre rule, on every
p-level with p in place of k.

The rules are memoised (read-only arrays): the mesh code asks for the same
rule once per cell.

Pinned by tests against closed forms (k=2 nodes {0, 1/2, 1}; 2-point Gauss
1/2 -+ 1/(2 sqrt 3)), sum of weights = 1, exact integration of x^m for
m <= 2n-1, and agreement with numpy's leggauss.
"""
import functools

import numpy as np

_LD = np.longdouble


def _frozen(*arrays):
    for a in arrays:
        a.flags.writeable = False
    return arrays if len(arrays) > 1 else arrays[0]


def _legendre(n, x):
    """P_n(x) and P_{n-1}(x) by the three-term recurrence (x in [-1, 1])."""
    p0 = np.ones_like(x)
    if n == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    for j in range(2, n + 1):
        p0, p1 = p1, ((2 * j - 1) * x * p1 - (j - 1) * p0) / j
    return p1, p0


@functools.lru_cache(maxsize=None)
def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [0, 1]: (points, weights), ascending.

    Roots of P_n by Newton iteration in long double, started from the
    asymptotic guess cos(pi (i + 3/4) / (n + 1/2)); weights
    2 / ((1 - x^2) P_n'(x)^2) on [-1, 1], halved for [0, 1].
    """
    if n < 1:
        raise ValueError("n >= 1")
    i = np.arange(n, dtype=_LD)
    x = np.cos(_LD(np.pi) * (i + _LD(0.75)) / (n + _LD(0.5)))
    for _ in range(100):
        pn, pm = _legendre(n, x)
        dp = n * (pm - x * pn) / (1 - x * x)
        dx = pn / dp
        x = x - dx
        if np.max(np.abs(dx)) < _LD(1e-30):
            break
    pn, pm = _legendre(n, x)
    dp = n * (pm - x * pn) / (1 - x * x)
    w = 2 / ((1 - x * x) * dp * dp)
    order = np.argsort(x)
    x, w = x[order], w[order]
    return _frozen(np.asarray((x + 1) / 2, dtype=np.float64), np.asarray(w / 2, dtype=np.float64))


@functools.lru_cache(maxsize=None)
def gauss_lobatto_nodes(k):
    """The k+1 Gauss-Lobatto points on [0, 1] (endpoints included), ascending.

    Interior points are the roots of P_k'; found by Newton iteration in long
    double on P_k' with P_k'' from Legendre's equation
    (1 - x^2) P'' = 2 x P' - k (k + 1) P, started from the Chebyshev-Lobatto
    points -cos(pi i / k).
    """
    if k < 1:
        raise ValueError("k >= 1")
    if k == 1:
        return _frozen(np.array([0.0, 1.0]))
    i = np.arange(1, k, dtype=_LD)
    x = -np.cos(_LD(np.pi) * i / k)
    for _ in range(100):
        pk, pm = _legendre(k, x)
        d1 = k * (pm - x * pk) / (1 - x * x)
        d2 = (2 * x * d1 - k * (k + 1) * pk) / (1 - x * x)
        dx = d1 / d2
        x = x - dx
        if np.max(np.abs(dx)) < _LD(1e-30):
            break
    x = np.sort(x)
    full = np.concatenate([[_LD(-1)], x, [_LD(1)]])
    return _frozen(np.asarray((full + 1) / 2, dtype=np.float64))


def lagrange_values(nodes, x):
    """V[q, a] = phi_a(x_q) for the Lagrange basis on ``nodes``.

    phi_a(x) = prod_{b != a} (x - xi_b) / (xi_a - xi_b).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    V = np.ones((len(x), n))
    for a in range(n):
        for b in range(n):
            if b != a:
                V[:, a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
    return V


def lagrange_derivatives(nodes, x):
    """D[q, a] = phi_a'(x_q), by the product rule applied to phi_a:

    phi_a'(x) = sum_{c != a} 1/(xi_a - xi_c) prod_{b != a, c} (x - xi_b)/(xi_a - xi_b).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    D = np.zeros((len(x), n))
    for a in range(n):
        for c in range(n):
            if c == a:
                continue
            term = np.full(len(x), 1.0 / (nodes[a] - nodes[c]))
            for b in range(n):
                if b != a and b != c:
                    term *= (x - nodes[b]) / (nodes[a] - nodes[b])
            D[:, a] += term
    return D


def reference_matrices_1d(k, nq=None):
    """1D reference mass and stiffness on [0, 1] for the degree-k GLL basis:

    M_ab = sum_q w_q phi_a(x_q) phi_b(x_q),  K_ab = sum_q w_q phi_a'(x_q) phi_b'(x_q),
    with the nq-point Gauss rule (default k+1, exact for these integrands).
    """
    nq = k + 1 if nq is None else nq
    xq, wq = gauss_legendre(nq)
    nodes = gauss_lobatto_nodes(k)
    V = lagrange_values(nodes, xq)
    D = lagrange_derivatives(nodes, xq)
    M = V.T @ (wq[:, None] * V)
    K = D.T @ (wq[:, None] * D)
    return M, K
