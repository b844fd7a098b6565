// Host-side numerical set-up of the library (float64 / long double):
// 1D Gauss-Lobatto nodes and Gauss rules, Lagrange bases, the reference and
// patch 1D matrices, p-transfers and h-prolongation tables that fill the
// per-degree coefficient block, and the default Jacobi damping per p-level.
//
// The nodal Q_k basis on Gauss-Lobatto points and (k+1)-point Gauss
// quadrature are the discretisation of the bilinear form of Eq. (3); the
// patch matrices are those of the patch operator A_{j,p} on a Cartesian
// vertex patch (§2.1, §3.2); the p-transfers are the embedding of degree
// q into degree p on the patch interior (§3.2).
#include "setup.h"

#include <cmath>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "pmg_common.cuh"

namespace pmg {
namespace host {

using LD = long double;

static void legendre(int n, LD x, LD& pn, LD& pm) {
  LD p0 = 1, p1 = x;
  if (n == 0) { pn = 1; pm = 0; return; }
  for (int j = 2; j <= n; ++j) {
    LD p2 = ((2 * j - 1) * x * p1 - (j - 1) * p0) / j;
    p0 = p1;
    p1 = p2;
  }
  pn = p1;
  pm = p0;
}

std::vector<double> gauss_points(int n, std::vector<double>* weights) {
  std::vector<LD> x(n), w(n);
  const LD pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < n; ++i) {
    LD z = std::cos(pi * (i + 0.75L) / (n + 0.5L));
    for (int it = 0; it < 100; ++it) {
      LD pn, pm;
      legendre(n, z, pn, pm);
      LD dp = n * (pm - z * pn) / (1 - z * z);
      LD dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-30L) break;
    }
    LD pn, pm;
    legendre(n, z, pn, pm);
    LD dp = n * (pm - z * pn) / (1 - z * z);
    x[i] = z;
    w[i] = 2 / ((1 - z * z) * dp * dp);
  }
  // ascending order on [0, 1]
  std::vector<double> out(n);
  if (weights) weights->assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    int j = n - 1 - i;  // roots came out descending
    out[i] = double((x[j] + 1) / 2);
    if (weights) (*weights)[i] = double(w[j] / 2);
  }
  return out;
}

std::vector<double> gll_points(int k) {
  std::vector<double> out(k + 1);
  out[0] = 0.0;
  out[k] = 1.0;
  const LD pi = 3.141592653589793238462643383279502884L;
  for (int i = 1; i < k; ++i) {
    LD z = -std::cos(pi * i / k);
    for (int it = 0; it < 100; ++it) {
      LD pk, pm;
      legendre(k, z, pk, pm);
      LD d1 = k * (pm - z * pk) / (1 - z * z);
      LD d2 = (2 * z * d1 - k * (k + 1) * pk) / (1 - z * z);
      LD dz = d1 / d2;
      z -= dz;
      if (std::fabs(dz) < 1e-30L) break;
    }
    out[i] = double((z + 1) / 2);
  }
  return out;
}

double lagrange(const std::vector<double>& nodes, int a, double x) {
  LD v = 1;
  for (size_t b = 0; b < nodes.size(); ++b)
    if ((int)b != a) v *= (LD(x) - nodes[b]) / (LD(nodes[a]) - nodes[b]);
  return double(v);
}

double lagrange_deriv(const std::vector<double>& nodes, int a, double x) {
  LD s = 0;
  for (size_t c = 0; c < nodes.size(); ++c) {
    if ((int)c == a) continue;
    LD t = 1 / (LD(nodes[a]) - nodes[c]);
    for (size_t b = 0; b < nodes.size(); ++b)
      if ((int)b != a && b != c) t *= (LD(x) - nodes[b]) / (LD(nodes[a]) - nodes[b]);
    s += t;
  }
  return double(s);
}

// Reference 1D mass and stiffness of degree p on [0, 1] with p+1 Gauss points.
void reference_1d(int p, std::vector<double>& M, std::vector<double>& Kst) {
  std::vector<double> w;
  auto xq = gauss_points(p + 1, &w);
  auto nd = gll_points(p);
  const int n = p + 1;
  M.assign(n * n, 0.0);
  Kst.assign(n * n, 0.0);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      LD m = 0, k = 0;
      for (int q = 0; q < n; ++q) {
        m += LD(w[q]) * lagrange(nd, a, xq[q]) * lagrange(nd, b, xq[q]);
        k += LD(w[q]) * lagrange_deriv(nd, a, xq[q]) * lagrange_deriv(nd, b, xq[q]);
      }
      M[a * n + b] = double(m);
      Kst[a * n + b] = double(k);
    }
}

// Patch-interior 1D matrices: assemble the degree-p reference matrices over
// the two cells of a patch and keep the 2p-1 interior nodes.
void patch_1d(int p, std::vector<double>& MP, std::vector<double>& KP) {
  std::vector<double> M, Kst;
  reference_1d(p, M, Kst);
  const int full = 2 * p + 1, m = 2 * p - 1, n = p + 1;
  std::vector<double> Mf(full * full, 0.0), Kf(full * full, 0.0);
  for (int c = 0; c < 2; ++c)
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        Mf[(p * c + a) * full + p * c + b] += M[a * n + b];
        Kf[(p * c + a) * full + p * c + b] += Kst[a * n + b];
      }
  MP.assign(m * m, 0.0);
  KP.assign(m * m, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      MP[i * m + j] = Mf[(i + 1) * full + j + 1];
      KP[i * m + j] = Kf[(i + 1) * full + j + 1];
    }
}

// Prolongation of the degree-q patch-interior basis to the degree-p
// interior nodes: T[i][j] = psi_j(s_i), (2p-1) x (2q-1).
std::vector<double> p_transfer(int q, int p) {
  auto nq = gll_points(q), np = gll_points(p);
  const int m = 2 * p - 1, mc = 2 * q - 1;
  std::vector<double> T(m * mc, 0.0);
  for (int i = 0; i < m; ++i) {
    double s = i < p ? np[i + 1] : 1.0 + np[i - p + 1];
    for (int cell = 0; cell < 2; ++cell) {
      if (s < cell || s > cell + 1) continue;
      for (int a = 0; a <= q; ++a) {
        int node = q * cell + a - 1;
        if (node < 0 || node >= mc) continue;
        double v = lagrange(nq, a, s - cell);
        if (std::fabs(v) < 1e-15) v = 0.0;
        T[i * mc + node] = v;
      }
    }
  }
  return T;
}

// Lanczos estimate of lambda_max(D^{-1} A) for the Cartesian patch operator
// A = sum_dir (KP on dir, MP elsewhere) at degree p in dimension d.
static double lambda_max_patch(int d, int p) {
  if (p == 1) return 1.0;
  std::vector<double> MP, KP;
  patch_1d(p, MP, KP);
  const int m = 2 * p - 1;
  const int N = d == 2 ? m * m : m * m * m;
  std::vector<double> diag(N);
  auto idx = [&](int i, int dd) { return dd == 0 ? i % m : (dd == 1 ? (i / m) % m : i / (m * m)); };
  for (int i = 0; i < N; ++i) {
    double s = 0;
    for (int dir = 0; dir < d; ++dir) {
      double t = 1;
      for (int dd = 0; dd < d; ++dd) {
        int ii = idx(i, dd);
        t *= dd == dir ? KP[ii * m + ii] : MP[ii * m + ii];
      }
      s += t;
    }
    diag[i] = s;
  }
  // y_axis = C applied along one axis of an m^d tensor (x fastest)
  auto along = [&](const std::vector<double>& in, std::vector<double>& out, const std::vector<double>& C,
                   int axis) {
    const int stride = axis == 0 ? 1 : (axis == 1 ? m : m * m);
    for (int i = 0; i < N; ++i) {
      const int ii = idx(i, axis);
      const int base = i - ii * stride;
      double s = 0;
      for (int j = 0; j < m; ++j) s += C[ii * m + j] * in[base + j * stride];
      out[i] = s;
    }
  };
  auto matvec = [&](const std::vector<double>& x, std::vector<double>& y) {
    // y = D^{-1/2} A D^{-1/2} x with A = sum_dir (KP on dir, MP elsewhere)
    std::vector<double> xs(N), t(N), u(N);
    for (int i = 0; i < N; ++i) xs[i] = x[i] / std::sqrt(diag[i]);
    std::fill(y.begin(), y.end(), 0.0);
    for (int dir = 0; dir < d; ++dir) {
      t = xs;
      for (int ax = 0; ax < d; ++ax) {
        along(t, u, ax == dir ? KP : MP, ax);
        t.swap(u);
      }
      for (int i = 0; i < N; ++i) y[i] += t[i];
    }
    for (int i = 0; i < N; ++i) y[i] /= std::sqrt(diag[i]);
  };
  const int steps = std::min(N, 60);
  std::vector<std::vector<double>> V;
  std::vector<double> alpha, beta;
  std::vector<double> v(N), w(N);
  for (int i = 0; i < N; ++i) v[i] = 1.0 + 0.37 * std::sin(1.3 * i + 0.1);
  double nv = 0;
  for (double t : v) nv += t * t;
  nv = std::sqrt(nv);
  for (double& t : v) t /= nv;
  double amax = 0;
  for (int j = 0; j < steps; ++j) {
    V.push_back(v);
    matvec(v, w);
    double a = 0;
    for (int i = 0; i < N; ++i) a += w[i] * v[i];
    alpha.push_back(a);
    for (int pass = 0; pass < 2; ++pass)  // full re-orthogonalisation, twice
      for (auto& q : V) {
        double c = 0;
        for (int i = 0; i < N; ++i) c += w[i] * q[i];
        for (int i = 0; i < N; ++i) w[i] -= c * q[i];
      }
    double b = 0;
    for (double t : w) b += t * t;
    b = std::sqrt(b);
    amax = std::max(amax, std::fabs(a));
    // an invariant Krylov subspace (repeated eigenvalues of the symmetric
    // patch) ends the recurrence: its Ritz values are then exact
    if (b < 1e-10 * amax || j == steps - 1) break;
    beta.push_back(b);
    for (int i = 0; i < N; ++i) v[i] = w[i] / b;
  }
  // largest eigenvalue of the tridiagonal matrix by Sturm bisection
  const int n = (int)alpha.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < n; ++i) {
    double r = (i > 0 ? std::fabs(beta[i - 1]) : 0) + (i < n - 1 ? std::fabs(beta[i]) : 0);
    lo = std::min(lo, alpha[i] - r);
    hi = std::max(hi, alpha[i] + r);
  }
  auto count_below = [&](double x) {
    int c = 0;
    double q = alpha[0] - x;
    if (q < 0) ++c;
    for (int i = 1; i < n; ++i) {
      if (q == 0) q = 1e-300;
      q = alpha[i] - x - beta[i - 1] * beta[i - 1] / q;
      if (q < 0) ++c;
    }
    return c;
  };
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= n) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

double default_omega_jacobi(int d, int p) {
  static std::mutex mu;
  static double cache[4][16] = {};
  std::lock_guard<std::mutex> g(mu);
  double& c = cache[d][p];
  if (c == 0.0) c = p == 1 ? 1.0 : 4.0 / (3.0 * lambda_max_patch(d, p));
  return c;
}

void fill_coefficients(int K, double* out) {
  const CoefLayout L = coef_layout(K);
  std::memset(out, 0, sizeof(double) * L.total);
  std::vector<double> M, Kst;
  reference_1d(K, M, Kst);
  for (int i = 0; i < (K + 1) * (K + 1); ++i) {
    out[L.Me + i] = M[i];
    out[L.Ke + i] = Kst[i];
  }
  auto nd = gll_points(K);
  for (int ch = 0; ch < 2; ++ch)
    for (int i = 0; i <= K; ++i)
      for (int a = 0; a <= K; ++a) {
        double v = lagrange(nd, a, (ch + nd[i]) / 2.0);
        if (std::fabs(v) < 1e-15) v = 0.0;
        out[L.Pt + (ch * (K + 1) + i) * (K + 1) + a] = v;
      }
  for (int l = 1; l < nlev(K); ++l) {
    const int p = plev(K, l), m = mp(p), q = plev(K, l - 1), mc = mp(q);
    std::vector<double> MP, KP;
    patch_1d(p, MP, KP);
    for (int i = 0; i < m * m; ++i) {
      out[L.MP[l] + i] = MP[i];
      out[L.KP[l] + i] = KP[i];
    }
    for (int i = 0; i < m; ++i) {
      out[L.dM[l] + i] = MP[i * m + i];
      out[L.dK[l] + i] = KP[i * m + i];
    }
    auto T = p_transfer(q, p);
    for (int i = 0; i < m * mc; ++i) out[L.Tr[l] + i] = T[i];
  }
  for (int l = 0; l < nlev(K); ++l) {
    const int p = plev(K, l);
    std::vector<double> S, Dq, W;
    cell_tables(p, S, Dq, W);
    for (int i = 0; i < (p + 1) * (p + 1); ++i) {
      out[L.S[l] + i] = S[i];
      out[L.Dq[l] + i] = Dq[i];
    }
    for (int a = 0; a <= p; ++a) out[L.W[l] + a] = W[a];
  }
  out[L.dM0] = 2.0 / 3.0;
  out[L.dK0] = 2.0;
}

// Global-fine-level variants of S / Dq / W for degree K (used by the cell
// operator of the deformed apply); same formulas as the level-top entries.
void cell_tables(int p, std::vector<double>& S, std::vector<double>& Dq, std::vector<double>& W) {
  auto xq = gauss_points(p + 1, &W);
  auto np = gll_points(p);
  S.assign((p + 1) * (p + 1), 0.0);
  Dq.assign((p + 1) * (p + 1), 0.0);
  for (int a = 0; a <= p; ++a)
    for (int b = 0; b <= p; ++b) {
      S[a * (p + 1) + b] = lagrange(np, b, xq[a]);
      Dq[a * (p + 1) + b] = lagrange_deriv(xq, b, xq[a]);
    }
}

}  // namespace host
}  // namespace pmg
