// Compile-time structure shared by the kernels and the host set-up of the
// p-multigrid vertex-patch library: the degree hierarchy of the local
// p-multigrid (§2.2: 1, 3, 7, ... capped at the target degree), patch sizes,
// structural zeros of the 1D patch and transfer matrices, and the layout of
// the per-degree coefficient block that lives in __constant__ memory.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pmg {

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// Number of p-levels for target degree K: every 2^l - 1 below K, then K.
__host__ __device__ constexpr int nlev(int K) {
  int n = 0;
  for (int p = 1; p < K; p = 2 * p + 1) ++n;
  return n + 1;
}
// Degree of p-level l (0 = coarsest = 1).
__host__ __device__ constexpr int plev(int K, int l) {
  return l == nlev(K) - 1 ? K : (1 << (l + 1)) - 1;
}
// Patch-interior points per direction at degree p.
__host__ __device__ constexpr int mp(int p) { return 2 * p - 1; }
// Row pitch of a shared-memory tile whose rows hold e values: e rounded up
// to odd, so that rows (and planes of an even number of rows) start on
// different banks.
__host__ __device__ constexpr int tpitch(int e) { return e | 1; }

// Patch-interior node i (0..2p-2) of degree p: 0 = strictly in the first
// cell, 1 = the patch centre (shared), 2 = strictly in the second cell.
__host__ __device__ constexpr int node_side(int p, int i) { return i < p - 1 ? 0 : (i == p - 1 ? 1 : 2); }
// Entry (i, j) of a patch matrix (degree p rows, degree q columns) can be
// non-zero only if the two nodes share a cell.
__host__ __device__ constexpr bool pnz(int p, int q, int i, int j) {
  return !((node_side(p, i) == 0 && node_side(q, j) == 2) || (node_side(p, i) == 2 && node_side(q, j) == 0));
}

// ---------------------------------------------------------------------------
// Coefficient block for degree K (doubles; a float copy mirrors it):
//   Me, Ke        (K+1)^2   reference 1D mass / stiffness on [0,1]
//   Pt            2 (K+1)^2 h-prolongation: Pt[ch][i][a] = phi_a((ch + xi_i)/2)
//   per level l = 0..nlev-1 (p = plev(K,l)):
//     S           (p+1)^2   GLL -> Gauss interpolation (rows = Gauss points)
//     Dq          (p+1)^2   derivative at Gauss points of the Gauss-point
//                           Lagrange basis (collocation derivative)
//     W           (p+1)     Gauss weights
//   per level l = 1..nlev-1 (m = 2p-1, mc = m of level l-1):
//     MP, KP      m^2       patch-interior 1D mass / stiffness (two cells)
//     dM, dK      m         their diagonals
//     Tr          m * mc    p-transfer (prolongation) from level l-1
//   level 0 (p = 1): dM0 = 2/3, dK0 = 2 (the 1x1 patch matrices)
// ---------------------------------------------------------------------------
struct CoefLayout {
  int Me, Ke, Pt;
  int MP[4], KP[4], dM[4], dK[4], Tr[4], S[4], Dq[4], W[4];
  int dM0, dK0;
  int total;
};

__host__ __device__ constexpr CoefLayout coef_layout(int K) {
  CoefLayout L{};
  int o = 0;
  L.Me = o; o += (K + 1) * (K + 1);
  L.Ke = o; o += (K + 1) * (K + 1);
  L.Pt = o; o += 2 * (K + 1) * (K + 1);
  for (int l = 0; l < 4; ++l) { L.MP[l] = L.KP[l] = L.dM[l] = L.dK[l] = L.Tr[l] = L.S[l] = L.Dq[l] = L.W[l] = 0; }
  for (int l = 0; l < nlev(K); ++l) {
    const int p = plev(K, l);
    L.S[l] = o; o += (p + 1) * (p + 1);
    L.Dq[l] = o; o += (p + 1) * (p + 1);
    L.W[l] = o; o += p + 1;
  }
  for (int l = 1; l < nlev(K); ++l) {
    const int p = plev(K, l), m = mp(p), mc = mp(plev(K, l - 1));
    L.MP[l] = o; o += m * m;
    L.KP[l] = o; o += m * m;
    L.dM[l] = o; o += m;
    L.dK[l] = o; o += m;
    L.Tr[l] = o; o += m * mc;
  }
  L.dM0 = o; o += 1;
  L.dK0 = o; o += 1;
  L.total = o;
  return L;
}

constexpr int kMaxCoef = 2048;   // >= coef_layout(8).total
// Dynamic shared memory any kernel of the library may request: the 227 KB
// per-block opt-in of sm_103a minus room for the kernels' static arrays.
constexpr int kMaxDynSmem = 220 * 1024;

// Unsigned 32-bit division by a divisor fixed for a launch, by multiplying
// with a precomputed reciprocal (Granlund and Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994, unsigned case):
// l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1, then for any 32-bit n
// t = mulhi(m, n) and n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0).
// The grid-stride line kernels decode their item index with it instead of
// 64-bit division (tens of instructions per divide).  1 <= d < 2^31.
struct FastDiv {
  uint32_t d, m, s1, s2;
  __host__ __device__ FastDiv() : d(1), m(1), s1(0), s2(0) {}
  __host__ explicit FastDiv(uint32_t d_) : d(d_) {
    uint32_t l = 0;
    while (l < 31 && (uint64_t(1) << l) < d) ++l;
    m = (uint32_t)((((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d) + 1);
    s1 = l < 1 ? l : 1;
    s2 = l > 1 ? l - 1 : 0;
  }
  __host__ __device__ __forceinline__ uint32_t div(uint32_t n) const {
#ifdef __CUDA_ARCH__
    const uint32_t t = __umulhi(m, n);
#else
    const uint32_t t = (uint32_t)(((uint64_t)m * n) >> 32);
#endif
    return (t + ((n - t) >> s1)) >> s2;
  }
};
// work items of a grid-stride loop that the 32-bit decoding covers
constexpr int64_t kFastDivItems = int64_t(1) << 32;

// Argument table of a grouped launch: one kernel launch does the work of up
// to kMaxGroup jobs (the same operation on the vectors of different systems,
// possibly of different sizes), passed by value as a __grid_constant__
// kernel parameter (no device copy of the table, so graph capture needs no
// allocation either).
// Element-wise and line kernels spread the concatenation of the jobs' work
// items over the grid (start: prefix sums of the items per job), so that a
// thread handles about one item, as in an ungrouped launch.
constexpr int kMaxGroup = 32;
template <class J>
struct GroupOf {
  int count;
  int64_t start[kMaxGroup + 1];
  J job[kMaxGroup];
};

// the job that global work item t belongs to (binary search in start)
template <class J>
__device__ __forceinline__ int group_find(const GroupOf<J>& G, int64_t t) {
  int lo = 0, hi = G.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (G.start[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// A grid-stride step that ends a body's loop after its first item: the
// grouped kernels call the ungrouped bodies one item at a time.
constexpr int64_t kOneItem = int64_t(1) << 62;

// Per-call scalars of the patch smoother (host fills, passed by value).
template <typename T>
struct PatchParams {
  T scale;        // h^{d-2}: Cartesian stiffness scale on this level
  T omega_as;     // additive-Schwarz damping
  T omega[4];     // Jacobi damping per p-level
  T inv_a0;       // 1 / A_{j,1} on Cartesian meshes (uniform)
  T inv_scale;    // 1 / scale
  int half;       // 1: half local V-cycle (post-smoothing dropped, §3.2.2)
  int colour;     // -1: all patches (additive); c >= 0: patches of parity colour c
};

// Interior vertices (patches) of a level with n cells per side: all (n-1)^d,
// or those of parity colour c (bit d of c = parity of the d-th vertex index;
// odd indices 1, 3, ... number n / 2, even ones 2, 4, ... (n - 1) / 2).
__host__ __device__ inline int patch_count_1d(int n, int colour, int d) {
  if (colour < 0) return n - 1;
  return ((colour >> d) & 1) ? n / 2 : (n - 1) / 2;
}
__host__ __device__ inline int64_t patch_count(int dim, int n, int colour) {
  int64_t c = 1;
  for (int d = 0; d < dim; ++d) c *= patch_count_1d(n, colour, d);
  return n < 2 ? 0 : c;
}

}  // namespace pmg
