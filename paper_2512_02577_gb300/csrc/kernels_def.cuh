// Deformed-geometry kernels for one degree K (included by inst_k.cuh after
// kernels.cuh).  The operator is the general sum-factorised form of Eq. (3):
// per cell, interpolate the nodal values from the Gauss-Lobatto nodes to the
// (p+1)^d Gauss points (d 1D contractions with S), take reference gradients
// by collocation derivatives at the Gauss points (Dq), multiply by the stored
// symmetric tensor G_q = w_q det J J^{-1} J^{-T} (stored in FP32 or FP64,
// §3's quadrature-point "evaluation kernel"), and apply the transposed steps.
// Cells of one parity colour share no node, so colour-by-colour launches
// accumulate without atomics and in a fixed order.
#pragma once
#include <algorithm>
#include <type_traits>

namespace pmg {
namespace PMG_KNS {

template <int DIM>
__host__ __device__ constexpr int ncomp() { return DIM == 3 ? 6 : 3; }

// y = C x (TR = false) or y = C^T x (TR = true) for an n x n row-major C.
template <int n, bool TR, typename T>
__device__ __forceinline__ void mvn(const T* C, const T* x, T* y) {
#pragma unroll
  for (int i = 0; i < n; ++i) {
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < n; ++j) acc += (TR ? C[j * n + i] : C[i * n + j]) * x[j];
    y[i] = acc;
  }
}

// Cell tiles of a block: item (g, c) -- group g (a patch, or one cell of the
// global apply), cell c < NC of the group -- owns 5 tiles of (p+1)^DIM
// values A0, A1, B0, B1, B2 at tile(g, c).  One axis contraction of every
// tile, the (item, line) pairs spread over the block's threads:
// dst = C src along AX (TR: C^T; ACC: dst += ...).
template <int DIM, int n, int NC, int AX, bool TR, bool ACC, typename T, class Tile>
__device__ __forceinline__ void tiles_axis(const T* C, int ng, const Tile& tile, int src, int dst) {
  constexpr int EZ = DIM == 3 ? n : 1;
  constexpr int nl = n * EZ;
  constexpr int st = AX == 0 ? 1 : (AX == 1 ? n : n * n);
  pfor_n<NC * nl>(ng, [&](int g, int t) {
    const int c = t / nl, L = t - c * nl;
    T* A = tile(g, c);
    const int b = line_base<AX, n, n, EZ>(L);
    T x[n], y[n];
#pragma unroll
    for (int j = 0; j < n; ++j) x[j] = A[src + b + j * st];
    mvn<n, TR>(C, x, y);
#pragma unroll
    for (int i = 0; i < n; ++i) {
      if (ACC) A[dst + b + i * st] += y[i];
      else A[dst + b + i * st] = y[i];
    }
  });
}

// Cell operator of p-level l on every tile of the block: A0 (nodal values
// in) -> A0 (cell contribution out); gptr(g, c) is the cell's tensor block
// [component][point].  Every thread of the block must call it.
template <int DIM, int l, int NC, typename T, class Tile, class GPtr>
__device__ __forceinline__ void cell_op(int ng, const Tile& tile, const GPtr& gptr) {
  constexpr int p = plev(K, l);
  constexpr int n1 = p + 1;
  constexpr int NP = ipow(n1, DIM);
  constexpr int A0 = 0, A1 = NP, B0 = 2 * NP, B1 = 3 * NP, B2 = 4 * NP;
  const T* Sm = ctab<T>() + LAY.S[l];
  const T* Dm = ctab<T>() + LAY.Dq[l];
  if constexpr (DIM == 3) {
    tiles_axis<3, n1, NC, 0, false, false>(Sm, ng, tile, A0, A1);
    __syncthreads();
    tiles_axis<3, n1, NC, 1, false, false>(Sm, ng, tile, A1, A0);
    __syncthreads();
    tiles_axis<3, n1, NC, 2, false, false>(Sm, ng, tile, A0, A1);
    __syncthreads();
    tiles_axis<3, n1, NC, 0, false, false>(Dm, ng, tile, A1, B0);
    tiles_axis<3, n1, NC, 1, false, false>(Dm, ng, tile, A1, B1);
    tiles_axis<3, n1, NC, 2, false, false>(Dm, ng, tile, A1, B2);
    __syncthreads();
    pfor_n<NC * NP>(ng, [&](int g, int t) {
      const int c = t / NP, q = t - c * NP;
      T* A = tile(g, c);
      const auto* Gc = gptr(g, c);
      const T g0 = A[B0 + q], g1 = A[B1 + q], g2 = A[B2 + q];
      const T G00 = (T)Gc[0 * NP + q], G01 = (T)Gc[1 * NP + q], G02 = (T)Gc[2 * NP + q];
      const T G11 = (T)Gc[3 * NP + q], G12 = (T)Gc[4 * NP + q], G22 = (T)Gc[5 * NP + q];
      A[B0 + q] = G00 * g0 + G01 * g1 + G02 * g2;
      A[B1 + q] = G01 * g0 + G11 * g1 + G12 * g2;
      A[B2 + q] = G02 * g0 + G12 * g1 + G22 * g2;
    });
    __syncthreads();
    tiles_axis<3, n1, NC, 0, true, false>(Dm, ng, tile, B0, A1);
    __syncthreads();
    tiles_axis<3, n1, NC, 1, true, true>(Dm, ng, tile, B1, A1);
    __syncthreads();
    tiles_axis<3, n1, NC, 2, true, true>(Dm, ng, tile, B2, A1);
    __syncthreads();
    tiles_axis<3, n1, NC, 2, true, false>(Sm, ng, tile, A1, A0);
    __syncthreads();
    tiles_axis<3, n1, NC, 1, true, false>(Sm, ng, tile, A0, A1);
    __syncthreads();
    tiles_axis<3, n1, NC, 0, true, false>(Sm, ng, tile, A1, A0);
    __syncthreads();
  } else {
    tiles_axis<2, n1, NC, 0, false, false>(Sm, ng, tile, A0, A1);
    __syncthreads();
    tiles_axis<2, n1, NC, 1, false, false>(Sm, ng, tile, A1, A0);
    __syncthreads();
    tiles_axis<2, n1, NC, 0, false, false>(Dm, ng, tile, A0, B0);
    tiles_axis<2, n1, NC, 1, false, false>(Dm, ng, tile, A0, B1);
    __syncthreads();
    pfor_n<NC * NP>(ng, [&](int g, int t) {
      const int c = t / NP, q = t - c * NP;
      T* A = tile(g, c);
      const auto* Gc = gptr(g, c);
      const T g0 = A[B0 + q], g1 = A[B1 + q];
      const T G00 = (T)Gc[0 * NP + q], G01 = (T)Gc[1 * NP + q], G11 = (T)Gc[2 * NP + q];
      A[B0 + q] = G00 * g0 + G01 * g1;
      A[B1 + q] = G01 * g0 + G11 * g1;
    });
    __syncthreads();
    tiles_axis<2, n1, NC, 0, true, false>(Dm, ng, tile, B0, A1);
    __syncthreads();
    tiles_axis<2, n1, NC, 1, true, true>(Dm, ng, tile, B1, A1);
    __syncthreads();
    tiles_axis<2, n1, NC, 1, true, false>(Sm, ng, tile, A1, A0);
    __syncthreads();
    tiles_axis<2, n1, NC, 0, true, false>(Sm, ng, tile, A0, A1);
    __syncthreads();
    pfor_n<NC * NP>(ng, [&](int g, int t) {
      const int c = t / NP, q = t - c * NP;
      T* A = tile(g, c);
      A[A0 + q] = A[A1 + q];
    });
    __syncthreads();
  }
}

// Global deformed apply, all cells in one launch: the cell results go to a
// per-cell buffer (cell-major, (K+1)^DIM values each) and cell_gather_kernel
// sums, per node, the contributions of the (at most 2^d) cells holding it in
// a fixed order.  `cpb` cells per block.  TG: storage type of G_q.
template <int DIM, typename T, typename TG>
__global__ void def_cell_kernel(const T* __restrict__ x, T* __restrict__ cellout, const TG* __restrict__ G, int n,
                                int cpb) {
  constexpr int l = nlev(K) - 1;
  constexpr int n1 = K + 1;
  constexpr int NP = ipow(n1, DIM);
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int cell_of[kMaxPatchesPerBlock][4];
  T* base = reinterpret_cast<T*>(smraw);
  const int64_t ncell = DIM == 3 ? (int64_t)n * n * n : (int64_t)n * n;
  for (int g = threadIdx.x; g < cpb; g += blockDim.x) {
    const int64_t cid = (int64_t)blockIdx.x * cpb + g;
    int64_t t = cid < ncell ? cid : 0;
    cell_of[g][0] = (int)(t % n);
    t /= n;
    cell_of[g][1] = (int)(t % n);
    cell_of[g][2] = DIM == 3 ? (int)(t / n) : 0;
    cell_of[g][3] = cid < ncell;
  }
  __syncthreads();
  const int N1 = K * n + 1;
  auto tile = [&](int g, int) { return base + g * 5 * NP; };
  pfor_n<NP>(cpb, [&](int g, int i) {
    const int ax = i % n1, ay = (i / n1) % n1, az = DIM == 3 ? i / (n1 * n1) : 0;
    const int gx = K * cell_of[g][0] + ax, gy = K * cell_of[g][1] + ay, gz = K * cell_of[g][2] + az;
    const bool bnd = gx == 0 || gx == N1 - 1 || gy == 0 || gy == N1 - 1 || (DIM == 3 && (gz == 0 || gz == N1 - 1));
    tile(g, 0)[i] = (cell_of[g][3] && !bnd) ? x[gx + (int64_t)N1 * (gy + (int64_t)N1 * gz)] : T(0);
  });
  __syncthreads();
  auto gptr = [&](int g, int) {
    const int64_t cell = cell_of[g][0] + (int64_t)n * (cell_of[g][1] + (int64_t)n * cell_of[g][2]);
    return G + cell * ncomp<DIM>() * NP;
  };
  cell_op<DIM, l, 1, T>(cpb, tile, gptr);
  pfor_n<NP>(cpb, [&](int g, int i) {
    if (cell_of[g][3]) cellout[((int64_t)blockIdx.x * cpb + g) * NP + i] = tile(g, 0)[i];
  });
}

// y = sum of the cell contributions at each node (b == nullptr), or
// y = b - that sum; boundary nodes of y are 0.
template <int DIM, typename T>
__global__ void __launch_bounds__(256) cell_gather_kernel(const T* __restrict__ cellout, T* __restrict__ y,
                                                          const T* __restrict__ b, int n) {
  constexpr int n1 = K + 1;
  const int N1 = K * n + 1;
  const int64_t N = DIM == 3 ? (int64_t)N1 * N1 * N1 : (int64_t)N1 * N1;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
    const int gd[3] = {(int)(t % N1), (int)((t / N1) % N1), DIM == 3 ? (int)(t / ((int64_t)N1 * N1)) : 0};
    bool bnd = false;
    int clo[3], ccnt[3];
    for (int d = 0; d < DIM; ++d) {
      const int g = gd[d];
      bnd |= g == 0 || g == N1 - 1;
      const int c = g / K, a = g - K * c;
      int lo = (a == 0 && c > 0) ? c - 1 : c, hi = c;
      hi = hi > n - 1 ? n - 1 : hi;
      clo[d] = lo;
      ccnt[d] = hi - lo + 1;
    }
    if (bnd) {
      y[t] = T(0);
      continue;
    }
    T s = T(0);
    const int cz = DIM == 3 ? ccnt[2] : 1;
    for (int jz = 0; jz < cz; ++jz)
      for (int jy = 0; jy < ccnt[1]; ++jy)
        for (int jx = 0; jx < ccnt[0]; ++jx) {
          const int cx = clo[0] + jx, cy = clo[1] + jy, czz = DIM == 3 ? clo[2] + jz : 0;
          const int ax = gd[0] - K * cx, ay = gd[1] - K * cy, az = DIM == 3 ? gd[2] - K * czz : 0;
          const int64_t cell = cx + (int64_t)n * (cy + (int64_t)n * czz);
          s += cellout[cell * ipow(n1, DIM) + ax + n1 * (ay + n1 * az)];
        }
    y[t] = b ? b[t] - s : s;
  }
}

// ---------------------------------------------------------------------------
// Deformed apply for degrees K <= 3 in 3D: one half-warp per cell, every 1D
// contraction in registers.  Each of the (K+1)^2 active lanes owns one line
// of K+1 values along x (lane (y, z)), y (lane (x, z)) or z (lane (x, y));
// between directions the lines are transposed through a padded shared tile
// of the cell (each value stored and loaded once, __syncwarp only).  The
// gradient at the Gauss points is formed with the derivative folded into
// the interpolation passes (DS = Dq S: derivative of the nodal basis at the
// points): grad_x = S_z S_y DS_x u, grad_y = S_z DS_y S_x u, grad_z =
// DS_z S_y S_x u; after the q-op with the stored G_q, the transposed passes
// run in reverse.  Cells of one parity colour share no node, so launch c
// adds the contributions of the cells of colour c straight into y: the
// cell of lowest colour among those holding a node (even parity in every
// direction in which the node is shared) initialises it (y = s, or b - s),
// the others add -- deterministic, no per-cell buffer, no atomics.
// Arithmetic of the half-warp kernel: AF32 (FP32 vectors, float lines) or
// AFF (FP64 vectors, float-float lines: each value a pair of floats, every
// product and sum by the error-free transformations of cart_pass_ff; the
// FP32-stored G_q enters the products exactly).  W = floats per line value.
struct AF32 {
  using IO = float;
  using V = float;
  using Acc = float;
  static constexpr int W = 1;
  static __device__ __forceinline__ V zero() { return 0.f; }
  static __device__ __forceinline__ void mac(Acc& a, double c, V x) { a += (float)c * x; }
  static __device__ __forceinline__ void macg(Acc& a, float g, V x) { a += g * x; }
  static __device__ __forceinline__ V val(const Acc& a) { return a; }
  static __device__ __forceinline__ V in(IO v) { return v; }
  static __device__ __forceinline__ IO out(V v) { return v; }
  static __device__ __forceinline__ void put(float* t, int stride, V v) { t[0] = v; }
  static __device__ __forceinline__ V get(const float* t, int stride) { return t[0]; }
};
struct AFF {
  using IO = double;
  using V = ff;
  using Acc = ff_acc;
  static constexpr int W = 2;
  static __device__ __forceinline__ V zero() { return ff{0.f, 0.f}; }
  static __device__ __forceinline__ void mac(Acc& a, double c, V x) { a.mac(ff_const(c), x); }
  static __device__ __forceinline__ void macg(Acc& a, float g, V x) { a.mac(ff{g, 0.f}, x); }
  static __device__ __forceinline__ V val(const Acc& a) { return a.value(); }
  static __device__ __forceinline__ V in(IO v) { return ff_of(v); }
  static __device__ __forceinline__ IO out(V v) { return ff_to_double(v); }
  static __device__ __forceinline__ void put(float* t, int stride, V v) { t[0] = v.hi; t[stride] = v.lo; }
  static __device__ __forceinline__ V get(const float* t, int stride) { return ff{t[0], t[stride]}; }
};

template <class A>
struct DefFast {
  static constexpr int n1 = K + 1;
  static constexpr int PY = n1;                                 // tile row pitch
  static constexpr int PZ = n1 * n1 + (n1 == 4 ? 4 : 1);        // tile plane pitch (bank spread)
  static constexpr int TILE = PZ * n1;
  static constexpr int CELL = 3 * TILE * A::W;                  // three tiles per cell (floats)
  static constexpr int CELLS = 16;                              // largest cells (half-warps) per block
};

// The cell operator of the half-warp kernel for one cell: lane (la, lb) holds
// the nodal x-line u (y = la, z = lb) and G_q at its z-line points (x = la,
// y = lb, z = q); res receives A_cell u on the lane's x-line.  tl: the
// half-warp's three transposition tiles (F::CELL floats); every lane of the
// warp calls it (lanes with on = false hold zeros and store nothing).
template <class A>
__device__ __forceinline__ void def_fast_core(const typename A::V (&u)[K + 1], const float (&gq)[6][K + 1], float* tl,
                                              bool on, int la, int lb, typename A::V (&res)[K + 1]) {
  using F = DefFast<A>;
  using V = typename A::V;
  using Acc = typename A::Acc;
  constexpr int n1 = F::n1, L = nlev(K) - 1;
  constexpr int PY = F::PY, PZ = F::PZ, TILE = F::TILE;
  constexpr int OS = LAY.S[L], OD = LAY.Dq[L];
  const double* C = ctab<double>();
  auto S = [&](int q, int a) -> double { return C[OS + q * n1 + a]; };
  auto DS = [&](int q, int a) -> double {  // derivative of nodal basis a at point q
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < n1; ++j) s += C[OD + q * n1 + j] * C[OS + j * n1 + a];
    return s;
  };
  auto put = [&](int k, int ix, int iy, int iz, V v) {
    if (on) A::put(tl + k * TILE + ix + PY * iy + PZ * iz, 3 * TILE, v);
  };
  auto get = [&](int k, int ix, int iy, int iz) -> V {
    return on ? A::get(tl + k * TILE + ix + PY * iy + PZ * iz, 3 * TILE) : A::zero();
  };
  // ---- X-own (lane (y = la, z = lb)): P = S_x u, Pd = DS_x u
  V P[n1], Pd[n1];
#pragma unroll
  for (int q = 0; q < n1; ++q) {
    Acc s0{}, s1{};
#pragma unroll
    for (int i = 0; i < n1; ++i) { A::mac(s0, S(q, i), u[i]); A::mac(s1, DS(q, i), u[i]); }
    P[q] = A::val(s0);
    Pd[q] = A::val(s1);
  }
  // ---- X -> Y: lane (x = la, z = lb)
#pragma unroll
  for (int q = 0; q < n1; ++q) { put(0, q, la, lb, P[q]); put(1, q, la, lb, Pd[q]); }
  __syncwarp();
#pragma unroll
  for (int j = 0; j < n1; ++j) { P[j] = get(0, la, j, lb); Pd[j] = get(1, la, j, lb); }
  __syncwarp();
  V Q[n1], Qx[n1], Qy[n1];  // S_y P, S_y P', DS_y P
#pragma unroll
  for (int q = 0; q < n1; ++q) {
    Acc s0{}, s1{}, s2{};
#pragma unroll
    for (int j = 0; j < n1; ++j) { A::mac(s0, S(q, j), P[j]); A::mac(s1, S(q, j), Pd[j]); A::mac(s2, DS(q, j), P[j]); }
    Q[q] = A::val(s0);
    Qx[q] = A::val(s1);
    Qy[q] = A::val(s2);
  }
  // ---- Y -> Z: lane (x = la, y = lb)
#pragma unroll
  for (int q = 0; q < n1; ++q) { put(0, la, q, lb, Q[q]); put(1, la, q, lb, Qx[q]); put(2, la, q, lb, Qy[q]); }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < n1; ++k) { Q[k] = get(0, la, lb, k); Qx[k] = get(1, la, lb, k); Qy[k] = get(2, la, lb, k); }
  __syncwarp();
  // gradients at the points (la, lb, q) and the q-op with G_q
  V fx[n1], fy[n1], fz[n1];
#pragma unroll
  for (int q = 0; q < n1; ++q) {
    Acc a0{}, a1{}, a2{};
#pragma unroll
    for (int k = 0; k < n1; ++k) { A::mac(a0, S(q, k), Qx[k]); A::mac(a1, S(q, k), Qy[k]); A::mac(a2, DS(q, k), Q[k]); }
    const V gx = A::val(a0), gy2 = A::val(a1), gz2 = A::val(a2);
    Acc f0{}, f1{}, f2{};
    A::macg(f0, gq[0][q], gx); A::macg(f0, gq[1][q], gy2); A::macg(f0, gq[2][q], gz2);
    A::macg(f1, gq[1][q], gx); A::macg(f1, gq[3][q], gy2); A::macg(f1, gq[4][q], gz2);
    A::macg(f2, gq[2][q], gx); A::macg(f2, gq[4][q], gy2); A::macg(f2, gq[5][q], gz2);
    fx[q] = A::val(f0);
    fy[q] = A::val(f1);
    fz[q] = A::val(f2);
  }
  // ---- transposed passes: Z-own A1 = S_z^T fx, A2 = S_z^T fy, A3 = DS_z^T fz
#pragma unroll
  for (int k = 0; k < n1; ++k) {
    Acc s0{}, s1{}, s2{};
#pragma unroll
    for (int q = 0; q < n1; ++q) { A::mac(s0, S(q, k), fx[q]); A::mac(s1, S(q, k), fy[q]); A::mac(s2, DS(q, k), fz[q]); }
    Q[k] = A::val(s0);
    Qx[k] = A::val(s1);
    Qy[k] = A::val(s2);
  }
  // ---- Z -> Y: lane (x = la, z = lb)
#pragma unroll
  for (int k = 0; k < n1; ++k) { put(0, la, lb, k, Q[k]); put(1, la, lb, k, Qx[k]); put(2, la, lb, k, Qy[k]); }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < n1; ++q) { Q[q] = get(0, la, q, lb); Qx[q] = get(1, la, q, lb); Qy[q] = get(2, la, q, lb); }
  __syncwarp();
  // B1 = S_y^T A1, B23 = DS_y^T A2 + S_y^T A3
#pragma unroll
  for (int j = 0; j < n1; ++j) {
    Acc s0{}, s1{};
#pragma unroll
    for (int q = 0; q < n1; ++q) { A::mac(s0, S(q, j), Q[q]); A::mac(s1, DS(q, j), Qx[q]); A::mac(s1, S(q, j), Qy[q]); }
    P[j] = A::val(s0);
    Pd[j] = A::val(s1);
  }
  // ---- Y -> X: lane (y = la, z = lb)
#pragma unroll
  for (int j = 0; j < n1; ++j) { put(0, la, j, lb, P[j]); put(1, la, j, lb, Pd[j]); }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < n1; ++q) { P[q] = get(0, q, la, lb); Pd[q] = get(1, q, la, lb); }
  // out = DS_x^T B1 + S_x^T B23
#pragma unroll
  for (int i = 0; i < n1; ++i) {
    Acc s{};
#pragma unroll
    for (int q = 0; q < n1; ++q) { A::mac(s, DS(q, i), P[q]); A::mac(s, S(q, i), Pd[q]); }
    res[i] = A::val(s);
  }
}

template <bool RESID, class A>
__global__ void __launch_bounds__(256) def_fast_kernel(const typename A::IO* __restrict__ x,
                                                       typename A::IO* __restrict__ y,
                                                       const typename A::IO* __restrict__ b,
                                                       const float* __restrict__ G, int n, int colour) {
  using F = DefFast<A>;
  using V = typename A::V;
  using IO = typename A::IO;
  constexpr int n1 = F::n1, NP = n1 * n1 * n1;
  __shared__ float tiles[F::CELLS * F::CELL];
  const int hw = threadIdx.x >> 4, lane = threadIdx.x & 15;
  const bool on = lane < n1 * n1;
  const int la = on ? lane % n1 : 0, lb = on ? lane / n1 : 0;
  float* tl = tiles + hw * F::CELL;
  // this half-warp's cell among those of parity colour `colour`
  int bit[3], cnt[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    bit[d] = (colour >> d) & 1;
    cnt[d] = (n - bit[d] + 1) / 2;
  }
  const int64_t ncol = (int64_t)cnt[0] * cnt[1] * cnt[2];
  const int64_t cid = (int64_t)blockIdx.x * (blockDim.x >> 4) + hw;
  const bool live = on && cid < ncol;
  int c[3];
  {
    int64_t t = live ? cid : 0;
    c[0] = bit[0] + 2 * (int)(t % cnt[0]);
    t /= cnt[0];
    c[1] = bit[1] + 2 * (int)(t % cnt[1]);
    c[2] = bit[2] + 2 * (int)(t / cnt[1]);
  }
  const int N1 = K * n + 1;
  // ---- every global load of the cell first (one memory latency per cell):
  // the nodal x-line, the value each output node starts from (y of an
  // earlier colour, b, or nothing), and G_q at this lane's points of the
  // z-line ownership used by the q-op.  G_q is read once per apply and is
  // most of its bytes: streaming loads (evict first) keep it from pushing x
  // and y, which the colour launches revisit, out of L2.
  V u[n1];
  IO prior[n1];
  bool first[n1], bnd[n1];
  const int gy = K * c[1] + la, gz = K * c[2] + lb;
  const bool yz_bnd = gy == 0 || gy == N1 - 1 || gz == 0 || gz == N1 - 1;
  const int64_t row = (int64_t)N1 * (gy + (int64_t)N1 * gz) + K * c[0];
#pragma unroll
  for (int i = 0; i < n1; ++i) {
    const int gx = K * c[0] + i;
    bnd[i] = yz_bnd || gx == 0 || gx == N1 - 1;
    const int li[3] = {i, la, lb};
    bool f = true;  // lowest colour among the cells holding this node
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const bool shared = (li[d] == 0 && c[d] > 0) || (li[d] == K && c[d] < n - 1);
      if (shared && (c[d] & 1)) f = false;
    }
    first[i] = f;
    u[i] = (live && !bnd[i]) ? A::in(x[row + i]) : A::zero();
    prior[i] = (live && !bnd[i]) ? (f ? (RESID ? b[row + i] : IO(0)) : y[row + i]) : IO(0);
  }
  const int64_t cell = c[0] + (int64_t)n * (c[1] + (int64_t)n * c[2]);
  const float* Gc = G + cell * 6 * NP + la + n1 * lb;
  float gq[6][n1];
#pragma unroll
  for (int q = 0; q < n1; ++q)
#pragma unroll
    for (int m = 0; m < 6; ++m) gq[m][q] = live ? __ldcs(Gc + m * NP + n1 * n1 * q) : 0.f;

  V res[n1];
  def_fast_core<A>(u, gq, tl, on, la, lb, res);
  // added into y node by node
#pragma unroll
  for (int i = 0; i < n1; ++i) {
    if (!live || (bnd[i] && !first[i])) continue;
    const IO v = A::out(res[i]);
    y[row + i] = bnd[i] ? IO(0) : (RESID ? prior[i] - v : prior[i] + v);
  }
}

// the 2^3 colour launches of the half-warp kernel (3D, k <= 3)
// cpb: cells (half-warps) per block, 4, 8 or 16 (0: 16)
template <class A>
static cudaError_t def_fast_apply(const typename A::IO* x, typename A::IO* y, const typename A::IO* b,
                                  const float* G, int n, int cpb, cudaStream_t st) {
  if constexpr (K <= 3) {
    if (cpb == 0) cpb = DefFast<A>::CELLS;
    if (cpb != 4 && cpb != 8 && cpb != 16) return cudaErrorInvalidValue;
    for (int colour = 0; colour < 8; ++colour) {
      int64_t ncol = 1;
      for (int d = 0; d < 3; ++d) ncol *= (n - ((colour >> d) & 1) + 1) / 2;
      if (ncol == 0) continue;
      const unsigned blocks = (unsigned)((ncol + cpb - 1) / cpb);
      if (b) def_fast_kernel<true, A><<<blocks, 16 * cpb, 0, st>>>(x, y, b, G, n, colour);
      else def_fast_kernel<false, A><<<blocks, 16 * cpb, 0, st>>>(x, y, b, G, n, colour);
      g_launches += 1;
    }
    return cudaGetLastError();
  } else {
    return cudaErrorInvalidValue;
  }
}

// FP64 deformed apply in float-float arithmetic (3D, k <= 3, FP32-stored
// G_q); cudaErrorInvalidValue for other parts
static cudaError_t def_apply_ff(int dim, const double* x, double* y, const double* b, const float* G, int n, int cpb,
                                cudaStream_t st) {
  if (dim != 3 || PMG_DIM != 3 || K > 3) return cudaErrorInvalidValue;
  return def_fast_apply<AFF>(x, y, b, G, n, cpb, st);
}

// true when the fast deformed apply covers this degree, dimension and
// precision: FP32 only -- it spends about 28% more multiply-adds per cell than
// the shared-memory cell operator (the derivative folded into the
// interpolation passes), which pays where memory bounds the apply (FP32) and
// not where GB300's FP64 rate does
template <int DIM, typename T>
constexpr bool def_fast_ok() { return DIM == 3 && K <= 3 && sizeof(T) == 4; }

// cpb: cells per block (0: the rule below); the half-warp kernel takes 4, 8
// or 16, the shared-memory cell kernel any count whose tiles fit
template <int DIM, typename T, typename TG>
static cudaError_t def_apply_t(const T* x, T* y, const T* b, const TG* G, T* cellbuf, int n, int cpb,
                               cudaStream_t st) {
  if constexpr (def_fast_ok<DIM, T>() && sizeof(TG) == 4) {
    return def_fast_apply<AF32>(x, y, b, G, n, cpb, st);
  }
  constexpr int n1 = K + 1;
  constexpr int NP = ipow(n1, DIM);
  constexpr int LINES = ipow(n1, DIM - 1);
  if (cpb <= 0) {
    cpb = 256 / LINES;
    while (cpb > 1 && cpb * 5 * NP * (int)sizeof(T) > 96 * 1024) --cpb;
  }
  if (cpb < 1) cpb = 1;
  if (cpb > kMaxPatchesPerBlock) cpb = kMaxPatchesPerBlock;
  if (cpb * LINES > 1024) return cudaErrorInvalidValue;
  const int threads = std::min(256, (cpb * LINES + 31) / 32 * 32);
  const int smem = cpb * 5 * NP * (int)sizeof(T);
  if (smem > kMaxDynSmem) return cudaErrorInvalidConfiguration;
  const int64_t ncell = DIM == 3 ? (int64_t)n * n * n : (int64_t)n * n;
  def_cell_kernel<DIM, T, TG><<<(unsigned)((ncell + cpb - 1) / cpb), threads, smem, st>>>(x, cellbuf, G, n, cpb);
  const int64_t N = ipow(K * n + 1, DIM);
  cell_gather_kernel<DIM, T><<<grid_for(N, 256), 256, 0, st>>>(cellbuf, y, b, n);
  g_launches += 2;
  return cudaGetLastError();
}

static cudaError_t def_apply(int dim, int prec, const void* x, void* y, const void* b, const void* G, int gprec,
                             void* cellbuf, int n, int cpb, cudaStream_t s) {
  if (dim != PMG_DIM || prec != PMG_PREC) return cudaErrorInvalidValue;
  using TP = std::conditional_t<PMG_PREC == 0, double, float>;
  if (gprec == 0)
    return def_apply_t<PMG_DIM, TP, double>((const TP*)x, (TP*)y, (const TP*)b, (const double*)G, (TP*)cellbuf, n,
                                            cpb, s);
  return def_apply_t<PMG_DIM, TP, float>((const TP*)x, (TP*)y, (const TP*)b, (const float*)G, (TP*)cellbuf, n, cpb,
                                         s);
}

// cells-per-block candidates of this part's deformed apply (3D k <= 3 FP32:
// the half-warp kernel; else the shared-memory cell kernel)
static int def_apply_candidates(int dim, int prec, int gprec, int* out, int max) {
  if (dim != PMG_DIM || prec != PMG_PREC) return 0;
  using TP = std::conditional_t<PMG_PREC == 0, double, float>;
  int c = 0;
  if (def_fast_ok<PMG_DIM, TP>() && gprec == 1) {
    for (int v : {4, 8, 16})
      if (c < max) out[c++] = v;
    return c;
  }
  constexpr int n1 = K + 1;
  constexpr int NP = ipow(n1, PMG_DIM);
  constexpr int LINES = ipow(n1, PMG_DIM - 1);
  for (int v : {1, 2, 4, 8, 16, 32})
    if (v * LINES <= 1024 && v * 5 * NP * (int)sizeof(TP) <= kMaxDynSmem && c < max) out[c++] = v;
  return c;
}

// ---------------------------------------------------------------------------
// Deformed vertex-patch smoother.  The patch vmult (§3.2.1) distributes the
// patch-interior vector to the 2^d cells of the patch (zero on the patch
// boundary), applies the cell operator with each cell's stored G, and sums
// the cell results back onto the interior nodes.  Inverse diagonals come
// from the global degree-p diagonal of the level (a patch-interior DoF has
// its whole support inside the patch, so diag(A_{j,p}) is that diagonal).
// ---------------------------------------------------------------------------
// Patch-level sum factorisation on the (2p+1)^d patch grid: per direction
// the two cells' Gauss points (2(p+1)) are reached from the 2p+1 nodes by a
// block-diagonal interpolation (each cell's (p+1) x (p+1) GLL->Gauss block,
// sharing the centre node), gradients by block-diagonal collocation
// derivatives, the q-op uses the stored G_q of the cell holding each point,
// and the transposed steps sum the two cells' contributions at shared nodes.
template <int DIM>
struct DefShape {
  using PS = PatchShape<DIM>;
  static constexpr int QT = 2 * (K + 1);                    // Gauss points per direction (top level)
  static constexpr int BUF = tpitch(QT) * ipow(QT, DIM - 1);  // padded (QT)^DIM tile, >= (2K+1)^DIM
  static constexpr int LINES = ipow(QT, DIM - 1);           // lines of the largest step, per patch
  static constexpr int WORK = (DIM == 3 ? 4 : 3) * BUF;
  template <typename T>
  static constexpr int elems() { return PS::ELEMS + WORK; }
};

template <typename T, typename TG>
struct DefLevelT {
  const TG* G[4];
  const T* dinv[4];
};

// Along axis AX of a tile with extents (EX, EY, EZ): src extent NI -> dst
// extent NO.  OP 0: interpolation nodes -> points (NI = 2p+1, NO = 2(p+1));
// OP 1: its transpose; OP 2: block-diagonal derivative (NI = NO = 2(p+1));
// OP 3: its transpose.  ACC: dst += result.  A tile with x extent e is
// stored with row pitch tpitch(e) (odd) and plane pitch tpitch(e) * (y
// extent): with the even point counts 2(p+1) an unpadded tile would put the
// lines of a warp on a few banks (x lines 2(p+1) apart, y lines
// 4(p+1)^2 apart).
template <int DIM, int p, int AX, int OP, bool ACC, int EX, int EY, int EZ, typename T>
__device__ __forceinline__ void patch_axis(const T* Sm, const T* Dm, const PBlock<T, 0>& pb, int src, int dst) {
  constexpr int nq = p + 1, mf = 2 * p + 1, Q = 2 * nq;
  constexpr int NI = (OP == 0) ? mf : (OP == 1 ? Q : Q);
  constexpr int NO = (OP == 0) ? Q : (OP == 1 ? mf : Q);
  constexpr int IX = AX == 0 ? NI : EX, IY = AX == 1 ? NI : EY, IZ = AX == 2 ? NI : EZ;
  constexpr int OX = AX == 0 ? NO : EX, OY = AX == 1 ? NO : EY;
  constexpr int RXI = tpitch(IX), RYI = RXI * IY;  // input row / plane pitch
  constexpr int RXO = tpitch(OX), RYO = RXO * OY;  // output row / plane pitch
  constexpr int SI = AX == 0 ? 1 : (AX == 1 ? RXI : RYI);
  constexpr int SO = AX == 0 ? 1 : (AX == 1 ? RXO : RYO);
  constexpr int NL = IX * IY * IZ / NI;
  pfor<NL>(pb, [&](int g, int L) {
    auto sm = pb.at(g);
    int bi, bo;
    if constexpr (AX == 0) {  // line (y, z)
      const int y = L % IY, z = L / IY;
      bi = RXI * y + RYI * z;
      bo = RXO * y + RYO * z;
    } else if constexpr (AX == 1) {  // line (x, z)
      const int x = L % IX, z = L / IX;
      bi = x + RYI * z;
      bo = x + RYO * z;
    } else {  // line (x, y)
      const int x = L % IX, y = L / IX;
      bi = x + RXI * y;
      bo = x + RXO * y;
    }
    T x[NI], y[NO];
#pragma unroll
    for (int j = 0; j < NI; ++j) x[j] = sm[src + bi + j * SI];
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      T acc = T(0);
      if constexpr (OP == 0) {  // point o of cell o / nq from nodes p c .. p c + p
        const int c = o / nq, q = o % nq;
#pragma unroll
        for (int jj = 0; jj <= p; ++jj) acc += Sm[q * nq + jj] * x[p * c + jj];
      } else if constexpr (OP == 1) {  // node o from the points of the cells holding it
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int jj = o - p * c;
          if (jj >= 0 && jj <= p) {
#pragma unroll
            for (int q = 0; q < nq; ++q) acc += Sm[q * nq + jj] * x[c * nq + q];
          }
        }
      } else if constexpr (OP == 2) {
        const int c = o / nq, q = o % nq;
#pragma unroll
        for (int qq = 0; qq < nq; ++qq) acc += Dm[q * nq + qq] * x[c * nq + qq];
      } else {
        const int c = o / nq, q = o % nq;
#pragma unroll
        for (int qq = 0; qq < nq; ++qq) acc += Dm[qq * nq + q] * x[c * nq + qq];
      }
      if (ACC) sm[dst + bo + o * SO] += acc;
      else sm[dst + bo + o * SO] = acc;
    }
  });
}

// Deformed patch geometry: patch vmult by patch-level sum factorisation
// (§3.2.1); inverse diagonals from the level's global degree-p diagonals.
template <int DIM, typename T, typename TG>
struct DefGeo {
  DefLevelT<T, TG> lev;
  const PatchMeta* meta;
  const T* inv_a0;  // per patch of the block (shared memory)
  int n;

  __device__ __forceinline__ T dinv_at(int g, int l, int i) const {
    const int p = plev(K, l);
    const int m = 2 * p - 1, N1 = p * n + 1;
    const int* v = meta[g].v;
    const int ix = i % m, iy = (i / m) % m, iz = DIM == 3 ? i / (m * m) : 0;
    const int gx = p * (v[0] - 1) + 1 + ix, gy = p * (v[1] - 1) + 1 + iy;
    const int gz = DIM == 3 ? p * (v[2] - 1) + 1 + iz : 0;
    return lev.dinv[l][gx + (int64_t)N1 * (gy + (int64_t)N1 * gz)];
  }
  __device__ __forceinline__ T a0inv(int g) const { return inv_a0[g]; }

  static constexpr bool kFusedSmoothing = false;  // Jacobi steps as separate pointwise passes

  // The top level of an FP32 patch (FP32 G_q, 3D, K = 2, 3) applies its
  // operator cell by cell with the half-warp cell operator of the deformed
  // apply (def_fast_core: line contractions in registers, shared memory only
  // for the transpositions) instead of sum factorisation on the whole patch
  // grid: the patch residual is r - sum over the patch's 8 cells of A_cell d
  // (d extended by zero to the patch boundary), each cell's results summed
  // into a node in a fixed cell order.
  template <int l>
  static constexpr bool cellwise() {
    return DIM == 3 && K >= 2 && K <= 3 && l == nlev(K) - 1 && std::is_same<T, float>::value &&
           std::is_same<TG, float>::value;
  }

  template <int l, class PB>
  __device__ __forceinline__ void resid_cells(const PB& pb, int od, int orr, int oo) const {
    using F = DefFast<AF32>;
    constexpr int n1 = K + 1, NP = n1 * n1 * n1, m = mp(K), mf = 2 * K + 1;
    constexpr int W = PatchShape<3>::ELEMS, CT = F::CELL;  // cell c's tiles at W + c CT
    static_assert(8 * CT <= DefShape<3>::WORK, "the cells' tiles fit the work area of a patch");
    // (patch, cell, lane) items: a half-warp per cell, the two half-warps of
    // a warp on two cells of one patch
    pfor<8 * 16>(pb, [&](int g, int it) {
      float* sm = &pb.at(g)[0];
      const int c = it >> 4, lane = it & 15;
      const bool on = lane < n1 * n1;
      const int la = on ? lane % n1 : 0, lb = on ? lane / n1 : 0;
      const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
      const bool live = on && meta[g].active;
      float* tl = sm + W + c * CT;
      // the cell's nodal x-line (y = la, z = lb): d on the patch interior, 0 on its boundary
      float u[n1];
      const int fy = K * cy + la, fz = K * cz + lb;
      const bool yz_in = fy >= 1 && fy <= mf - 2 && fz >= 1 && fz <= mf - 2;
#pragma unroll
      for (int i = 0; i < n1; ++i) {
        const int fx = K * cx + i;
        u[i] = (live && yz_in && fx >= 1 && fx <= mf - 2) ? sm[od + (fx - 1) + m * ((fy - 1) + m * (fz - 1))] : 0.f;
      }
      const int* v = meta[g].v;
      const int64_t cell =
          live ? (v[0] - 1 + cx) + (int64_t)n * ((v[1] - 1 + cy) + (int64_t)n * (v[2] - 1 + cz)) : 0;
      const float* Gc = reinterpret_cast<const float*>(lev.G[l]) + cell * 6 * NP + la + n1 * lb;
      float gq[6][n1];
#pragma unroll
      for (int q = 0; q < n1; ++q)
#pragma unroll
        for (int mm = 0; mm < 6; ++mm) gq[mm][q] = live ? Gc[mm * NP + n1 * n1 * q] : 0.f;
      float res[n1];
      def_fast_core<AF32>(u, gq, tl, on, la, lb, res);
      __syncwarp();  // the half-warp's last reads of its tiles are done
      if (on) {
#pragma unroll
        for (int i = 0; i < n1; ++i) tl[i + n1 * (la + n1 * lb)] = res[i];
      }
    });
    __syncthreads();
    pfor<m * m * m>(pb, [&](int g, int i) {
      auto sm = pb.at(g);
      const int f[3] = {i % m + 1, (i / m) % m + 1, i / (m * m) + 1};
      float acc = 0.f;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        int ix[3];
        bool in = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          ix[d] = f[d] - K * ((c >> d) & 1);
          in = in && ix[d] >= 0 && ix[d] <= K;
        }
        if (in) acc += sm[W + c * CT + ix[0] + n1 * (ix[1] + n1 * ix[2])];
      }
      sm[oo + i] = sm[orr + i] - acc;
    });
    __syncthreads();
  }

  template <int l, class PB>
  __device__ __forceinline__ void resid(const PB& pb, int od, int orr, int oo) const {
    if constexpr (cellwise<l>()) {
      resid_cells<l>(pb, od, orr, oo);
      return;
    }
    constexpr int p = plev(K, l);
    constexpr int m = mp(p), mf = 2 * p + 1, nq = p + 1, Q = 2 * nq;
    constexpr int NPc = ipow(nq, DIM);  // points per cell
    constexpr int B = DefShape<DIM>::BUF;
    constexpr int W = PatchShape<DIM>::ELEMS;
    constexpr int B0 = W, B1 = W + B, B2 = W + 2 * B, B3 = W + 3 * B;
    const T* Sm = ctab<T>() + LAY.S[l];
    const T* Dm = ctab<T>() + LAY.Dq[l];
    constexpr int MZ = DIM == 3 ? mf : 1, QZ = DIM == 3 ? Q : 1;
    // expand d onto the patch grid (zero on its boundary) in B0: (mf, mf, MZ)
    pfor<ipow(mf, DIM)>(pb, [&](int g, int i) {
      auto sm = pb.at(g);
      const int fx = i % mf, fy = (i / mf) % mf, fz = DIM == 3 ? i / (mf * mf) : 1;
      const bool in = fx > 0 && fx < mf - 1 && fy > 0 && fy < mf - 1 && (DIM == 2 || (fz > 0 && fz < mf - 1));
      sm[B0 + i] = in ? sm[od + (fx - 1) + m * ((fy - 1) + m * (DIM == 3 ? fz - 1 : 0))] : T(0);
    });
    __syncthreads();
    // values at the Gauss points: (mf,mf,MZ) -> (Q,mf,MZ) -> (Q,Q,MZ) -> (Q,Q,QZ)
    patch_axis<DIM, p, 0, 0, false, mf, mf, MZ>(Sm, Dm, pb, B0, B1);
    __syncthreads();
    patch_axis<DIM, p, 1, 0, false, Q, mf, MZ>(Sm, Dm, pb, B1, B0);
    __syncthreads();
    if constexpr (DIM == 3) {
      patch_axis<DIM, p, 2, 0, false, Q, Q, mf>(Sm, Dm, pb, B0, B1);
      __syncthreads();
    }
    constexpr int U = DIM == 3 ? B1 : B0;  // values at the points
    constexpr int GX = DIM == 3 ? B0 : B1, GY = B2, GZ = B3;
    patch_axis<DIM, p, 0, 2, false, Q, Q, QZ>(Sm, Dm, pb, U, GX);
    patch_axis<DIM, p, 1, 2, false, Q, Q, QZ>(Sm, Dm, pb, U, GY);
    if constexpr (DIM == 3) patch_axis<DIM, p, 2, 2, false, Q, Q, QZ>(Sm, Dm, pb, U, GZ);
    __syncthreads();
    // q-op with the stored G_q of the cell holding each point; points visited
    // cell by cell so that G_q reads are contiguous
    pfor<(1 << DIM) * NPc>(pb, [&](int g, int t) {
      auto sm = pb.at(g);
      const int c = t / NPc, pt = t - c * NPc;
      const int px = pt % nq, py = (pt / nq) % nq, pz = DIM == 3 ? pt / (nq * nq) : 0;
      const int qx = (c & 1) * nq + px, qy = ((c >> 1) & 1) * nq + py;
      const int qz = DIM == 3 ? ((c >> 2) & 1) * nq + pz : 0;
      const int qi = qx + tpitch(Q) * (qy + Q * qz);  // padded (Q, Q, QZ) tile
      const int* v = meta[g].v;
      const int64_t cell = (v[0] - 1 + (c & 1)) +
                           (int64_t)n * ((v[1] - 1 + ((c >> 1) & 1)) + (int64_t)n * (DIM == 3 ? v[2] - 1 + ((c >> 2) & 1) : 0));
      const TG* Gc = lev.G[l] + cell * ncomp<DIM>() * NPc + pt;
      if constexpr (DIM == 3) {
        const T g0 = sm[GX + qi], g1 = sm[GY + qi], g2 = sm[GZ + qi];
        const T G00 = (T)Gc[0], G01 = (T)Gc[NPc], G02 = (T)Gc[2 * NPc];
        const T G11 = (T)Gc[3 * NPc], G12 = (T)Gc[4 * NPc], G22 = (T)Gc[5 * NPc];
        sm[GX + qi] = G00 * g0 + G01 * g1 + G02 * g2;
        sm[GY + qi] = G01 * g0 + G11 * g1 + G12 * g2;
        sm[GZ + qi] = G02 * g0 + G12 * g1 + G22 * g2;
      } else {
        const T g0 = sm[GX + qi], g1 = sm[GY + qi];
        const T G00 = (T)Gc[0], G01 = (T)Gc[NPc], G11 = (T)Gc[2 * NPc];
        sm[GX + qi] = G00 * g0 + G01 * g1;
        sm[GY + qi] = G01 * g0 + G11 * g1;
      }
    });
    __syncthreads();
    // divergence back to the points, then to the nodes
    patch_axis<DIM, p, 0, 3, false, Q, Q, QZ>(Sm, Dm, pb, GX, U);
    __syncthreads();
    patch_axis<DIM, p, 1, 3, true, Q, Q, QZ>(Sm, Dm, pb, GY, U);
    __syncthreads();
    if constexpr (DIM == 3) {
      patch_axis<DIM, p, 2, 3, true, Q, Q, QZ>(Sm, Dm, pb, GZ, U);
      __syncthreads();
      patch_axis<DIM, p, 2, 1, false, Q, Q, Q>(Sm, Dm, pb, U, B0);   // (Q,Q,Q) -> (Q,Q,mf)
      __syncthreads();
      patch_axis<DIM, p, 1, 1, false, Q, Q, mf>(Sm, Dm, pb, B0, B2);  // -> (Q,mf,mf)
      __syncthreads();
      patch_axis<DIM, p, 0, 1, false, Q, mf, mf>(Sm, Dm, pb, B2, B0); // -> (mf,mf,mf)
      __syncthreads();
    } else {
      patch_axis<DIM, p, 1, 1, false, Q, Q, 1>(Sm, Dm, pb, U, B2);    // (Q,Q) -> (Q,mf)
      __syncthreads();
      patch_axis<DIM, p, 0, 1, false, Q, mf, 1>(Sm, Dm, pb, B2, B1);  // -> (mf,mf)
      __syncthreads();
    }
    constexpr int R = DIM == 3 ? B0 : B1;
    pfor<ipow(m, DIM)>(pb, [&](int g, int i) {
      auto sm = pb.at(g);
      const int fx = i % m + 1, fy = (i / m) % m + 1, fz = DIM == 3 ? i / (m * m) + 1 : 0;
      sm[oo + i] = sm[orr + i] - sm[R + fx + mf * (fy + mf * fz)];
    });
    __syncthreads();
  }
};

template <int DIM, typename T, typename TG>
__global__ void patch_def_kernel(const T* __restrict__ r, T* __restrict__ dst, int n, int np, int n_iter,
                                 DefLevelT<T, TG> lev, const T* __restrict__ dinv1, PatchParams<T> P) {
  using S = PatchShape<DIM>;
  using DS = DefShape<DIM>;
  constexpr int SZT = S::SZT;
  constexpr int RT = S::off_r(S::L - 1), DT = S::off_d(S::L - 1);
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ PatchMeta meta[kMaxPatchesPerBlock];
  __shared__ T inv_a0[kMaxPatchesPerBlock];
  constexpr int EL = DS::template elems<T>();
  const int stride = EL + (n_iter > 1 ? 2 * SZT : 0);
  const PBlock<T, 0> pb{reinterpret_cast<T*>(smraw), stride, np};
  patch_meta_init<DIM>(meta, np, n, P.colour);
  __syncthreads();
  for (int g = threadIdx.x; g < np; g += blockDim.x) {  // p = 1: the vertex's inverse Q1 diagonal
    const int* v = meta[g].v;
    inv_a0[g] = dinv1[v[0] + (int64_t)(n + 1) * (v[1] + (int64_t)(n + 1) * v[2])];
  }
  const int N1 = K * n + 1;
  pfor<SZT>(pb, [&](int g, int i) {
    const PatchMeta& m = meta[g];
    pb.at(g)[RT + i] = m.active ? r[patch_node<DIM>(m, i, N1)] : T(0);
  });
  __syncthreads();
  DefGeo<DIM, T, TG> geo;
  geo.lev = lev;
  geo.meta = meta;
  geo.inv_a0 = inv_a0;
  geo.n = n;
  local_solve<DIM>(pb, geo, P, n_iter, EL);
  const int64_t NN = DIM == 3 ? (int64_t)N1 * N1 * N1 : (int64_t)N1 * N1;
  pfor<SZT>(pb, [&](int g, int i) {
    const PatchMeta& m = meta[g];
    if (!m.active) return;
    if (P.colour < 0) dst[patch_colour<DIM>(m) * NN + patch_node<DIM>(m, i, N1)] = P.omega_as * pb.at(g)[DT + i];
    else dst[patch_node<DIM>(m, i, N1)] += pb.at(g)[DT + i];  // one patch of the colour per node
  });
}

// threads needed per patch for full warps in the largest step
static int patch_def_threads(int dim) { return dim == 3 ? DefShape<3>::LINES : DefShape<2>::LINES; }

static int patch_def_smem(int dim, int prec, int n_iter) {
  const int es = prec == 0 ? 8 : 4;
  int elems;
  if (dim == 3) elems = (prec == 0 ? DefShape<3>::elems<double>() : DefShape<3>::elems<float>()) +
                        (n_iter > 1 ? 2 * PatchShape<3>::SZT : 0);
  else elems = (prec == 0 ? DefShape<2>::elems<double>() : DefShape<2>::elems<float>()) +
               (n_iter > 1 ? 2 * PatchShape<2>::SZT : 0);
  return elems * es;
}

template <int DIM, typename T, typename TG>
static cudaError_t patch_def_t(const T* r, T* dst, int n, int np, int n_iter, const DefLevel& L,
                               const PatchParamsHost& H, cudaStream_t st) {
  const int64_t npatch = patch_count(DIM, n, H.colour);
  if (npatch == 0) return cudaSuccess;
  if (np < 1 || np > kMaxPatchesPerBlock) return cudaErrorInvalidValue;
  const int smem = np * patch_def_smem(DIM, sizeof(T) == 8 ? 0 : 1, n_iter);
  if (smem > kMaxDynSmem) return cudaErrorInvalidConfiguration;
  const int threads = std::min(1024, (np * DefShape<DIM>::LINES + 31) / 32 * 32);
  DefLevelT<T, TG> lev;
  for (int i = 0; i < 4; ++i) {
    lev.G[i] = (const TG*)L.G[i];
    lev.dinv[i] = (const T*)L.dinv[i];
  }
  const unsigned blocks = (unsigned)((npatch + np - 1) / np);
  patch_def_kernel<DIM, T, TG><<<blocks, threads, smem, st>>>(r, dst, n, np, n_iter, lev, (const T*)L.dinv1,
                                                              to_params<T>(H));
  g_launches += 1;
  return cudaGetLastError();
}

static cudaError_t patch_def(int dim, int prec, const void* r, void* dst, int n, int np, int n_iter,
                             const DefLevel& L, const PatchParamsHost& P, cudaStream_t s) {
  if (dim != PMG_DIM || prec != PMG_PREC) return cudaErrorInvalidValue;
  using TP = std::conditional_t<PMG_PREC == 0, double, float>;
  if (L.gprec == 0) return patch_def_t<PMG_DIM, TP, double>((const TP*)r, (TP*)dst, n, np, n_iter, L, P, s);
  return patch_def_t<PMG_DIM, TP, float>((const TP*)r, (TP*)dst, n, np, n_iter, L, P, s);
}

}  // namespace PMG_KNS
}  // namespace pmg
