// Degree-templated CUDA kernels of the p-multigrid vertex-patch library.
// Included once per degree K by inst_k<K>.cu, which instantiates the launch
// wrappers into a per-degree function table.
//
// Layout on the device: every level vector is the full (K n + 1)^DIM nodal
// grid, x fastest; boundary entries are zero.  The per-degree 1D matrices
// (reference mass/stiffness, patch matrices, p-transfers, h-prolongation
// tables, Gauss tables) live in __constant__ memory of this translation unit,
// in float64 and float32 copies (coef_layout in pmg_common.cuh).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "pmg_common.cuh"
#include "coef_tables.h"
#include "pmg_kernels_api.h"
#include "vec.h"

namespace pmg {
namespace PMG_KNS {

constexpr int K = PMG_K;
constexpr CoefLayout LAY = coef_layout(K);

static __constant__ double c_coef64[kMaxCoef];
static __constant__ float c_coef32[kMaxCoef];

// The same coefficient block as compile-time tables (generated at build time
// from the host set-up, coef_tables.h).  Every contraction whose indices are
// known after unrolling reads these: the compiler folds the entries into the
// arithmetic instead of loading them for every line.  Reads with run-time
// indices (the h-transfer passes) use the constant-memory copy above.
#define PMG_TAB_(prec, k) PMG_COEF##prec##_K##k
#define PMG_TAB(prec, k) PMG_TAB_(prec, k)
static __device__ constexpr double c_tab64[] = PMG_TAB(64, PMG_K);
static __device__ constexpr float c_tab32[] = PMG_TAB(32, PMG_K);

static inline int grid_for(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  const int64_t cap = 152 * 16;  // 152 SMs x resident blocks; grid-stride beyond
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

template <typename T>
__device__ __forceinline__ const T* coef();
template <>
__device__ __forceinline__ const double* coef<double>() { return c_coef64; }
template <>
__device__ __forceinline__ const float* coef<float>() { return c_coef32; }

template <typename T>
__device__ __forceinline__ const T* ctab();
template <>
__device__ __forceinline__ const double* ctab<double>() { return c_tab64; }
template <>
__device__ __forceinline__ const float* ctab<float>() { return c_tab32; }

// ===========================================================================
// Cartesian operator A = s * sum_dir (K on dir, M elsewhere), applied by one
// pass per direction over the global grid (the 1D matrices are the
// reference element matrices assembled along each grid line, i.e. banded
// with bandwidth K).  Sum factorisation with the 1D Gauss-quadrature
// matrices folded into M and K, exact for Cartesian cells (Eq. (3)).
//
// MODE 0 (first axis):  out0 = M in0, out1 = K in0   (in0 read with y_B = 0)
// MODE 1 (middle axis): out0 = M in0, out1 = K in0 + M in1
// MODE 2 (last axis):   out0 = s (K in0 + M in1)   or  b - s (...) (RESID)
// One thread owns the K outputs of one cell segment of one grid line.
// ===========================================================================
template <int DIM, int AX, int MODE, bool RESID, typename T>
__device__ __forceinline__ void cart_pass_body(const T* __restrict__ in0, const T* __restrict__ in1,
                                               T* __restrict__ out0, T* __restrict__ out1,
                                               const T* __restrict__ bvec, int n, T s, FastDiv dnp1, FastDiv dN1,
                                               int64_t t0, int64_t tstep) {
  const int N1 = K * n + 1;
  const int64_t lines = DIM == 3 ? (int64_t)N1 * N1 : (int64_t)N1;
  const int64_t total = (int64_t)(n + 1) * lines;
  const T* C = ctab<T>();
  const bool fast = total < kFastDivItems;
  for (int64_t t = t0; t < total; t += tstep) {
    int c, p, q;
    if (fast) {  // 32-bit decoding by the launch's reciprocals
      const uint32_t u = (uint32_t)t;
      if (AX == 0) {
        const uint32_t r = dnp1.div(u);
        c = (int)(u - r * dnp1.d);
        q = (int)dN1.div(r);
        p = (int)(r - (uint32_t)q * dN1.d);
      } else {
        const uint32_t r = dN1.div(u);
        p = (int)(u - r * dN1.d);
        q = (int)dnp1.div(r);
        c = (int)(r - (uint32_t)q * dnp1.d);
      }
    } else if (AX == 0) {
      c = (int)(t % (n + 1));
      const int64_t r = t / (n + 1);
      p = (int)(r % N1);
      q = (int)(r / N1);
    } else {
      p = (int)(t % N1);
      const int64_t r = t / N1;
      c = (int)(r % (n + 1));
      q = (int)(r / (n + 1));
    }
    int64_t base, stride;
    if (DIM == 3) {
      if (AX == 0) { base = ((int64_t)q * N1 + p) * N1; stride = 1; }
      else if (AX == 1) { base = (int64_t)q * N1 * N1 + p; stride = N1; }
      else { base = (int64_t)q * N1 + p; stride = (int64_t)N1 * N1; }
    } else {
      if (AX == 0) { base = (int64_t)p * N1; stride = 1; }
      else { base = p; stride = N1; }
    }
    if (c == n) {  // the last grid node of the line is on the boundary
      const int64_t o = base + (int64_t)K * n * stride;
      out0[o] = T(0);
      if (MODE != 2) out1[o] = T(0);
      continue;
    }
    bool line_zero = false;
    if (MODE == 0) line_zero = (p == 0 || p == N1 - 1 || (DIM == 3 && (q == 0 || q == N1 - 1)));
    T xr0[K + 1], xl0[K + 1], xr1[K + 1], xl1[K + 1];
#pragma unroll
    for (int b = 0; b <= K; ++b) {
      const int g = K * c + b;
      T v = in0[base + (int64_t)g * stride];
      if (MODE == 0 && (line_zero || g == 0 || g == K * n)) v = T(0);
      xr0[b] = v;
      xr1[b] = MODE == 0 ? T(0) : in1[base + (int64_t)g * stride];
      if (c > 0) {
        const int gl = K * (c - 1) + b;
        T w = in0[base + (int64_t)gl * stride];
        if (MODE == 0 && (line_zero || gl == 0)) w = T(0);
        xl0[b] = w;
        xl1[b] = MODE == 0 ? T(0) : in1[base + (int64_t)gl * stride];
      } else {
        xl0[b] = T(0);
        xl1[b] = T(0);
      }
    }
    const T* Me = C + LAY.Me;
    const T* Ke = C + LAY.Ke;
#pragma unroll
    for (int a = 0; a < K; ++a) {
      const int g = K * c + a;
      T m0 = 0, k0 = 0, m1 = 0;
#pragma unroll
      for (int b = 0; b <= K; ++b) {
        m0 += Me[a * (K + 1) + b] * xr0[b];
        k0 += Ke[a * (K + 1) + b] * xr0[b];
        if (MODE != 0) m1 += Me[a * (K + 1) + b] * xr1[b];
      }
      if (a == 0) {  // vertex node: add the row of the left cell
#pragma unroll
        for (int b = 0; b <= K; ++b) {
          m0 += Me[K * (K + 1) + b] * xl0[b];
          k0 += Ke[K * (K + 1) + b] * xl0[b];
          if (MODE != 0) m1 += Me[K * (K + 1) + b] * xl1[b];
        }
      }
      // node 0 of the line is a boundary node; for the last axis, so is any
      // node whose other coordinates lie on the boundary (y_B = 0, r_B = 0)
      const bool bnd = (g == 0) || (MODE == 2 && (p == 0 || p == N1 - 1 || (DIM == 3 && (q == 0 || q == N1 - 1))));
      const int64_t o = base + (int64_t)g * stride;
      if (MODE == 0) {
        out0[o] = bnd ? T(0) : m0;
        out1[o] = bnd ? T(0) : k0;
      } else if (MODE == 1) {
        out0[o] = bnd ? T(0) : m0;
        out1[o] = bnd ? T(0) : k0 + m1;
      } else {
        T v = s * (k0 + m1);
        if (RESID) v = bvec[o] - v;
        out0[o] = bnd ? T(0) : v;
      }
    }
  }
}

template <int DIM, int AX, int MODE, bool RESID, typename T>
__global__ void __launch_bounds__(256) cart_pass(const T* __restrict__ in0, const T* __restrict__ in1,
                                                 T* __restrict__ out0, T* __restrict__ out1,
                                                 const T* __restrict__ bvec, int n, T s, FastDiv dnp1,
                                                 FastDiv dN1) {
  cart_pass_body<DIM, AX, MODE, RESID, T>(in0, in1, out0, out1, bvec, n, s, dnp1, dN1,
                                          (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                                          (int64_t)gridDim.x * blockDim.x);
}

// ===========================================================================
// First two passes of the 3D apply in one launch (x and y directions of one
// z plane; FP32, where the three passes are bound by memory traffic): a
// block loads a tile of x on plane z -- TO x TO owned nodes plus the rows and
// columns of the neighbouring cells that the 1D matrices reach (K before,
// one after) -- into shared memory, applies M and K along x to every loaded
// row, then M and K along y to the owned nodes, and writes the two results
// of cart_pass MODE 1 (t2 = M_y M_x x, t3 = K_y M_x x + M_y K_x x) for the
// last pass (MODE 2).  x is read about 1.3 times (tile halos, mostly from
// L2) instead of the x pass writing and the y pass re-reading two
// intermediates: 6 words of traffic per node instead of 10.  Every output is
// formed with cart_pass's arithmetic in cart_pass's order, so the results
// are bitwise those of the first two passes.
// ===========================================================================
template <typename T>
struct CartXY {
  static constexpr int CX = K >= 32 ? 1 : 32 / K;  // cells per tile side
  static constexpr int TO = K * CX;                // owned nodes per side
  static constexpr int TH = TO + K + 1;            // loaded nodes per side
  static constexpr int PT = TO | 1;                // row pitch of the x-pass results (odd: no bank conflicts)
};

template <typename T>
__global__ void __launch_bounds__(256) cart_xy_kernel(const T* __restrict__ x, T* __restrict__ t2,
                                                      T* __restrict__ t3, int n) {
  using X = CartXY<T>;
  constexpr int TH = X::TH, PT = X::PT, CX = X::CX, TO = X::TO;
  constexpr int NT = 256;       // threads per block (the launch bound)
  constexpr int RS = NT / TH;   // rows loaded per step of the load loop
  __shared__ T xs[TH * TH];
  __shared__ T s0[TH * PT];
  __shared__ T s1[TH * PT];
  const int N1 = K * n + 1;
  // grid: (tile x, tile y, z plane)
  const int cx0 = blockIdx.x * CX, cy0 = blockIdx.y * CX;
  const int ncx = min(CX, n - cx0), ncy = min(CX, n - cy0);
  const int gz = blockIdx.z;
  const int64_t plane = (int64_t)gz * N1 * N1;
  const bool last_x = cx0 + ncx == n, last_y = cy0 + ncy == n;
  const int OX = K * ncx + (last_x ? 1 : 0), OY = K * ncy + (last_y ? 1 : 0);  // owned nodes
  if (gz == 0 || gz == N1 - 1) {  // x is zero on the boundary planes: so are both results
    for (int i = threadIdx.x; i < OX * OY; i += NT) {
      const int64_t o = plane + (int64_t)(K * cy0 + i / OX) * N1 + K * cx0 + i % OX;
      t2[o] = T(0);
      t3[o] = T(0);
    }
    return;
  }
  const T* C = ctab<T>();
  const T* Me = C + LAY.Me;
  const T* Ke = C + LAY.Ke;
  // x restricted to the free nodes: rows K (cy0 - 1) .. K (cy0 + ncy), columns
  // likewise.  A thread loads one column, every RS-th row.
  const int RY = K * (ncy + 1) + 1, RX = K * (ncx + 1) + 1;
  {
    const int c = threadIdx.x % TH, r0 = threadIdx.x / TH;
    if (r0 < RS && c < RX) {
      const int gx = K * (cx0 - 1) + c;
      const bool col_free = gx >= 1 && gx <= N1 - 2;
      int gy = K * (cy0 - 1) + r0;
      int64_t off = plane + (int64_t)gy * N1 + gx;  // read only where the node is free
      for (int r = r0; r < RY; r += RS, gy += RS, off += (int64_t)RS * N1)
        xs[r * TH + c] = (col_free && gy >= 1 && gy <= N1 - 2) ? x[off] : T(0);
    }
  }
  __syncthreads();
  // x pass (cart_pass MODE 0) on every loaded row, owned cells; rows fastest
  for (int i = threadIdx.x; i < TH * CX; i += NT) {
    const int cc = i / TH, r = i - cc * TH, c = cx0 + cc;
    if (r >= RY || cc >= ncx) continue;  // outside a partial tile
    T xr0[K + 1], xl0[K + 1];
#pragma unroll
    for (int b = 0; b <= K; ++b) {
      xr0[b] = xs[r * TH + K * (cc + 1) + b];
      xl0[b] = c > 0 ? xs[r * TH + K * cc + b] : T(0);
    }
#pragma unroll
    for (int a = 0; a < K; ++a) {
      T m0 = 0, k0 = 0;
#pragma unroll
      for (int b = 0; b <= K; ++b) {
        m0 += Me[a * (K + 1) + b] * xr0[b];
        k0 += Ke[a * (K + 1) + b] * xr0[b];
      }
      if (a == 0) {
#pragma unroll
        for (int b = 0; b <= K; ++b) {
          m0 += Me[K * (K + 1) + b] * xl0[b];
          k0 += Ke[K * (K + 1) + b] * xl0[b];
        }
      }
      const bool bnd = K * c + a == 0;
      s0[r * PT + K * cc + a] = bnd ? T(0) : m0;
      s1[r * PT + K * cc + a] = bnd ? T(0) : k0;
    }
  }
  __syncthreads();
  // y pass (cart_pass MODE 1) on the owned nodes; columns fastest (coalesced stores)
  const int CW = K * ncx;
  for (int i = threadIdx.x; i < TO * CX; i += NT) {
    const int cc = i / TO, j = i - cc * TO, cy = cy0 + cc;
    if (j >= CW || cc >= ncy) continue;
    T xr0[K + 1], xl0[K + 1], xr1[K + 1], xl1[K + 1];
#pragma unroll
    for (int b = 0; b <= K; ++b) {
      xr0[b] = s0[(K * (cc + 1) + b) * PT + j];
      xr1[b] = s1[(K * (cc + 1) + b) * PT + j];
      xl0[b] = cy > 0 ? s0[(K * cc + b) * PT + j] : T(0);
      xl1[b] = cy > 0 ? s1[(K * cc + b) * PT + j] : T(0);
    }
    const int64_t col = plane + K * cx0 + j;
#pragma unroll
    for (int a = 0; a < K; ++a) {
      T m0 = 0, k0 = 0, m1 = 0;
#pragma unroll
      for (int b = 0; b <= K; ++b) {
        m0 += Me[a * (K + 1) + b] * xr0[b];
        k0 += Ke[a * (K + 1) + b] * xr0[b];
        m1 += Me[a * (K + 1) + b] * xr1[b];
      }
      if (a == 0) {
#pragma unroll
        for (int b = 0; b <= K; ++b) {
          m0 += Me[K * (K + 1) + b] * xl0[b];
          k0 += Ke[K * (K + 1) + b] * xl0[b];
          m1 += Me[K * (K + 1) + b] * xl1[b];
        }
      }
      const int g = K * cy + a;
      const bool bnd = g == 0;
      const int64_t o = col + (int64_t)g * N1;
      t2[o] = bnd ? T(0) : m0;
      t3[o] = bnd ? T(0) : k0 + m1;
    }
  }
  // the last node of a line is on the boundary: zero (as the passes write it)
  if (last_y)
    for (int j = threadIdx.x; j < OX; j += NT) {
      const int64_t o = plane + (int64_t)(N1 - 1) * N1 + K * cx0 + j;
      t2[o] = T(0);
      t3[o] = T(0);
    }
  if (last_x)
    for (int r = threadIdx.x; r < K * ncy; r += NT) {
      const int64_t o = plane + (int64_t)(K * cy0 + r) * N1 + N1 - 1;
      t2[o] = T(0);
      t3[o] = T(0);
    }
}

// Grouped launch: the same pass over every job's level (jobs of one launch
// may have different n); the grid covers the concatenated work items of the
// jobs (G.start), each computed by the ungrouped body, so a job's outputs
// are those of its own launch.
template <typename T>
struct CartPassJob {
  const T* in0;
  const T* in1;
  T* out0;
  T* out1;
  const T* bvec;
  int n;
  T s;
  FastDiv dnp1, dN1;  // n + 1, K n + 1
};

template <int DIM, int AX, int MODE, bool RESID, typename T>
__global__ void __launch_bounds__(256) cart_pass_group(const __grid_constant__ GroupOf<CartPassJob<T>> G) {
  const int64_t total = G.start[G.count];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = group_find(G, t);
    const CartPassJob<T>& a = G.job[j];
    cart_pass_body<DIM, AX, MODE, RESID, T>(a.in0, a.in1, a.out0, a.out1, a.bvec, a.n, a.s, a.dnp1, a.dN1,
                                            t - G.start[j], kOneItem);
  }
}

// ===========================================================================
// The same three passes in float-float arithmetic: FP64 input x and output y,
// every product and sum carried as an unevaluated pair of floats (hi + lo,
// about 48 significant bits) on the FP32 pipes, which on GB300 run about 60x
// faster than FP64.  Error-free transformations: Knuth's TwoSum (s + e = a + b
// exactly) and the FMA TwoProduct (p + e = a b exactly); sums keep their hi
// part by TwoSum and collect every low-order part in a float accumulator,
// renormalised at the end (Dekker's FastTwoSum).  Coefficients are split
// into float pairs from the FP64 tables at compile time.  Intermediates are
// float-pair planes: a vector of N pairs stored as N his then N los.
// ===========================================================================
struct ff {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ ff ff_of(double v) {
  const float h = (float)v;
  return ff{h, (float)(v - (double)h)};
}

// hi/lo split of the FP64 coefficient c (constant-folded when c is)
__device__ __forceinline__ ff ff_const(double c) { return ff_of(c); }

// running sum of products c_j x_j
struct ff_acc {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void mac(ff c, ff x) {
    const float p = c.hi * x.hi;
    float t = __fmaf_rn(c.hi, x.hi, -p);  // exact: p + t = c.hi x.hi
    t = __fmaf_rn(c.hi, x.lo, t);
    t = __fmaf_rn(c.lo, x.hi, t);
    float e;
    two_sum(hi, p, hi, e);
    lo += e + t;
  }
  __device__ __forceinline__ void add(ff_acc o) {
    float e;
    two_sum(hi, o.hi, hi, e);
    lo += e + o.lo;
  }
  __device__ __forceinline__ ff value() const {
    const float s = hi + lo;  // FastTwoSum (|hi| >= |lo|)
    return ff{s, lo - (s - hi)};
  }
};

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = a.hi * b.hi;
  float t = __fmaf_rn(a.hi, b.hi, -p);
  t = __fmaf_rn(a.hi, b.lo, t);
  t = __fmaf_rn(a.lo, b.hi, t);
  const float s = p + t;
  return ff{s, t - (s - p)};
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// MODE as cart_pass; in0 is FP64 in MODE 0 (x), else a float-pair plane;
// out0 / out1 are float-pair planes in MODE 0, 1; in MODE 2 out0 is FP64.
template <int DIM, int AX, int MODE, bool RESID>
__device__ __forceinline__ void cart_pass_ff_body(const void* __restrict__ in0_, const float* __restrict__ in1,
                                                  void* __restrict__ out0_, float* __restrict__ out1,
                                                  const double* __restrict__ bvec, int n, ff s, FastDiv dnp1,
                                                  FastDiv dN1, int64_t t0, int64_t tstep) {
  const int N1 = K * n + 1;
  const int64_t lines = DIM == 3 ? (int64_t)N1 * N1 : (int64_t)N1;
  const int64_t total = (int64_t)(n + 1) * lines;
  const int64_t NN = DIM == 3 ? (int64_t)N1 * N1 * N1 : (int64_t)N1 * N1;  // plane length
  const double* xin = static_cast<const double*>(in0_);
  const float* in0 = static_cast<const float*>(in0_);
  float* out0 = static_cast<float*>(out0_);
  double* yout = static_cast<double*>(out0_);
  const double* C = ctab<double>();
  auto load0 = [&](int64_t o) -> ff {
    if constexpr (MODE == 0) return ff_of(xin[o]);
    else return ff{in0[o], in0[NN + o]};
  };
  auto load1 = [&](int64_t o) -> ff { return ff{in1[o], in1[NN + o]}; };
  auto store = [&](float* pl, int64_t o, ff v) {
    pl[o] = v.hi;
    pl[NN + o] = v.lo;
  };
  const bool fast = total < kFastDivItems;
  for (int64_t t = t0; t < total; t += tstep) {
    int c, p, q;
    if (fast) {  // 32-bit decoding by the launch's reciprocals
      const uint32_t u = (uint32_t)t;
      if (AX == 0) {
        const uint32_t r = dnp1.div(u);
        c = (int)(u - r * dnp1.d);
        q = (int)dN1.div(r);
        p = (int)(r - (uint32_t)q * dN1.d);
      } else {
        const uint32_t r = dN1.div(u);
        p = (int)(u - r * dN1.d);
        q = (int)dnp1.div(r);
        c = (int)(r - (uint32_t)q * dnp1.d);
      }
    } else if (AX == 0) {
      c = (int)(t % (n + 1));
      const int64_t r = t / (n + 1);
      p = (int)(r % N1);
      q = (int)(r / N1);
    } else {
      p = (int)(t % N1);
      const int64_t r = t / N1;
      c = (int)(r % (n + 1));
      q = (int)(r / (n + 1));
    }
    int64_t base, stride;
    if (DIM == 3) {
      if (AX == 0) { base = ((int64_t)q * N1 + p) * N1; stride = 1; }
      else if (AX == 1) { base = (int64_t)q * N1 * N1 + p; stride = N1; }
      else { base = (int64_t)q * N1 + p; stride = (int64_t)N1 * N1; }
    } else {
      if (AX == 0) { base = (int64_t)p * N1; stride = 1; }
      else { base = p; stride = N1; }
    }
    if (c == n) {  // the last grid node of the line is on the boundary
      const int64_t o = base + (int64_t)K * n * stride;
      if (MODE == 2) yout[o] = 0.0;
      else { store(out0, o, ff{0.f, 0.f}); store(out1, o, ff{0.f, 0.f}); }
      continue;
    }
    bool line_zero = false;
    if (MODE == 0) line_zero = (p == 0 || p == N1 - 1 || (DIM == 3 && (q == 0 || q == N1 - 1)));
    ff xr0[K + 1], xl0[K + 1], xr1[K + 1], xl1[K + 1];
#pragma unroll
    for (int b = 0; b <= K; ++b) {
      const int g = K * c + b;
      ff v = load0(base + (int64_t)g * stride);
      if (MODE == 0 && (line_zero || g == 0 || g == K * n)) v = ff{0.f, 0.f};
      xr0[b] = v;
      xr1[b] = MODE == 0 ? ff{0.f, 0.f} : load1(base + (int64_t)g * stride);
      if (c > 0) {
        const int gl = K * (c - 1) + b;
        ff w = load0(base + (int64_t)gl * stride);
        if (MODE == 0 && (line_zero || gl == 0)) w = ff{0.f, 0.f};
        xl0[b] = w;
        xl1[b] = MODE == 0 ? ff{0.f, 0.f} : load1(base + (int64_t)gl * stride);
      } else {
        xl0[b] = ff{0.f, 0.f};
        xl1[b] = ff{0.f, 0.f};
      }
    }
#pragma unroll
    for (int a = 0; a < K; ++a) {
      const int g = K * c + a;
      ff_acc m0, k0, m1;
#pragma unroll
      for (int b = 0; b <= K; ++b) {
        const ff me = ff_const(C[LAY.Me + a * (K + 1) + b]), ke = ff_const(C[LAY.Ke + a * (K + 1) + b]);
        m0.mac(me, xr0[b]);
        k0.mac(ke, xr0[b]);
        if (MODE != 0) m1.mac(me, xr1[b]);
      }
      if (a == 0) {  // vertex node: add the row of the left cell
#pragma unroll
        for (int b = 0; b <= K; ++b) {
          const ff me = ff_const(C[LAY.Me + K * (K + 1) + b]), ke = ff_const(C[LAY.Ke + K * (K + 1) + b]);
          m0.mac(me, xl0[b]);
          k0.mac(ke, xl0[b]);
          if (MODE != 0) m1.mac(me, xl1[b]);
        }
      }
      const bool bnd = (g == 0) || (MODE == 2 && (p == 0 || p == N1 - 1 || (DIM == 3 && (q == 0 || q == N1 - 1))));
      const int64_t o = base + (int64_t)g * stride;
      if (MODE == 0) {
        store(out0, o, bnd ? ff{0.f, 0.f} : m0.value());
        store(out1, o, bnd ? ff{0.f, 0.f} : k0.value());
      } else if (MODE == 1) {
        k0.add(m1);
        store(out0, o, bnd ? ff{0.f, 0.f} : m0.value());
        store(out1, o, bnd ? ff{0.f, 0.f} : k0.value());
      } else {
        k0.add(m1);
        double v = ff_to_double(ff_mul(s, k0.value()));
        if (RESID) v = bvec[o] - v;
        yout[o] = bnd ? 0.0 : v;
      }
    }
  }
}

template <int DIM, int AX, int MODE, bool RESID>
__global__ void __launch_bounds__(256) cart_pass_ff(const void* __restrict__ in0, const float* __restrict__ in1,
                                                    void* __restrict__ out0, float* __restrict__ out1,
                                                    const double* __restrict__ bvec, int n, ff s, FastDiv dnp1,
                                                    FastDiv dN1) {
  cart_pass_ff_body<DIM, AX, MODE, RESID>(in0, in1, out0, out1, bvec, n, s, dnp1, dN1,
                                          (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                                          (int64_t)gridDim.x * blockDim.x);
}

struct CartPassFFJob {
  const void* in0;
  const float* in1;
  void* out0;
  float* out1;
  const double* bvec;
  int n;
  ff s;
  FastDiv dnp1, dN1;
};

template <int DIM, int AX, int MODE, bool RESID>
__global__ void __launch_bounds__(256) cart_pass_ff_group(const __grid_constant__ GroupOf<CartPassFFJob> G) {
  const int64_t total = G.start[G.count];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = group_find(G, t);
    const CartPassFFJob& a = G.job[j];
    cart_pass_ff_body<DIM, AX, MODE, RESID>(a.in0, a.in1, a.out0, a.out1, a.bvec, a.n, a.s, a.dnp1, a.dN1,
                                            t - G.start[j], kOneItem);
  }
}

// ===========================================================================
// Vertex-patch smoother with the local p-multigrid solver (§2.1, §2.2, §3).
// A thread block owns `np` patches, processed in lockstep.  Every step of
// the local V-cycle is a set of independent 1D line contractions (or
// element-wise updates); the (patch, line) pairs of all patches of the block
// are spread over all threads, so warps stay full at every p-level (an idle
// lane of an active warp still occupies the FP64 pipe; an idle warp does
// not).  Per-patch shared memory, in elements of T:
//   [t0 | t1 | r_top | d_top | r_{top-1} | d_{top-1} | ... | r_0 d_0 | (rj | ds)]
// ===========================================================================
template <int DIM>
struct PatchShape {
  static constexpr int L = nlev(K);
  static constexpr int M(int l) { return mp(plev(K, l)); }
  static constexpr int MT = mp(K);
  static constexpr int SZ(int l) { return ipow(M(l), DIM); }
  static constexpr int SZT = ipow(MT, DIM);
  static constexpr int TPP = ipow(MT, DIM - 1);  // lines of a top-level step
  static constexpr int off_r(int l) {
    int o = 2 * SZT;
    for (int j = L - 1; j > l; --j) o += 2 * SZ(j);
    return o;
  }
  static constexpr int off_d(int l) { return off_r(l) + (l == 0 ? 1 : SZ(l)); }
  static constexpr int ELEMS = ((off_r(0) + 2) + 1) / 2 * 2;
  // Elements between consecutive patches of a block in the patch-major
  // layout (N_iter > 1 adds r_j and the running correction).  FP32: padded
  // to 17 mod 32 so that the lines of the two patches a warp may straddle
  // fall on different banks (a bank model of the residual passes at k = 4
  // gives 1.76 instead of 1.94 wavefronts per warp access).  FP64 work is
  // bound by the FP64 pipe, not by shared memory: unpadded.
  template <typename T>
  static constexpr int stride(int n_iter) {
    const int e = ELEMS + (n_iter > 1 ? 2 * SZT : 0);
    return sizeof(T) == 8 ? e : e + ((17 - e % 32) + 32) % 32;
  }
};

constexpr int kMaxPatchesPerBlock = 64;

// Inverse-diagonal tables of the Cartesian patch levels p > 1 (scale-free,
// one table per level): a block stages them in shared memory when they are
// small; the larger tables of k >= 6 (6-23 KB per block) are read through
// L1 instead, which leaves that shared memory to further blocks on the SM
// (at k = 7 a block of 5 patches otherwise takes 190 KB, one block per SM).
template <int DIM>
constexpr int patch_dinv_len() {
  int len = 0;
  for (int l = 1; l < nlev(K); ++l) len += ipow(mp(plev(K, l)), DIM);
  return len;
}
template <int DIM, typename T>
constexpr bool stage_dinv() { return patch_dinv_len<DIM>() * (int)sizeof(T) <= 4096; }

template <int AX, int EX, int EY, int EZ>
__device__ __forceinline__ int line_base(int L) {
  if constexpr (AX == 0) return L * EX;
  else if constexpr (AX == 1) return (L % EX) + EX * EY * (L / EX);
  else return L;
}

// Shared memory of the patches of one block, in one of two layouts.
//   IL = 0: patch-major; patch g's elements at base + g * stride (np patches).
//   IL > 0: element-major, IL patches interleaved; element e of patch g at
//           base[e * IL + g] (np = IL).  Work items are mapped patch-fastest,
//           so a warp's lanes hold IL patches at 32 / IL consecutive items.
//           Every tile of the patch has odd row and plane pitches (2p - 1 is
//           odd), so consecutive lines start at addresses of alternating
//           parity: with IL = 16 an FP32 warp access touches 32 distinct
//           banks and an FP64 one two 128-byte rows -- no bank conflicts,
//           whatever the line direction (the lanes of the paper's SIMD
//           vectorisation across cells, here across patches).
template <typename T, int IL_>
struct PBlock {
  using value_type = T;
  static constexpr int IL = IL_;
  T* base;
  int stride;  // elements per patch
  int np;      // patches in the block
  struct Ref {
    T* p;
    __device__ __forceinline__ T& operator[](int e) const { return p[IL ? e * IL : e]; }
  };
  __device__ __forceinline__ Ref at(int g) const { return Ref{IL ? base + g : base + g * stride}; }
};

// for every (g, i), g < np, i < COUNT, spread over the block's threads
template <int COUNT, class F>
__device__ __forceinline__ void pfor_n(int np, F&& f) {
  const int total = np * COUNT;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int g = t / COUNT;
    f(g, t - g * COUNT);
  }
}

// the same over the patches of a PBlock, in its layout's item order
template <int COUNT, class PB, class F>
__device__ __forceinline__ void pfor(const PB& pb, F&& f) {
  if constexpr (PB::IL == 0) {
    pfor_n<COUNT>(pb.np, f);
  } else {
    constexpr int total = PB::IL * COUNT;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
      const int i = t / PB::IL;
      f(t - i * PB::IL, i);
    }
  }
}

// y = C x for a patch matrix of degree p (m x m, row-major), skipping the
// structural zeros between the two cells of the patch.
template <int p, typename T>
__device__ __forceinline__ void pmv(const T* C, const T* x, T* y) {
  constexpr int m = mp(p);
#pragma unroll
  for (int i = 0; i < m; ++i) {
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < m; ++j)
      if (pnz(p, p, i, j)) acc += C[i * m + j] * x[j];
    y[i] = acc;
  }
}

// Cartesian patch geometry: A_{j,p} = s sum_dir (KP on dir, MP elsewhere);
// inverse diagonal from a table shared by all patches (scale-free).
template <int DIM, typename T>
struct CartGeo {
  const T* dinv;  // concatenated per-level tables, level l at dinv_off(l)
  T scale;
  T inv_scale;
  T inv_a0;

  static constexpr int dinv_off(int l) {
    int o = 0;
    for (int j = 1; j < l; ++j) o += ipow(mp(plev(K, j)), DIM);
    return o;
  }
  __device__ __forceinline__ T dinv_at(int, int l, int i) const { return dinv[dinv_off(l) + i] * inv_scale; }
  __device__ __forceinline__ T a0inv(int) const { return inv_a0; }

  // The Jacobi steps of Algorithm 3 fold into the line passes of the
  // residual (no separate pointwise pass over the patch):
  //   MODE 0: out = r - A_l d;
  //   MODE 1: d = om D^-1 r first (pre-smoothing from a zero guess, written
  //           to d by the first pass), then out = r - A_l d;
  //   MODE 2: d += om D^-1 (r - A_l d) (post-smoothing; out not written).
  // Offsets within a patch; out may be t0 = offset 0; d and r distinct from
  // t0, t1.
  static constexpr bool kFusedSmoothing = true;
  template <int l, int MODE = 0, class PB>
  __device__ __forceinline__ void resid(const PB& pb, int od, int orr, int oo, T om = T(0)) const {
    constexpr int p = plev(K, l);
    constexpr int m = mp(p);
    constexpr int SZT = PatchShape<DIM>::SZT;
    const T* MP = ctab<T>() + LAY.MP[l];
    const T* KP = ctab<T>() + LAY.KP[l];
    const T s = scale;
    // first pass, along x: x = d (MODE 1: computed from r and stored)
    auto first = [&](auto sm, int b, T* x) {
#pragma unroll
      for (int j = 0; j < m; ++j) {
        if constexpr (MODE == 1) {
          const T v = om * dinv_at(0, l, b + j) * sm[orr + b + j];
          sm[od + b + j] = v;
          x[j] = v;
        } else {
          x[j] = sm[od + b + j];
        }
      }
    };
    // last pass: the residual t_e at patch element e
    auto last = [&](auto sm, int e, T t) {
      if constexpr (MODE == 2) sm[od + e] += om * dinv_at(0, l, e) * t;
      else sm[oo + e] = t;
    };
    if constexpr (DIM == 3) {
      pfor<m * m>(pb, [&](int g, int L) {
        auto sm = pb.at(g);
        const int b = line_base<0, m, m, m>(L);
        T x[m], y0[m], y1[m];
        first(sm, b, x);
        pmv<p>(MP, x, y0);
        pmv<p>(KP, x, y1);
#pragma unroll
        for (int i = 0; i < m; ++i) { sm[b + i] = y0[i]; sm[SZT + b + i] = y1[i]; }
      });
      __syncthreads();
      pfor<m * m>(pb, [&](int g, int L) {
        auto sm = pb.at(g);
        const int b = line_base<1, m, m, m>(L);
        T a[m], c[m], y0[m], y1[m], y2[m];
#pragma unroll
        for (int j = 0; j < m; ++j) { a[j] = sm[b + j * m]; c[j] = sm[SZT + b + j * m]; }
        pmv<p>(MP, a, y0);
        pmv<p>(KP, a, y1);
        pmv<p>(MP, c, y2);
#pragma unroll
        for (int i = 0; i < m; ++i) { sm[b + i * m] = y0[i]; sm[SZT + b + i * m] = y1[i] + y2[i]; }
      });
      __syncthreads();
      pfor<m * m>(pb, [&](int g, int L) {
        auto sm = pb.at(g);
        const int b = line_base<2, m, m, m>(L);
        T a[m], c[m], y1[m], y2[m];
#pragma unroll
        for (int j = 0; j < m; ++j) { a[j] = sm[b + j * m * m]; c[j] = sm[SZT + b + j * m * m]; }
        pmv<p>(KP, a, y1);
        pmv<p>(MP, c, y2);
#pragma unroll
        for (int i = 0; i < m; ++i) last(sm, b + i * m * m, sm[orr + b + i * m * m] - s * (y1[i] + y2[i]));
      });
      __syncthreads();
    } else {
      pfor<m>(pb, [&](int g, int L) {
        auto sm = pb.at(g);
        const int b = line_base<0, m, m, 1>(L);
        T x[m], y0[m], y1[m];
        first(sm, b, x);
        pmv<p>(MP, x, y0);
        pmv<p>(KP, x, y1);
#pragma unroll
        for (int i = 0; i < m; ++i) { sm[b + i] = y0[i]; sm[SZT + b + i] = y1[i]; }
      });
      __syncthreads();
      pfor<m>(pb, [&](int g, int L) {
        auto sm = pb.at(g);
        const int b = line_base<1, m, m, 1>(L);
        T a[m], c[m], y1[m], y2[m];
#pragma unroll
        for (int j = 0; j < m; ++j) { a[j] = sm[b + j * m]; c[j] = sm[SZT + b + j * m]; }
        pmv<p>(KP, a, y1);
        pmv<p>(MP, c, y2);
#pragma unroll
        for (int i = 0; i < m; ++i) last(sm, b + i * m, sm[orr + b + i * m] - s * (y1[i] + y2[i]));
      });
      __syncthreads();
    }
  }
};

// Restriction: level l-1 residual at `dst` = T_l^T (level-l vector in t0),
// using t1 (and t0 again in 3D) as intermediates.
template <int DIM, int l, class PB>
__device__ __forceinline__ void restrict_p(const PB& pb, int dst) {
  using T = typename PB::value_type;
  constexpr int pf = plev(K, l), pc = plev(K, l - 1);
  constexpr int m = mp(pf), mc = mp(pc);
  constexpr int SZT = PatchShape<DIM>::SZT;
  constexpr int EZ = DIM == 3 ? m : 1;
  const T* Tr = ctab<T>() + LAY.Tr[l];  // m x mc, row-major
  // x: (m, m, EZ) in t0 -> (mc, m, EZ) in t1
  pfor<m * EZ>(pb, [&](int g, int L) {
    auto sm = pb.at(g);
    const int bi = line_base<0, m, m, EZ>(L), bo = line_base<0, mc, m, EZ>(L);
    T x[m];
#pragma unroll
    for (int j = 0; j < m; ++j) x[j] = sm[bi + j];
#pragma unroll
    for (int i = 0; i < mc; ++i) {
      T acc = T(0);
#pragma unroll
      for (int j = 0; j < m; ++j)
        if (pnz(pf, pc, j, i)) acc += Tr[j * mc + i] * x[j];
      sm[SZT + bo + i] = acc;
    }
  });
  __syncthreads();
  // y: (mc, m, EZ) in t1 -> (mc, mc, EZ) in t0 (2D: directly into dst)
  const int ydst = DIM == 3 ? 0 : dst;
  pfor<mc * EZ>(pb, [&](int g, int L) {
    auto sm = pb.at(g);
    const int bi = line_base<1, mc, m, EZ>(L), bo = line_base<1, mc, mc, EZ>(L);
    T x[m];
#pragma unroll
    for (int j = 0; j < m; ++j) x[j] = sm[SZT + bi + j * mc];
#pragma unroll
    for (int i = 0; i < mc; ++i) {
      T acc = T(0);
#pragma unroll
      for (int j = 0; j < m; ++j)
        if (pnz(pf, pc, j, i)) acc += Tr[j * mc + i] * x[j];
      sm[ydst + bo + i * mc] = acc;
    }
  });
  __syncthreads();
  if constexpr (DIM == 3) {
    pfor<mc * mc>(pb, [&](int g, int L) {
      auto sm = pb.at(g);
      const int bi = line_base<2, mc, mc, m>(L), bo = line_base<2, mc, mc, mc>(L);
      T x[m];
#pragma unroll
      for (int j = 0; j < m; ++j) x[j] = sm[bi + j * mc * mc];
#pragma unroll
      for (int i = 0; i < mc; ++i) {
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < m; ++j)
          if (pnz(pf, pc, j, i)) acc += Tr[j * mc + i] * x[j];
        sm[dst + bo + i * mc * mc] = acc;
      }
    });
    __syncthreads();
  }
}

// Prolongation: level-l vector at `dst` += T_l (level l-1 vector at `src`),
// using t0, t1.
template <int DIM, int l, class PB>
__device__ __forceinline__ void prolong_p(const PB& pb, int src, int dst) {
  using T = typename PB::value_type;
  constexpr int pf = plev(K, l), pc = plev(K, l - 1);
  constexpr int m = mp(pf), mc = mp(pc);
  constexpr int SZT = PatchShape<DIM>::SZT;
  constexpr int EZC = DIM == 3 ? mc : 1;
  const T* Tr = ctab<T>() + LAY.Tr[l];
  // x: (mc, mc, EZC) -> (m, mc, EZC) in t0
  pfor<mc * EZC>(pb, [&](int g, int L) {
    auto sm = pb.at(g);
    const int bi = line_base<0, mc, mc, EZC>(L), bo = line_base<0, m, mc, EZC>(L);
    T x[mc];
#pragma unroll
    for (int j = 0; j < mc; ++j) x[j] = sm[src + bi + j];
#pragma unroll
    for (int i = 0; i < m; ++i) {
      T acc = T(0);
#pragma unroll
      for (int j = 0; j < mc; ++j)
        if (pnz(pf, pc, i, j)) acc += Tr[i * mc + j] * x[j];
      sm[bo + i] = acc;
    }
  });
  __syncthreads();
  if constexpr (DIM == 3) {
    // y: (m, mc, mc) in t0 -> (m, m, mc) in t1
    pfor<m * mc>(pb, [&](int g, int L) {
      auto sm = pb.at(g);
      const int bi = line_base<1, m, mc, mc>(L), bo = line_base<1, m, m, mc>(L);
      T x[mc];
#pragma unroll
      for (int j = 0; j < mc; ++j) x[j] = sm[bi + j * m];
#pragma unroll
      for (int i = 0; i < m; ++i) {
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < mc; ++j)
          if (pnz(pf, pc, i, j)) acc += Tr[i * mc + j] * x[j];
        sm[SZT + bo + i * m] = acc;
      }
    });
    __syncthreads();
    // z: (m, m, mc) in t1 -> (m, m, m) added into dst
    pfor<m * m>(pb, [&](int g, int L) {
      auto sm = pb.at(g);
      const int bi = line_base<2, m, m, mc>(L), bo = line_base<2, m, m, m>(L);
      T x[mc];
#pragma unroll
      for (int j = 0; j < mc; ++j) x[j] = sm[SZT + bi + j * m * m];
#pragma unroll
      for (int i = 0; i < m; ++i) {
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < mc; ++j)
          if (pnz(pf, pc, i, j)) acc += Tr[i * mc + j] * x[j];
        sm[dst + bo + i * m * m] += acc;
      }
    });
    __syncthreads();
  } else {
    // y: (m, mc) in t0 -> (m, m) added into dst
    pfor<m>(pb, [&](int g, int L) {
      auto sm = pb.at(g);
      const int bi = line_base<1, m, mc, 1>(L), bo = line_base<1, m, m, 1>(L);
      T x[mc];
#pragma unroll
      for (int j = 0; j < mc; ++j) x[j] = sm[bi + j * m];
#pragma unroll
      for (int i = 0; i < m; ++i) {
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < mc; ++j)
          if (pnz(pf, pc, i, j)) acc += Tr[i * mc + j] * x[j];
        sm[dst + bo + i * m] += acc;
      }
    });
    __syncthreads();
  }
}

// Algorithm 3 on p-level l for the residuals r_l of all patches of the
// block, results in d_l; level 0 (p = 1) is the exact 1x1 solve (§3.2).
// Full V-cycle, or with P.half the half V-cycle of §3.2.2 (pre-smoothing,
// coarse correction, no post-smoothing).
template <int DIM, int l, class PB, class Geo>
__device__ void pvcycle(const PB& pb, const Geo& geo, const PatchParams<typename PB::value_type>& P) {
  using T = typename PB::value_type;
  using S = PatchShape<DIM>;
  if constexpr (l == 0) {
    pfor<1>(pb, [&](int g, int) {
      auto sm = pb.at(g);
      sm[S::off_d(0)] = sm[S::off_r(0)] * geo.a0inv(g);
    });
    __syncthreads();
  } else {
    constexpr int SZ = S::SZ(l);
    constexpr int R = S::off_r(l), D = S::off_d(l);
    const T om = P.omega[l];
    if constexpr (Geo::kFusedSmoothing) {
      geo.template resid<l, 1>(pb, D, R, 0, om);  // pre-smoothing (zero guess) + residual into t0
    } else {
      pfor<SZ>(pb, [&](int g, int i) {  // pre-smoothing (zero initial guess)
        auto sm = pb.at(g);
        sm[D + i] = om * geo.dinv_at(g, l, i) * sm[R + i];
      });
      __syncthreads();
      geo.template resid<l>(pb, D, R, 0);  // residual into t0
    }
    restrict_p<DIM, l>(pb, S::off_r(l - 1));    // restrict
    pvcycle<DIM, l - 1>(pb, geo, P);            // recurse
    prolong_p<DIM, l>(pb, S::off_d(l - 1), D);  // prolongate, add
    if (P.half) return;  // half V-cycle (§3.2.2): no post-smoothing (uniform per block)
    if constexpr (Geo::kFusedSmoothing) {
      geo.template resid<l, 2>(pb, D, R, 0, om);  // residual + post-smoothing
    } else {
      geo.template resid<l>(pb, D, R, 0);  // residual
      pfor<SZ>(pb, [&](int g, int i) {     // post-smoothing
        auto sm = pb.at(g);
        sm[D + i] += om * geo.dinv_at(g, l, i) * sm[i];
      });
      __syncthreads();
    }
  }
}

// Algorithm 2 around Algorithm 3 for every patch of the block: the top-level
// residual in r_top on entry, the correction in d_top on exit.
template <int DIM, class PB, class Geo>
__device__ __forceinline__ void local_solve(const PB& pb, const Geo& geo,
                                            const PatchParams<typename PB::value_type>& P, int n_iter, int extra) {
  using T = typename PB::value_type;
  using S = PatchShape<DIM>;
  constexpr int L = S::L, SZT = S::SZT;
  constexpr int RT = S::off_r(L - 1), DT = S::off_d(L - 1);
  if (n_iter <= 1) {
    pvcycle<DIM, L - 1>(pb, geo, P);
    return;
  }
  const int RJ = extra, DS = extra + SZT;  // keep r_j and the running correction
  pfor<SZT>(pb, [&](int g, int i) { auto sm = pb.at(g); sm[RJ + i] = sm[RT + i]; });
  __syncthreads();
  pvcycle<DIM, L - 1>(pb, geo, P);
  pfor<SZT>(pb, [&](int g, int i) { auto sm = pb.at(g); sm[DS + i] = sm[DT + i]; });
  __syncthreads();
  for (int it = 1; it < n_iter; ++it) {
    geo.template resid<L - 1>(pb, DS, RJ, RT);
    pvcycle<DIM, L - 1>(pb, geo, P);
    pfor<SZT>(pb, [&](int g, int i) { auto sm = pb.at(g); sm[DS + i] += sm[DT + i]; });
    __syncthreads();
  }
  pfor<SZT>(pb, [&](int g, int i) { auto sm = pb.at(g); sm[DT + i] = sm[DS + i]; });
  __syncthreads();
}

// All patches of a level in one launch: patch index pid, lexicographic over
// the interior vertices (x fastest).  Every patch reads the same residual
// (additive smoother), so no colouring is needed to compute the corrections;
// each patch writes omega_AS d_j to its own slot of a per-patch buffer and
// patch_gather_kernel sums, per node, the contributions of the (at most 2^d)
// patches whose interior holds it, in a fixed order.
struct PatchMeta {
  int v[3];
  int g0[3];
  int active;
};

// Patch pid of the launch: lexicographic (x fastest) over all interior
// vertices (colour < 0) or over those of parity colour `colour` (vertex
// index 2 i + 1 for an odd parity bit, 2 i + 2 for an even one).
template <int DIM>
__device__ __forceinline__ void patch_meta_init(PatchMeta* meta, int np, int n, int colour,
                                                int64_t batch = -1) {
  if (batch < 0) batch = blockIdx.x;
  const int c0 = patch_count_1d(n, colour, 0), c1 = patch_count_1d(n, colour, 1);
  const int64_t npatch = patch_count(DIM, n, colour);
  const int step = colour < 0 ? 1 : 2;
  const int b0 = colour < 0 || (colour & 1) ? 1 : 2, b1 = colour < 0 || ((colour >> 1) & 1) ? 1 : 2;
  const int b2 = colour < 0 || ((colour >> 2) & 1) ? 1 : 2;
  for (int g = threadIdx.x; g < np; g += blockDim.x) {
    const int64_t pid = batch * np + g;
    PatchMeta m;
    m.active = pid < npatch;
    int64_t t = m.active ? pid : 0;
    m.v[0] = b0 + step * (int)(t % c0);
    t /= c0;
    m.v[1] = b1 + step * (int)(t % c1);
    t /= c1;
    m.v[2] = DIM == 3 ? b2 + step * (int)t : 0;
    for (int d = 0; d < 3; ++d) m.g0[d] = (d < DIM) ? K * (m.v[d] - 1) + 1 : 0;
    meta[g] = m;
  }
}

// Parity colour of a patch's vertex; patches of one colour have disjoint
// interiors, so each node has at most one patch per colour.
template <int DIM>
__device__ __forceinline__ int patch_colour(const PatchMeta& m) {
  return (m.v[0] & 1) | ((m.v[1] & 1) << 1) | (DIM == 3 ? ((m.v[2] & 1) << 2) : 0);
}

template <int DIM>
__device__ __forceinline__ int64_t patch_node(const PatchMeta& m, int i, int N1) {
  constexpr int MT = mp(K);
  const int ix = i % MT, iy = (i / MT) % MT, iz = DIM == 3 ? i / (MT * MT) : 0;
  return (int64_t)(m.g0[0] + ix) + (int64_t)N1 * ((m.g0[1] + iy) + (int64_t)N1 * (m.g0[2] + iz));
}

// Cartesian patches: gather r_j, Algorithm 2/3, write omega_AS d_j
// (additive), or add d_j to u for the patches of one colour (multiplicative).
// FP64, degrees up to 4: at most 256 threads per block and three blocks per
// SM (registers <= 85), so that 24 warps keep the FP64 pipe fed.  Higher
// degrees need more registers per line than that without spilling, and the
// FP32 kernels (40 registers, shared-memory bound) run fastest with the
// compiler's own choice and larger blocks (measured: bounding k = 7 to 256
// threads made its FP32 launch 40% slower, k = 4 FP32 3% slower).
#if PMG_K <= 4 && PMG_PREC == 0
#define PMG_PATCH_BOUNDS __launch_bounds__(256, 3)
constexpr int kPatchMaxThreads = 256;
#else
#define PMG_PATCH_BOUNDS
constexpr int kPatchMaxThreads = 1024;
#endif

// Interleave width of this part's interleaved patch kernel: the largest
// power of two up to 16 whose block of patches (one local V-cycle each,
// N_iter = 1) fits the shared memory a block may request, or 0 (no
// interleaved kernel; 3D FP64 k = 8).
template <int DIM, typename T>
constexpr int patch_il() {
  constexpr int per_patch = PatchShape<DIM>::ELEMS * (int)sizeof(T);
  int il = 16;
  while (il > 1 && il * per_patch > kMaxDynSmem - 8 * 1024) il /= 2;
  return il > 1 ? il : 0;
}

// Body of the Cartesian patch kernels: gather r_j, Algorithm 2/3, write
// omega_AS d_j (additive), or add d_j to u for the patches of one colour
// (multiplicative).  IL: layout of the block's patches (PBlock).
// Body of the Cartesian patch kernels for the patches of batch `batch` (np
// patches, lexicographic): gather r_j, Algorithm 2/3, write omega_AS d_j
// (additive), or add d_j to u for the patches of one colour
// (multiplicative).  IL: layout of the block's patches (PBlock); sdinv: the
// inverse-diagonal tables, already staged in shared memory.
template <int DIM, typename T, int IL>
__device__ __forceinline__ void patch_cart_body(const T* __restrict__ r, T* __restrict__ dst, int n, int np,
                                                int n_iter, const T* sdinv, const PatchParams<T>& P,
                                                int64_t batch, PatchMeta* meta, T* smem) {
  using S = PatchShape<DIM>;
  constexpr int SZT = S::SZT;
  constexpr int RT = S::off_r(S::L - 1), DT = S::off_d(S::L - 1);
  const int stride = IL ? S::ELEMS + (n_iter > 1 ? 2 * SZT : 0) : S::template stride<T>(n_iter);
  const PBlock<T, IL> pb{smem, stride, np};
  patch_meta_init<DIM>(meta, np, n, P.colour, batch);
  __syncthreads();
  const int N1 = K * n + 1;
  pfor<SZT>(pb, [&](int g, int i) {  // gather r_j = Pi_j r
    const PatchMeta& m = meta[g];
    pb.at(g)[RT + i] = m.active ? r[patch_node<DIM>(m, i, N1)] : T(0);
  });
  __syncthreads();
  const CartGeo<DIM, T> geo{sdinv, P.scale, P.inv_scale, P.inv_a0};
  local_solve<DIM>(pb, geo, P, n_iter, S::ELEMS);
  const int64_t N = DIM == 3 ? (int64_t)N1 * N1 * N1 : (int64_t)N1 * N1;
  pfor<SZT>(pb, [&](int g, int i) {
    const PatchMeta& m = meta[g];
    if (!m.active) return;
    if (P.colour < 0) dst[patch_colour<DIM>(m) * N + patch_node<DIM>(m, i, N1)] = P.omega_as * pb.at(g)[DT + i];
    else dst[patch_node<DIM>(m, i, N1)] += pb.at(g)[DT + i];  // one patch of the colour per node
  });
}

// Driver of the body.  counter == nullptr: one batch per block (batch =
// blockIdx.x).  Otherwise persistent: the block stages the inverse-diagonal
// tables once, then takes batches of patches from the launch's work counter
// (reset to 0 before every launch) until none is left, so the grid is sized
// to the resident blocks of the GPU and the last batches go to whichever
// blocks finish first.  Each patch's output goes to fixed locations, so the
// result does not depend on which block computed it.
template <int DIM, typename T, int IL>
__device__ __forceinline__ void patch_cart_persistent(const T* __restrict__ r, T* __restrict__ dst, int n, int np,
                                                      int n_iter, const T* __restrict__ dinv, int dinv_len,
                                                      const PatchParams<T>& P, int* counter, int64_t nbatch) {
  using S = PatchShape<DIM>;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ PatchMeta meta[kMaxPatchesPerBlock];
  __shared__ int64_t s_batch;
  const int stride = IL ? S::ELEMS + (n_iter > 1 ? 2 * S::SZT : 0) : S::template stride<T>(n_iter);
  T* smem = reinterpret_cast<T*>(smraw);
  const T* sdinv = dinv;  // inverse-diagonal tables of all p-levels
  if constexpr (stage_dinv<DIM, T>()) {
    T* st = smem + np * stride;
    for (int i = threadIdx.x; i < dinv_len; i += blockDim.x) st[i] = dinv[i];
    sdinv = st;  // visible after the body's first barrier
  }
  if (!counter) {
    patch_cart_body<DIM, T, IL>(r, dst, n, np, n_iter, sdinv, P, blockIdx.x, meta, smem);
    return;
  }
  for (;;) {
    if (threadIdx.x == 0) s_batch = atomicAdd(counter, 1);
    __syncthreads();
    const int64_t batch = s_batch;
    if (batch >= nbatch) break;  // uniform over the block
    patch_cart_body<DIM, T, IL>(r, dst, n, np, n_iter, sdinv, P, batch, meta, smem);
    __syncthreads();  // the batch's shared memory and s_batch are free again
  }
}

// Patch-major layout, np patches per block.  FP64, degrees up to 4: at most
// 256 threads per block and three blocks per SM (registers <= 85), so that
// 24 warps keep the FP64 pipe fed.  Higher degrees need more registers per
// line than that without spilling, and the FP32 kernels (40 registers) run
// fastest with the compiler's own choice and larger blocks (measured:
// bounding k = 7 to 256 threads made its FP32 launch 40% slower, k = 4 FP32
// 3% slower).
template <int DIM, typename T>
__global__ void PMG_PATCH_BOUNDS
    patch_cart_kernel(const T* __restrict__ r, T* __restrict__ dst, int n, int np, int n_iter,
                      const T* __restrict__ dinv, int dinv_len, PatchParams<T> P, int* counter, int64_t nbatch) {
  patch_cart_persistent<DIM, T, 0>(r, dst, n, np, n_iter, dinv, dinv_len, P, counter, nbatch);
}

// Interleaved layout, patch_il() patches per block (np = IL): conflict-free
// shared-memory accesses; the thread count is the autotuner's choice.
#if PMG_PREC == 0
#define PMG_PATCH_IL_BOUNDS __launch_bounds__(768, 1)
#else
#define PMG_PATCH_IL_BOUNDS
#endif
template <int DIM, typename T>
__global__ void PMG_PATCH_IL_BOUNDS
    patch_cart_il_kernel(const T* __restrict__ r, T* __restrict__ dst, int n, int n_iter,
                         const T* __restrict__ dinv, int dinv_len, PatchParams<T> P, int* counter, int64_t nbatch) {
  constexpr int IL = patch_il<DIM, T>() > 0 ? patch_il<DIM, T>() : 1;
  patch_cart_persistent<DIM, T, IL>(r, dst, n, IL, n_iter, dinv, dinv_len, P, counter, nbatch);
}

// Grouped patch launch: the batches of every job (one level of one system;
// the jobs of a launch may differ in n, damping and scale) are numbered job
// after job (G.start: prefix sums of the jobs' batches), and a block finds
// the job of its batch by group_find.  Patch-major layout; counter as patch_cart_persistent (the
// batches of all jobs are one work list, so blocks that finish a small
// system's patches go on to the next system's).  The inverse-diagonal
// tables depend only on the dimension, degree and precision, which every
// job of a launch shares.
template <typename T>
struct PatchJob {
  const T* r;
  T* dst;
  int n;
  PatchParams<T> P;
};

template <int DIM, typename T>
__global__ void PMG_PATCH_BOUNDS patch_cart_group_kernel(int np, int n_iter, const T* __restrict__ dinv, int dinv_len,
                                                         int* counter, int64_t nbatch,
                                                         const __grid_constant__ GroupOf<PatchJob<T>> G) {
  using S = PatchShape<DIM>;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ PatchMeta meta[kMaxPatchesPerBlock];
  __shared__ int64_t s_batch;
  const int stride = S::template stride<T>(n_iter);
  T* smem = reinterpret_cast<T*>(smraw);
  const T* sdinv = dinv;
  if constexpr (stage_dinv<DIM, T>()) {
    T* st = smem + np * stride;
    for (int i = threadIdx.x; i < dinv_len; i += blockDim.x) st[i] = dinv[i];
    sdinv = st;
  }
  int64_t b = blockIdx.x;
  for (;;) {
    if (counter) {
      if (threadIdx.x == 0) s_batch = atomicAdd(counter, 1);
      __syncthreads();
      b = s_batch;
    }
    if (b >= nbatch) break;  // uniform over the block
    const int j = group_find(G, b);
    const PatchJob<T>& J = G.job[j];
    patch_cart_body<DIM, T, 0>(J.r, J.dst, J.n, np, n_iter, sdinv, J.P, b - G.start[j], meta, smem);
    if (!counter) break;
    __syncthreads();  // the batch's shared memory and s_batch are free again
  }
}

// u (+)= sum over the patches whose interior holds the node of their
// correction.  The patch kernels write the correction of a patch of colour c
// at dst[c N + node] (N = nodes of the level); a node is covered by colour c
// when, in every direction, the vertex of parity bit_d(c) among the one or
// two vertices whose patch holds the node lies in 1..n-1.  Fixed order:
// colours 0..2^d-1.  Boundary nodes get no contribution.
template <int DIM, bool ADD, typename T>
__device__ __forceinline__ void patch_gather_body(const T* __restrict__ dst, T* __restrict__ u, int n, FastDiv dN1,
                                                  int64_t t0, int64_t tstep) {
  const int N1 = K * n + 1, nv = n - 1;
  const int64_t N = DIM == 3 ? (int64_t)N1 * N1 * N1 : (int64_t)N1 * N1;
  const bool fast = N < kFastDivItems;
  for (int64_t t = t0; t < N; t += tstep) {
    int gd[3];
    if (fast) {
      const uint32_t v = (uint32_t)t, r = dN1.div(v);
      gd[0] = (int)(v - r * dN1.d);
      if (DIM == 3) {
        const uint32_t z = dN1.div(r);
        gd[1] = (int)(r - z * dN1.d);
        gd[2] = (int)z;
      } else {
        gd[1] = (int)r;
        gd[2] = 0;
      }
    } else {
      gd[0] = (int)(t % N1);
      gd[1] = (int)((t / N1) % N1);
      gd[2] = DIM == 3 ? (int)(t / ((int64_t)N1 * N1)) : 0;
    }
    // per direction and parity: is there a vertex of that parity holding the node?
    unsigned has[3] = {0u, 0u, 0u};
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const int g = gd[d], c = g / K, a = g - K * c;
      if (c >= 1 && c <= nv) has[d] |= 1u << (c & 1);
      if (a != 0 && c + 1 >= 1 && c + 1 <= nv) has[d] |= 1u << ((c + 1) & 1);
    }
    T s = T(0);
#pragma unroll
    for (int col = 0; col < (1 << DIM); ++col) {
      const bool cov = ((has[0] >> (col & 1)) & 1u) && ((has[1] >> ((col >> 1) & 1)) & 1u) &&
                       (DIM == 2 || ((has[2] >> ((col >> 2) & 1)) & 1u));
      if (cov) s += dst[col * N + t];
    }
    if (ADD) u[t] += s;
    else u[t] = s;
  }
}

template <int DIM, bool ADD, typename T>
__global__ void __launch_bounds__(256) patch_gather_kernel(const T* __restrict__ dst, T* __restrict__ u, int n,
                                                           FastDiv dN1) {
  patch_gather_body<DIM, ADD, T>(dst, u, n, dN1, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                                 (int64_t)gridDim.x * blockDim.x);
}

template <typename T>
struct GatherJob {
  const T* dst;
  T* u;
  int n;
  FastDiv dN1;
};

template <int DIM, bool ADD, typename T>
__global__ void __launch_bounds__(256) patch_gather_group(const __grid_constant__ GroupOf<GatherJob<T>> G) {
  const int64_t total = G.start[G.count];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = group_find(G, t);
    patch_gather_body<DIM, ADD, T>(G.job[j].dst, G.job[j].u, G.job[j].n, G.job[j].dN1, t - G.start[j], kOneItem);
  }
}

// ===========================================================================
// h-transfers (Eq. (2)): prolongation = embedding, one pass per axis,
// restriction = its transpose, one pass per axis in reverse order.
// ===========================================================================
// Prolongation along AX: in has extent nc1 = K nc + 1 along AX, out nf1 =
// K (2 nc) + 1; e0, e1 are the extents of the two other axes (x-fastest order
// of the remaining axes).  ADD: out += result.
template <int AX, bool ADD, typename T>
__device__ __forceinline__ void hprolong_body(const T* __restrict__ in, T* __restrict__ out, int nc, int ex, int ey,
                                              int ez, FastDiv dex, FastDiv dey, int64_t t0, int64_t tstep) {
  // ex, ey, ez: extents of the OUTPUT array
  const int nf = 2 * nc;
  const int nc1 = K * nc + 1;
  const int64_t total = (int64_t)ex * ey * ez;
  const T* Pt = coef<T>() + LAY.Pt;
  const bool fast = total < kFastDivItems;
  for (int64_t t = t0; t < total; t += tstep) {
    int x, y, z;
    if (fast) {
      const uint32_t u = (uint32_t)t, rr = dex.div(u), zz = dey.div(rr);
      x = (int)(u - rr * dex.d);
      y = (int)(rr - zz * dey.d);
      z = (int)zz;
    } else {
      x = (int)(t % ex);
      const int64_t rr = t / ex;
      y = (int)(rr % ey);
      z = (int)(rr / ey);
    }
    const int gf = AX == 0 ? x : (AX == 1 ? y : z);
    const int cf = min(gf / K, nf - 1);
    const int a = gf - K * cf;
    const int cc = cf / 2, ch = cf % 2;
    // input extents: same as output except nc1 along AX
    const int ix = AX == 0 ? nc1 : ex, iy = AX == 1 ? nc1 : ey;
    T acc = T(0);
#pragma unroll
    for (int b = 0; b <= K; ++b) {
      const int gc = K * cc + b;
      const int64_t ii = AX == 0 ? (gc + (int64_t)ix * (y + (int64_t)iy * z))
                                 : (AX == 1 ? (x + (int64_t)ix * (gc + (int64_t)iy * z))
                                            : (x + (int64_t)ix * (y + (int64_t)iy * gc)));
      acc += Pt[(ch * (K + 1) + a) * (K + 1) + b] * in[ii];
    }
    if (ADD) out[t] += acc; else out[t] = acc;
  }
}

// Restriction along AX: in has extent nf1 along AX, out nc1; outputs on the
// boundary nodes of AX are zero (restriction acts on free DoFs).
template <int AX, typename T>
__device__ __forceinline__ void hrestrict_body(const T* __restrict__ in, T* __restrict__ out, int nc, int ex, int ey,
                                               int ez, FastDiv dex, FastDiv dey, int64_t t0, int64_t tstep) {
  const int nc1 = K * nc + 1;
  const int nf1 = 2 * K * nc + 1;
  const int64_t total = (int64_t)ex * ey * ez;
  const T* Pt = coef<T>() + LAY.Pt;
  const bool fast = total < kFastDivItems;
  for (int64_t t = t0; t < total; t += tstep) {
    int x, y, z;
    if (fast) {
      const uint32_t u = (uint32_t)t, rr = dex.div(u), zz = dey.div(rr);
      x = (int)(u - rr * dex.d);
      y = (int)(rr - zz * dey.d);
      z = (int)zz;
    } else {
      x = (int)(t % ex);
      const int64_t rr = t / ex;
      y = (int)(rr % ey);
      z = (int)(rr / ey);
    }
    const int gc = AX == 0 ? x : (AX == 1 ? y : z);
    if (gc == 0 || gc == nc1 - 1) { out[t] = T(0); continue; }
    const int ix = AX == 0 ? nf1 : ex, iy = AX == 1 ? nf1 : ey;
    auto at = [&](int gf) -> T {
      const int64_t ii = AX == 0 ? (gf + (int64_t)ix * (y + (int64_t)iy * z))
                                 : (AX == 1 ? (x + (int64_t)ix * (gf + (int64_t)iy * z))
                                            : (x + (int64_t)ix * (y + (int64_t)iy * gf)));
      return in[ii];
    };
    const int cc = gc / K, bb = gc - K * cc;
    T acc = T(0);
    if (bb == 0) {
      // vertex node: fine nodes of coarse cells cc-1 (local index K) and cc (local 0)
      const int Cl = cc - 1;
#pragma unroll
      for (int tt = 0; tt <= 2 * K; ++tt) {
        const int ch = tt < K ? 0 : 1, a = tt - K * ch;
        acc += Pt[(ch * (K + 1) + a) * (K + 1) + K] * at(2 * K * Cl + tt);
      }
#pragma unroll
      for (int tt = 1; tt <= 2 * K; ++tt) {
        const int ch = tt < K ? 0 : 1, a = tt - K * ch;
        acc += Pt[(ch * (K + 1) + a) * (K + 1) + 0] * at(2 * K * cc + tt);
      }
    } else {
#pragma unroll
      for (int tt = 0; tt <= 2 * K; ++tt) {
        const int ch = tt < K ? 0 : 1, a = tt - K * ch;
        acc += Pt[(ch * (K + 1) + a) * (K + 1) + bb] * at(2 * K * cc + tt);
      }
    }
    out[t] = acc;
  }
}

template <int AX, bool ADD, typename T>
__global__ void hprolong_pass(const T* __restrict__ in, T* __restrict__ out, int nc, int ex, int ey, int ez,
                              FastDiv dex, FastDiv dey) {
  hprolong_body<AX, ADD, T>(in, out, nc, ex, ey, ez, dex, dey,
                            (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                            (int64_t)gridDim.x * blockDim.x);
}

template <int AX, typename T>
__global__ void hrestrict_pass(const T* __restrict__ in, T* __restrict__ out, int nc, int ex, int ey, int ez,
                               FastDiv dex, FastDiv dey) {
  hrestrict_body<AX, T>(in, out, nc, ex, ey, ez, dex, dey,
                        (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                        (int64_t)gridDim.x * blockDim.x);
}

// one pass of a transfer over every job (extents of the job's output array)
template <typename T>
struct TransferJob {
  const T* in;
  T* out;
  int nc, ex, ey, ez;
  FastDiv dex, dey;
};

template <int AX, bool ADD, typename T>
__global__ void hprolong_group(const __grid_constant__ GroupOf<TransferJob<T>> G) {
  const int64_t total = G.start[G.count];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = group_find(G, t);
    const TransferJob<T>& a = G.job[j];
    hprolong_body<AX, ADD, T>(a.in, a.out, a.nc, a.ex, a.ey, a.ez, a.dex, a.dey, t - G.start[j], kOneItem);
  }
}

template <int AX, typename T>
__global__ void hrestrict_group(const __grid_constant__ GroupOf<TransferJob<T>> G) {
  const int64_t total = G.start[G.count];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = group_find(G, t);
    const TransferJob<T>& a = G.job[j];
    hrestrict_body<AX, T>(a.in, a.out, a.nc, a.ex, a.ey, a.ez, a.dex, a.dey, t - G.start[j], kOneItem);
  }
}

template <typename T>
static PatchParams<T> to_params(const PatchParamsHost& H) {
  PatchParams<T> P;
  P.scale = (T)H.scale;
  P.omega_as = (T)H.omega_as;
  for (int i = 0; i < 4; ++i) P.omega[i] = (T)H.omega[i];
  P.inv_a0 = (T)H.inv_a0;
  P.inv_scale = (T)(1.0 / H.scale);
  P.half = H.half;
  P.colour = H.colour;
  return P;
}

}  // namespace PMG_KNS
}  // namespace pmg
