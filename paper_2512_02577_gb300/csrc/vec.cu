// Degree-independent kernels: FP64 CG vector algebra with device-resident
// scalars (deterministic two-pass reductions: fixed grid, fixed summation
// order), precision casts, the dense coarse-level solve, and the set-up
// kernels for the deformed geometry (quadrature-point tensors G_q, operator
// diagonals), the manufactured right-hand side and the L2 error.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "vec.h"

namespace pmg {

std::atomic<int64_t> g_launches{0};

static inline int grid_for(int64_t work, int block, int cap = 152 * 8) {
  int64_t g = (work + block - 1) / block;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

// ------------------------------------------------------------ reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of v into out (thread 0 writes). blockDim.x == 256.
__device__ __forceinline__ void block_store_sum(double v, double* out) {
  __shared__ double ws[8];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < 8 ? ws[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) *out = t;
  }
}

// partial[b] = sum over this block's grid-stride slice of x*y
__global__ void __launch_bounds__(256) dot_partial_kernel(const double* __restrict__ x, const double* __restrict__ y,
                                                          int64_t n, double* __restrict__ partial) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += x[i] * y[i];
  block_store_sum(s, partial + blockIdx.x);
}

// out = sum of nb partials, in a fixed order (one block)
__global__ void __launch_bounds__(256) sum_partials_kernel(const double* __restrict__ partial, int nb,
                                                           double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
  block_store_sum(s, out);
}

cudaError_t dot(const double* x, const double* y, int64_t n, double* partial, double* out, cudaStream_t st) {
  dot_partial_kernel<<<kDotBlocks, 256, 0, st>>>(x, y, n, partial);
  sum_partials_kernel<<<1, 256, 0, st>>>(partial, kDotBlocks, out);
  g_launches += 2;
  return cudaGetLastError();
}

// x += alpha p, r -= alpha Ap with alpha = s[num] / s[den]; partial sums of
// r.r for the updated r.
__global__ void __launch_bounds__(256) cg_xr_kernel(double* __restrict__ x, double* __restrict__ r,
                                                    const double* __restrict__ p, const double* __restrict__ Ap,
                                                    int64_t n, const double* __restrict__ s, int num, int den,
                                                    double* __restrict__ partial) {
  const double alpha = s[num] / s[den];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * Ap[i];
    r[i] = ri;
    acc += ri * ri;
  }
  block_store_sum(acc, partial + blockIdx.x);
}

cudaError_t cg_update_xr(double* x, double* r, const double* p, const double* Ap, int64_t n, const double* s,
                         int num, int den, double* partial, double* rr_out, cudaStream_t st) {
  cg_xr_kernel<<<kDotBlocks, 256, 0, st>>>(x, r, p, Ap, n, s, num, den, partial);
  sum_partials_kernel<<<1, 256, 0, st>>>(partial, kDotBlocks, rr_out);
  g_launches += 2;
  return cudaGetLastError();
}

// p = z + beta p with beta = s[num] / s[den] (beta = 0 if first); then s[den] = s[num]
__global__ void __launch_bounds__(256) cg_p_kernel(double* __restrict__ p, const double* __restrict__ z, int64_t n,
                                                   const double* __restrict__ s, int num, int den, int first) {
  const double beta = first ? 0.0 : s[num] / s[den];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

__global__ void copy_scalar_kernel(double* s, int dst, int src) { s[dst] = s[src]; }

cudaError_t cg_update_p(double* p, const double* z, int64_t n, double* s, int num, int den, int first,
                        cudaStream_t st) {
  cg_p_kernel<<<grid_for(n, 256), 256, 0, st>>>(p, z, n, s, num, den, first);
  copy_scalar_kernel<<<1, 1, 0, st>>>(s, den, num);
  g_launches += 2;
  return cudaGetLastError();
}

// Flexible (Polak-Ribiere) variant: s[num] = r.z_new - r_old.z_new computed
// by the caller; identical structure.

// ------------------------------------------------------------ GMRES
// Flexible right-preconditioned GMRES (the outer solver of the half local
// V-cycle, §3.2.2).  The Krylov basis v_0..v_m and the preconditioned
// vectors z_0..z_{m-1} are FP64 columns of length n with stride ld; the
// Hessenberg matrix H is column-major with leading dimension m + 1.  The
// small state lives in one device array (GmresState offsets) so the host
// reads one number per step: the residual estimate |g_{j+1}|.

// partial[i * kDotBlocks + b] = block b's slice of v_i . w, i = blockIdx.y
__global__ void __launch_bounds__(256) multi_dot_partial_kernel(const double* __restrict__ V, int64_t ld,
                                                                const double* __restrict__ w, int64_t n,
                                                                double* __restrict__ partial) {
  const double* v = V + (int64_t)blockIdx.y * ld;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += v[i] * w[i];
  block_store_sum(s, partial + (int64_t)blockIdx.y * gridDim.x + blockIdx.x);
}

// out[i] = sum of the kDotBlocks partials of vector i, fixed order (block i)
__global__ void __launch_bounds__(256) multi_sum_kernel(const double* __restrict__ partial, int nb,
                                                        double* __restrict__ out) {
  const double* p = partial + (int64_t)blockIdx.x * nb;
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += p[i];
  block_store_sum(s, out + blockIdx.x);
}

cudaError_t multi_dot(const double* V, int64_t ld, int nv, const double* w, int64_t n, double* partial,
                      double* out, cudaStream_t st) {
  if (nv < 1 || nv > kMaxKrylov + 1) return cudaErrorInvalidValue;
  multi_dot_partial_kernel<<<dim3(kDotBlocks, nv), 256, 0, st>>>(V, ld, w, n, partial);
  multi_sum_kernel<<<nv, 256, 0, st>>>(partial, kDotBlocks, out);
  g_launches += 2;
  return cudaGetLastError();
}

// w += sgn sum_{i < nv} c_i v_i (coefficients staged in shared memory)
__global__ void __launch_bounds__(256) multi_axpy_kernel(double* __restrict__ w, const double* __restrict__ V,
                                                         int64_t ld, int nv, const double* __restrict__ c,
                                                         double sgn, int64_t n) {
  __shared__ double cs[kMaxKrylov + 1];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) cs[i] = sgn * c[i];
  __syncthreads();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double acc = w[k];
    for (int i = 0; i < nv; ++i) acc += cs[i] * V[i * ld + k];
    w[k] = acc;
  }
}

cudaError_t multi_axpy(double* w, const double* V, int64_t ld, int nv, const double* c, double sgn, int64_t n,
                       cudaStream_t st) {
  if (nv < 1 || nv > kMaxKrylov + 1) return cudaErrorInvalidValue;
  multi_axpy_kernel<<<grid_for(n, 256), 256, 0, st>>>(w, V, ld, nv, c, sgn, n);
  g_launches += 1;
  return cudaGetLastError();
}

// Start of a cycle: beta = sqrt(nrm2[0]); g = beta e_1; S[INV] = 1 / beta (0 if beta = 0)
__global__ void gmres_start_kernel(double* __restrict__ S, const double* __restrict__ nrm2, int m) {
  const double beta = sqrt(fmax(nrm2[0], 0.0));
  double* g = S + GmresState::g(m);
  g[0] = beta;
  for (int i = 1; i <= m; ++i) g[i] = 0.0;
  S[GmresState::inv(m)] = beta > 0.0 ? 1.0 / beta : 0.0;
}

// Step j: H(:, j) += h2 (second Gram-Schmidt pass), H(j+1, j) = ||w||, the
// earlier rotations on the column, a new rotation zeroing H(j+1, j), and
// g updated; S[EST] = |g_{j+1}|, S[INV] = 1 / ||w|| (0 on breakdown).
__global__ void gmres_givens_kernel(double* __restrict__ H, double* __restrict__ S, const double* __restrict__ nrm2,
                                    int j, int m) {
  double* h = H + (int64_t)j * (m + 1);
  const double* h2 = S + GmresState::h2(m);
  double* cs = S + GmresState::cs(m);
  double* sn = S + GmresState::sn(m);
  double* g = S + GmresState::g(m);
  for (int i = 0; i <= j; ++i) h[i] += h2[i];
  const double hn = sqrt(fmax(nrm2[0], 0.0));
  h[j + 1] = hn;
  S[GmresState::inv(m)] = hn > 0.0 ? 1.0 / hn : 0.0;
  for (int i = 0; i < j; ++i) {
    const double a = h[i], b = h[i + 1];
    h[i] = cs[i] * a + sn[i] * b;
    h[i + 1] = -sn[i] * a + cs[i] * b;
  }
  const double rho = hypot(h[j], h[j + 1]);
  const double c = rho > 0.0 ? h[j] / rho : 1.0, s = rho > 0.0 ? h[j + 1] / rho : 0.0;
  cs[j] = c;
  sn[j] = s;
  h[j] = rho;
  h[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  S[GmresState::est(m)] = fabs(g[j + 1]);
}

// dst = src * S[INV]
__global__ void __launch_bounds__(256) scale_by_kernel(double* __restrict__ dst, const double* __restrict__ src,
                                                       const double* __restrict__ f, int64_t n) {
  const double a = *f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = a * src[i];
}

// y = R^{-1} g(0:k) with R the leading k x k upper triangle of the rotated H
__global__ void gmres_backsolve_kernel(const double* __restrict__ H, double* __restrict__ S, int k, int m) {
  const double* g = S + GmresState::g(m);
  double* y = S + GmresState::y(m);
  for (int i = k - 1; i >= 0; --i) {
    double t = g[i];
    for (int c = i + 1; c < k; ++c) t -= H[(int64_t)c * (m + 1) + i] * y[c];
    const double d = H[(int64_t)i * (m + 1) + i];
    y[i] = d != 0.0 ? t / d : 0.0;
  }
}

cudaError_t gmres_start(double* S, const double* nrm2, int m, const double* r, double* v0, int64_t n,
                        cudaStream_t st) {
  gmres_start_kernel<<<1, 1, 0, st>>>(S, nrm2, m);
  scale_by_kernel<<<grid_for(n, 256), 256, 0, st>>>(v0, r, S + GmresState::inv(m), n);
  g_launches += 2;
  return cudaGetLastError();
}

cudaError_t gmres_givens(double* H, double* S, const double* nrm2, int j, int m, double* v, int64_t n,
                         cudaStream_t st) {
  gmres_givens_kernel<<<1, 1, 0, st>>>(H, S, nrm2, j, m);
  scale_by_kernel<<<grid_for(n, 256), 256, 0, st>>>(v, v, S + GmresState::inv(m), n);
  g_launches += 2;
  return cudaGetLastError();
}

cudaError_t gmres_update(const double* H, double* S, int k, int m, const double* Z, int64_t ld, double* x, int64_t n,
                         cudaStream_t st) {
  if (k < 1) return cudaSuccess;
  gmres_backsolve_kernel<<<1, 1, 0, st>>>(H, S, k, m);
  g_launches += 1;
  return multi_axpy(x, Z, ld, k, S + GmresState::y(m), 1.0, n, st);
}

// ------------------------------------------------------------ casts
__global__ void d2f_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void f2d_kernel(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

cudaError_t cast_d2f(const double* a, float* b, int64_t n, cudaStream_t st) {
  d2f_kernel<<<grid_for(n, 256), 256, 0, st>>>(a, b, n);
  g_launches += 1;
  return cudaGetLastError();
}
cudaError_t cast_f2d(const float* a, double* b, int64_t n, cudaStream_t st) {
  f2d_kernel<<<grid_for(n, 256), 256, 0, st>>>(a, b, n);
  g_launches += 1;
  return cudaGetLastError();
}

// ------------------------------------------------------------ coarse solve
// u[idx[i]] = sum_j Ainv[i][j] b[idx[j]]; one warp per row; boundary of u
// must be zero (caller clears u).
template <typename T>
__global__ void coarse_kernel(const T* __restrict__ Ainv, const int* __restrict__ idx, int nc, const T* __restrict__ b,
                              T* __restrict__ u) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= nc) return;
  T s = T(0);
  for (int j = lane; j < nc; j += 32) s += Ainv[(int64_t)warp * nc + j] * b[idx[j]];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) u[idx[warp]] = s;
}

cudaError_t coarse_solve(int prec, const void* Ainv, const int* idx, int nc, const void* b, void* u, int64_t N,
                         cudaStream_t st) {
  const size_t es = prec == 0 ? 8 : 4;
  cudaError_t e = cudaMemsetAsync(u, 0, es * (size_t)N, st);
  if (e != cudaSuccess) return e;
  if (nc == 0) return cudaSuccess;
  const int blocks = (nc * 32 + 255) / 256;
  if (prec == 0) coarse_kernel<double><<<blocks, 256, 0, st>>>((const double*)Ainv, idx, nc, (const double*)b, (double*)u);
  else coarse_kernel<float><<<blocks, 256, 0, st>>>((const float*)Ainv, idx, nc, (const float*)b, (float*)u);
  g_launches += 1;
  return cudaGetLastError();
}

// ------------------------------------------------------------ grouped forms
// Each reduction keeps its per-job grid (kDotBlocks blocks along x, the job
// along y) and its per-job partial sums, so a job's result is bitwise that of
// its own launch; element-wise kernels spread the concatenated elements of
// the jobs over the grid (GroupOf::start).
static bool group_ok(int count) { return count >= 1 && count <= kMaxGroup; }

// A warp forms the partial of one of the job's kDotBlocks reduction blocks
// (vb): lane l sums the elements of each of the block's 256 threads wl * 32 +
// l (wl = 0..7) exactly as that thread of dot_partial_kernel does, each of
// the eight warp sums is formed by the same shuffle tree, and the eight are
// combined as block_store_sum combines its warps -- the same partial, bitwise,
// without shared memory or block barriers (kDotBlocks / 8 blocks per job).
constexpr int kGroupDotBlocks = kDotBlocks / 8;
static_assert(kDotBlocks % 8 == 0, "a block of the grouped reductions covers 8 reduction blocks");

__device__ __forceinline__ double combine_warp_sums(const double (&s)[8]) {
  // s[wl]: this lane's share of warp wl's sum; lane 0 of warp_sum holds each total
  double t = 0.0;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int wl = 0; wl < 8; ++wl) {
    const double v = __shfl_sync(0xffffffffu, warp_sum(s[wl]), 0);
    if (lane == wl) t = v;
  }
  return warp_sum(t);  // lanes >= 8 hold 0, as in block_store_sum
}

__global__ void __launch_bounds__(256) dot_partial_group(const __grid_constant__ GroupOf<DotJob> G) {
  const DotJob& a = G.job[blockIdx.y];
  const int vb = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  double s[8];
#pragma unroll
  for (int wl = 0; wl < 8; ++wl) s[wl] = 0.0;
  // the eight threads' k-th elements together (independent loads), each
  // thread's elements in its own order
  for (int64_t base = (int64_t)vb * 256 + lane; base < a.n; base += (int64_t)kDotBlocks * 256) {
#pragma unroll
    for (int wl = 0; wl < 8; ++wl) {
      const int64_t i = base + wl * 32;
      if (i < a.n) s[wl] += a.x[i] * a.y[i];
    }
  }
  const double t = combine_warp_sums(s);
  if (lane == 0) a.partial[vb] = t;
}

__global__ void __launch_bounds__(256) sum_partials_group(const __grid_constant__ GroupOf<DotJob> G) {
  const DotJob& a = G.job[blockIdx.x];
  double s = 0.0;
  for (int i = threadIdx.x; i < kDotBlocks; i += blockDim.x) s += a.partial[i];
  block_store_sum(s, a.out);
}

cudaError_t dot_group(int count, const DotJob* jobs, cudaStream_t st) {
  if (!group_ok(count)) return cudaErrorInvalidValue;
  GroupOf<DotJob> G;
  G.count = count;
  for (int j = 0; j < count; ++j) G.job[j] = jobs[j];
  dot_partial_group<<<dim3(kGroupDotBlocks, count), 256, 0, st>>>(G);
  sum_partials_group<<<count, 256, 0, st>>>(G);
  g_launches += 2;
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) cg_xr_group(const __grid_constant__ GroupOf<CgXrJob> G) {
  const CgXrJob& a = G.job[blockIdx.y];
  const double alpha = a.s[a.num] / a.s[a.den];
  const int vb = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  double s[8];  // as dot_partial_group, for cg_xr_kernel's updates and sums
#pragma unroll
  for (int wl = 0; wl < 8; ++wl) s[wl] = 0.0;
  for (int64_t base = (int64_t)vb * 256 + lane; base < a.n; base += (int64_t)kDotBlocks * 256) {
#pragma unroll
    for (int wl = 0; wl < 8; ++wl) {
      const int64_t i = base + wl * 32;
      if (i < a.n) {
        a.x[i] += alpha * a.p[i];
        const double ri = a.r[i] - alpha * a.Ap[i];
        a.r[i] = ri;
        s[wl] += ri * ri;
      }
    }
  }
  const double t = combine_warp_sums(s);
  if (lane == 0) a.partial[vb] = t;
}

__global__ void __launch_bounds__(256) cg_xr_sum_group(const __grid_constant__ GroupOf<CgXrJob> G) {
  const CgXrJob& a = G.job[blockIdx.x];
  double s = 0.0;
  for (int i = threadIdx.x; i < kDotBlocks; i += blockDim.x) s += a.partial[i];
  block_store_sum(s, a.rr_out);
}

cudaError_t cg_update_xr_group(int count, const CgXrJob* jobs, cudaStream_t st) {
  if (!group_ok(count)) return cudaErrorInvalidValue;
  GroupOf<CgXrJob> G;
  G.count = count;
  for (int j = 0; j < count; ++j) G.job[j] = jobs[j];
  cg_xr_group<<<dim3(kGroupDotBlocks, count), 256, 0, st>>>(G);
  cg_xr_sum_group<<<count, 256, 0, st>>>(G);
  g_launches += 2;
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) cg_p_group(const __grid_constant__ GroupOf<CgPJob> G) {
  const int64_t total = G.start[G.count];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = group_find(G, t);
    const CgPJob& a = G.job[j];
    const int64_t i = t - G.start[j];
    const double beta = a.first ? 0.0 : a.s[a.num] / a.s[a.den];
    a.p[i] = a.z[i] + beta * a.p[i];
  }
}

__global__ void copy_scalar_group(const __grid_constant__ GroupOf<CgPJob> G) {
  const int j = threadIdx.x;
  if (j < G.count) G.job[j].s[G.job[j].den] = G.job[j].s[G.job[j].num];
}

cudaError_t cg_update_p_group(int count, const CgPJob* jobs, cudaStream_t st) {
  if (!group_ok(count)) return cudaErrorInvalidValue;
  GroupOf<CgPJob> G;
  G.count = count;
  G.start[0] = 0;
  int64_t work = 0;
  for (int j = 0; j < count; ++j) {
    G.job[j] = jobs[j];
    work += jobs[j].n;
    G.start[j + 1] = work;
  }
  cg_p_group<<<grid_for(work, 256), 256, 0, st>>>(G);
  copy_scalar_group<<<1, 32, 0, st>>>(G);
  g_launches += 2;
  return cudaGetLastError();
}

template <typename A, typename B>
__global__ void __launch_bounds__(256) convert_group(const __grid_constant__ GroupOf<CopyJob> G) {
  const int64_t total = G.start[G.count];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = group_find(G, t);
    const int64_t i = t - G.start[j];
    static_cast<B*>(G.job[j].b)[i] = (B) static_cast<const A*>(G.job[j].a)[i];
  }
}

template <typename A, typename B>
static cudaError_t convert_group_launch(int count, const CopyJob* jobs, cudaStream_t st) {
  if (!group_ok(count)) return cudaErrorInvalidValue;
  GroupOf<CopyJob> G;
  G.count = count;
  G.start[0] = 0;
  int64_t work = 0;
  for (int j = 0; j < count; ++j) {
    G.job[j] = jobs[j];
    work += jobs[j].n;
    G.start[j + 1] = work;
  }
  convert_group<A, B><<<grid_for(work, 256), 256, 0, st>>>(G);
  g_launches += 1;
  return cudaGetLastError();
}

cudaError_t cast_d2f_group(int count, const CopyJob* jobs, cudaStream_t st) {
  return convert_group_launch<double, float>(count, jobs, st);
}
cudaError_t cast_f2d_group(int count, const CopyJob* jobs, cudaStream_t st) {
  return convert_group_launch<float, double>(count, jobs, st);
}
cudaError_t copy_group(int count, const CopyJob* jobs, int elem_bytes, cudaStream_t st) {
  if (elem_bytes == 8) return convert_group_launch<double, double>(count, jobs, st);
  if (elem_bytes == 4) return convert_group_launch<float, float>(count, jobs, st);
  return cudaErrorInvalidValue;
}

__global__ void __launch_bounds__(256) zero_group_kernel(const __grid_constant__ GroupOf<ZeroJob> G) {
  const int64_t total = G.start[G.count];  // 4-byte words
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int j = group_find(G, t);
    static_cast<unsigned*>(G.job[j].p)[t - G.start[j]] = 0u;
  }
}

cudaError_t zero_group(int count, const ZeroJob* jobs, cudaStream_t st) {
  if (!group_ok(count)) return cudaErrorInvalidValue;
  GroupOf<ZeroJob> G;
  G.count = count;
  G.start[0] = 0;
  int64_t work = 0;
  for (int j = 0; j < count; ++j) {
    if (jobs[j].bytes % 4) return cudaErrorInvalidValue;
    G.job[j] = jobs[j];
    work += jobs[j].bytes / 4;
    G.start[j + 1] = work;
  }
  zero_group_kernel<<<grid_for(work, 256), 256, 0, st>>>(G);
  g_launches += 1;
  return cudaGetLastError();
}

// rows of every job's coarse solve (concatenated, G.start), one warp per
// row as coarse_kernel
template <typename T>
__global__ void coarse_group_kernel(const __grid_constant__ GroupOf<CoarseJob> G) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t rows = G.start[G.count];
  for (int64_t wg = w0; wg < rows; wg += nw) {  // uniform per warp
    const int j = group_find(G, wg);
    const CoarseJob& a = G.job[j];
    const int w = (int)(wg - G.start[j]);
    const T* Ainv = static_cast<const T*>(a.Ainv);
    const T* b = static_cast<const T*>(a.b);
    T s = T(0);
    for (int jj = lane; jj < a.nc; jj += 32) s += Ainv[(int64_t)w * a.nc + jj] * b[a.idx[jj]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) static_cast<T*>(a.u)[a.idx[w]] = s;
  }
}

cudaError_t coarse_solve_group(int prec, int count, const CoarseJob* jobs, cudaStream_t st) {
  if (!group_ok(count)) return cudaErrorInvalidValue;
  const int es = prec == 0 ? 8 : 4;
  ZeroJob Z[kMaxGroup];
  GroupOf<CoarseJob> G;
  G.count = 0;
  G.start[0] = 0;
  int64_t rows = 0;
  for (int j = 0; j < count; ++j) {
    Z[j] = ZeroJob{jobs[j].u, (int64_t)es * jobs[j].N};
    if (jobs[j].nc > 0) {
      G.job[G.count++] = jobs[j];
      rows += jobs[j].nc;
      G.start[G.count] = rows;
    }
  }
  cudaError_t e = zero_group(count, Z, st);
  if (e != cudaSuccess || G.count == 0) return e;
  const int blocks = (int)std::min<int64_t>((rows * 32 + 255) / 256, 152 * 16);
  if (prec == 0) coarse_group_kernel<double><<<blocks, 256, 0, st>>>(G);
  else coarse_group_kernel<float><<<blocks, 256, 0, st>>>(G);
  g_launches += 1;
  return cudaGetLastError();
}

// ------------------------------------------------------------ coarse set-up
// Dense coarse matrix A_0 on the free DoFs: row j = (A_0 e_j) restricted to
// the free nodes (A_0 is symmetric), then an in-place Gauss-Jordan inverse.
__global__ void unit_vector_kernel(double* __restrict__ x, int64_t N, int64_t pos) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = i == pos ? 1.0 : 0.0;
}
__global__ void gather_row_kernel(const double* __restrict__ y, const int* __restrict__ idx, int nc,
                                  double* __restrict__ A, int row) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
    A[(int64_t)row * nc + i] = y[idx[i]];
}
__global__ void symmetrize_kernel(double* A, int nc) {
  const int64_t n2 = (int64_t)nc * nc;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n2; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / nc), j = (int)(t % nc);
    if (j < i) {
      const double s = 0.5 * (A[(int64_t)i * nc + j] + A[(int64_t)j * nc + i]);
      A[(int64_t)i * nc + j] = s;
      A[(int64_t)j * nc + i] = s;
    }
  }
}
__global__ void gj_pivot_kernel(const double* __restrict__ A, int nc, int p, double* __restrict__ row,
                                double* __restrict__ col) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    row[i] = A[(int64_t)p * nc + i];
    col[i] = A[(int64_t)i * nc + p];
  }
}
// sweep of pivot p: a_ij -= c_i r_j / a_pp; a_pj = r_j / a_pp; a_ip = -c_i / a_pp; a_pp = 1 / a_pp
__global__ void gj_update_kernel(double* __restrict__ A, int nc, int p, const double* __restrict__ row,
                                 const double* __restrict__ col, int* __restrict__ bad) {
  const double piv = row[p];
  if (!(piv > 0.0)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *bad = 1;
    return;
  }
  const double ip = 1.0 / piv;
  const int64_t n2 = (int64_t)nc * nc;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n2; t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / nc), j = (int)(t % nc);
    double v;
    if (i == p && j == p) v = ip;
    else if (i == p) v = row[j] * ip;
    else if (j == p) v = -col[i] * ip;
    else v = A[t] - col[i] * row[j] * ip;
    A[t] = v;
  }
}
__global__ void store_inverse_kernel(const double* __restrict__ A, int64_t n2, void* out, int prec) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n2; t += (int64_t)gridDim.x * blockDim.x) {
    if (prec == 0) ((double*)out)[t] = A[t];
    else ((float*)out)[t] = (float)A[t];
  }
}

cudaError_t coarse_unit(double* x, int64_t N, int64_t pos, cudaStream_t st) {
  unit_vector_kernel<<<grid_for(N, 256), 256, 0, st>>>(x, N, pos);
  g_launches += 1;
  return cudaGetLastError();
}
cudaError_t coarse_gather_row(const double* y, const int* idx, int nc, double* A, int row, cudaStream_t st) {
  gather_row_kernel<<<grid_for(nc, 256), 256, 0, st>>>(y, idx, nc, A, row);
  g_launches += 1;
  return cudaGetLastError();
}
cudaError_t coarse_invert(double* A, int nc, double* row, double* col, int* bad, void* out, int prec,
                          cudaStream_t st) {
  const int64_t n2 = (int64_t)nc * nc;
  symmetrize_kernel<<<grid_for(n2, 256), 256, 0, st>>>(A, nc);
  for (int p = 0; p < nc; ++p) {
    gj_pivot_kernel<<<grid_for(nc, 256), 256, 0, st>>>(A, nc, p, row, col);
    gj_update_kernel<<<grid_for(n2, 256), 256, 0, st>>>(A, nc, p, row, col, bad);
  }
  store_inverse_kernel<<<grid_for(n2, 256), 256, 0, st>>>(A, n2, out, prec);
  g_launches += 2 + 2 * (int64_t)nc;
  return cudaGetLastError();
}

// ------------------------------------------------------------ geometry
// Deformation F(X) = X + a prod_m sin(2 pi X_m) (1, ..., 1) and
// dF_i/dX_j = delta_ij + a 2 pi cos(2 pi X_j) prod_{m != j} sin(2 pi X_m).
__device__ void map_point(int dim, double a, const double* X, double* x, double J[3][3]) {
  const double tp = 6.283185307179586476925286766559;
  double s[3], c[3];
  for (int m = 0; m < dim; ++m) {
    sincos(tp * X[m], &s[m], &c[m]);
  }
  double prod = 1.0;
  for (int m = 0; m < dim; ++m) prod *= s[m];
  for (int i = 0; i < dim; ++i) x[i] = X[i] + a * prod;
  for (int j = 0; j < dim; ++j) {
    double o = 1.0;
    for (int m = 0; m < dim; ++m)
      if (m != j) o *= s[m];
    const double dj = a * tp * c[j] * o;
    for (int i = 0; i < dim; ++i) J[i][j] = (i == j ? 1.0 : 0.0) + dj;
  }
}

// Trilinear (bilinear in 2D) cell c of a level with n cells per side, corners
// at the displaced vertices: with xi = n X - c, x = sum over corners s of
// prod_m N_{s_m}(xi_m) P_{c+s} (N_0 = 1 - t, N_1 = t), dx/dX = n dx/dxi.
__device__ void map_trilinear(int dim, const GeomDesc& g, int n, const int* c, const double* X, double* x,
                              double J[3][3]) {
  const int stride = g.n_fine / n, nv = g.n_fine + 1;
  double xi[3];
  for (int m = 0; m < dim; ++m) {
    xi[m] = n * X[m] - c[m];
    x[m] = 0.0;
    for (int j = 0; j < dim; ++j) J[m][j] = 0.0;
  }
  for (int s = 0; s < (1 << dim); ++s) {
    int64_t flat = 0, mul = 1;
    double N[3], dN[3];
    for (int m = 0; m < dim; ++m) {
      const int bit = (s >> m) & 1;
      flat += mul * (int64_t)((c[m] + bit) * stride);
      mul *= nv;
      N[m] = bit ? xi[m] : 1.0 - xi[m];
      dN[m] = bit ? 1.0 : -1.0;
    }
    const double* P = g.verts + flat * dim;
    double w = 1.0;
    for (int m = 0; m < dim; ++m) w *= N[m];
    for (int i = 0; i < dim; ++i) x[i] += w * P[i];
    for (int j = 0; j < dim; ++j) {
      double gj = n * dN[j];
      for (int m = 0; m < dim; ++m)
        if (m != j) gj *= N[m];
      for (int i = 0; i < dim; ++i) J[i][j] += gj * P[i];
    }
  }
}

// x = F(X) and J = dF/dX for the level's geometry (cell c holds X)
__device__ void map_geo(int dim, const GeomDesc& g, int n, const int* c, const double* X, double* x,
                        double J[3][3]) {
  if (g.kind == 2) {
    map_trilinear(dim, g, n, c, X, x, J);
  } else if (g.kind == 1) {
    map_point(dim, g.amp, X, x, J);
  } else {
    for (int i = 0; i < dim; ++i) {
      x[i] = X[i];
      for (int j = 0; j < dim; ++j) J[i][j] = i == j ? 1.0 : 0.0;
    }
  }
}

// G[cell][comp][q] = w_q det J J^{-1} J^{-T} with J = dF/dX h, stored in TG
// (float: rounded to nearest; double: as computed).
template <typename TG>
__global__ void geometry_kernel(int dim, int n, int p, GeomDesc geo, QuadTab tab, TG* __restrict__ G,
                                int* __restrict__ bad) {
  const int nq = p + 1;
  const int NP = dim == 3 ? nq * nq * nq : nq * nq;
  const int nc = dim == 3 ? 6 : 3;
  const int64_t ncell = dim == 3 ? (int64_t)n * n * n : (int64_t)n * n;
  const double h = 1.0 / n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ncell * NP;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(t % NP);
    const int64_t cell = t / NP;
    const int cidx[3] = {(int)(cell % n), (int)((cell / n) % n), dim == 3 ? (int)(cell / ((int64_t)n * n)) : 0};
    const int qi[3] = {q % nq, (q / nq) % nq, dim == 3 ? q / (nq * nq) : 0};
    double X[3], x[3], J[3][3];
    double w = 1.0;
    for (int m = 0; m < dim; ++m) {
      X[m] = h * (cidx[m] + tab.x[qi[m]]);
      w *= tab.w[qi[m]];
    }
    map_geo(dim, geo, n, cidx, X, x, J);
    for (int i = 0; i < dim; ++i)
      for (int j = 0; j < dim; ++j) J[i][j] *= h;
    double Gq[3][3];
    if (dim == 3) {
      const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
      const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
      const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
      const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
      if (!(det > 0.0)) atomicOr(bad, 1);
      double inv[3][3];
      inv[0][0] = c00 / det;
      inv[1][0] = c01 / det;
      inv[2][0] = c02 / det;
      inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
      inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
      inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
      inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
      inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
      inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
          double s = 0.0;
          for (int j = 0; j < 3; ++j) s += inv[i][j] * inv[k][j];
          Gq[i][k] = w * det * s;
        }
    } else {
      const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      if (!(det > 0.0)) atomicOr(bad, 1);
      double inv[2][2];
      inv[0][0] = J[1][1] / det;
      inv[0][1] = -J[0][1] / det;
      inv[1][0] = -J[1][0] / det;
      inv[1][1] = J[0][0] / det;
      for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 2; ++k) Gq[i][k] = w * det * (inv[i][0] * inv[k][0] + inv[i][1] * inv[k][1]);
    }
    TG* Gc = G + cell * nc * NP;
    if (dim == 3) {
      Gc[0 * NP + q] = (TG)Gq[0][0];
      Gc[1 * NP + q] = (TG)Gq[0][1];
      Gc[2 * NP + q] = (TG)Gq[0][2];
      Gc[3 * NP + q] = (TG)Gq[1][1];
      Gc[4 * NP + q] = (TG)Gq[1][2];
      Gc[5 * NP + q] = (TG)Gq[2][2];
    } else {
      Gc[0 * NP + q] = (TG)Gq[0][0];
      Gc[1 * NP + q] = (TG)Gq[0][1];
      Gc[2 * NP + q] = (TG)Gq[1][1];
    }
  }
}

cudaError_t compute_geometry(int dim, int n, int p, const GeomDesc& geo, const QuadTab& tab, void* G, int gprec,
                             int* bad, cudaStream_t st) {
  const int nq = p + 1;
  const int64_t work = (dim == 3 ? (int64_t)n * n * n * nq * nq * nq : (int64_t)n * n * nq * nq);
  if (gprec == 0)
    geometry_kernel<double><<<grid_for(work, 256, 152 * 32), 256, 0, st>>>(dim, n, p, geo, tab, (double*)G, bad);
  else
    geometry_kernel<float><<<grid_for(work, 256, 152 * 32), 256, 0, st>>>(dim, n, p, geo, tab, (float*)G, bad);
  g_launches += 1;
  return cudaGetLastError();
}

// Diagonal of the degree-p operator, one parity colour of cells:
// diag[node] += sum_q grad phi_a^T G_q grad phi_a.
template <typename TG>
__global__ void diag_kernel(int dim, int n, int p, QuadTab tab, const TG* __restrict__ G, double* __restrict__ diag,
                            int colour) {
  const int n1 = p + 1;
  const int NP = dim == 3 ? n1 * n1 * n1 : n1 * n1;
  const int nc = dim == 3 ? 6 : 3;
  const int cx = (colour & 1) ? n / 2 : (n + 1) / 2, cy = ((colour >> 1) & 1) ? n / 2 : (n + 1) / 2;
  const int cz = dim == 3 ? (((colour >> 2) & 1) ? n / 2 : (n + 1) / 2) : 1;
  const int64_t ncell = (int64_t)cx * cy * cz;
  const int N1 = p * n + 1;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ncell * NP;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(t % NP);
    int64_t ci = t / NP;
    const int c0 = 2 * (int)(ci % cx) + (colour & 1);
    ci /= cx;
    const int c1 = 2 * (int)(ci % cy) + ((colour >> 1) & 1);
    ci /= cy;
    const int c2 = dim == 3 ? 2 * (int)ci + ((colour >> 2) & 1) : 0;
    const int64_t cell = c0 + (int64_t)n * (c1 + (int64_t)n * c2);
    const int ai[3] = {a % n1, (a / n1) % n1, dim == 3 ? a / (n1 * n1) : 0};
    const TG* Gc = G + cell * nc * NP;
    double s = 0.0;
    for (int q = 0; q < NP; ++q) {
      const int qi[3] = {q % n1, (q / n1) % n1, dim == 3 ? q / (n1 * n1) : 0};
      double gr[3];
      for (int d = 0; d < dim; ++d) {
        double v = 1.0;
        for (int e = 0; e < dim; ++e) v *= (d == e ? tab.D[qi[e] * 12 + ai[e]] : tab.V[qi[e] * 12 + ai[e]]);
        gr[d] = v;
      }
      if (dim == 3) {
        s += gr[0] * ((double)Gc[0 * NP + q] * gr[0] + (double)Gc[1 * NP + q] * gr[1] + (double)Gc[2 * NP + q] * gr[2]);
        s += gr[1] * ((double)Gc[1 * NP + q] * gr[0] + (double)Gc[3 * NP + q] * gr[1] + (double)Gc[4 * NP + q] * gr[2]);
        s += gr[2] * ((double)Gc[2 * NP + q] * gr[0] + (double)Gc[4 * NP + q] * gr[1] + (double)Gc[5 * NP + q] * gr[2]);
      } else {
        s += gr[0] * ((double)Gc[0 * NP + q] * gr[0] + (double)Gc[1 * NP + q] * gr[1]);
        s += gr[1] * ((double)Gc[1 * NP + q] * gr[0] + (double)Gc[2 * NP + q] * gr[1]);
      }
    }
    const int gx = p * c0 + ai[0], gy = p * c1 + ai[1], gz = p * c2 + ai[2];
    diag[gx + (int64_t)N1 * (gy + (int64_t)N1 * gz)] += s;
  }
}

// inv = 1/diag on free nodes, 0 on the boundary (precision of inv: prec)
__global__ void invert_kernel(const double* __restrict__ diag, void* inv, int prec, int dim, int N1) {
  const int64_t N = dim == 3 ? (int64_t)N1 * N1 * N1 : (int64_t)N1 * N1;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N; t += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(t % N1), y = (int)((t / N1) % N1), z = dim == 3 ? (int)(t / ((int64_t)N1 * N1)) : 1;
    const bool bnd = x == 0 || x == N1 - 1 || y == 0 || y == N1 - 1 || (dim == 3 && (z == 0 || z == N1 - 1));
    const double v = bnd ? 0.0 : 1.0 / diag[t];
    if (prec == 0) ((double*)inv)[t] = v;
    else ((float*)inv)[t] = (float)v;
  }
}

cudaError_t compute_inverse_diagonal(int dim, int n, int p, const QuadTab& tab, const void* G, int gprec,
                                     double* diag_tmp, void* inv, int prec, cudaStream_t st) {
  const int N1 = p * n + 1;
  const int64_t N = dim == 3 ? (int64_t)N1 * N1 * N1 : (int64_t)N1 * N1;
  cudaError_t e = cudaMemsetAsync(diag_tmp, 0, sizeof(double) * N, st);
  if (e != cudaSuccess) return e;
  const int NP = dim == 3 ? (p + 1) * (p + 1) * (p + 1) : (p + 1) * (p + 1);
  for (int colour = 0; colour < (1 << dim); ++colour) {
    const int64_t work = (dim == 3 ? (int64_t)n * n * n : (int64_t)n * n) / (1 << dim) * NP + NP * 8;
    if (gprec == 0)
      diag_kernel<double><<<grid_for(work, 128, 152 * 32), 128, 0, st>>>(dim, n, p, tab, (const double*)G, diag_tmp,
                                                                         colour);
    else
      diag_kernel<float><<<grid_for(work, 128, 152 * 32), 128, 0, st>>>(dim, n, p, tab, (const float*)G, diag_tmp,
                                                                        colour);
    g_launches += 1;
  }
  invert_kernel<<<grid_for(N, 256), 256, 0, st>>>(diag_tmp, inv, prec, dim, N1);
  g_launches += 1;
  return cudaGetLastError();
}

// ------------------------------------------------------------ RHS, L2 error
// b_a += sum_q f(F(X_q)) phi_a(xi_q) w_q det J_q  for one colour of cells
__global__ void rhs_kernel(int dim, int n, int K, GeomDesc geo, QuadTab tab, double* __restrict__ b, int colour) {
  const int n1 = K + 1;
  const int NP = dim == 3 ? n1 * n1 * n1 : n1 * n1;
  const int nq = tab.nq;
  const int NQ = dim == 3 ? nq * nq * nq : nq * nq;
  const int cx = (colour & 1) ? n / 2 : (n + 1) / 2, cy = ((colour >> 1) & 1) ? n / 2 : (n + 1) / 2;
  const int cz = dim == 3 ? (((colour >> 2) & 1) ? n / 2 : (n + 1) / 2) : 1;
  const int64_t ncell = (int64_t)cx * cy * cz;
  const int N1 = K * n + 1;
  const double h = 1.0 / n;
  const double pi = 3.141592653589793238462643383279502884;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ncell * NP;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(t % NP);
    int64_t ci = t / NP;
    const int c[3] = {0, 0, 0};
    int cc[3];
    cc[0] = 2 * (int)(ci % cx) + (colour & 1);
    ci /= cx;
    cc[1] = 2 * (int)(ci % cy) + ((colour >> 1) & 1);
    ci /= cy;
    cc[2] = dim == 3 ? 2 * (int)ci + ((colour >> 2) & 1) : 0;
    (void)c;
    const int ai[3] = {a % n1, (a / n1) % n1, dim == 3 ? a / (n1 * n1) : 0};
    double s = 0.0;
    for (int q = 0; q < NQ; ++q) {
      const int qi[3] = {q % nq, (q / nq) % nq, dim == 3 ? q / (nq * nq) : 0};
      double X[3], x[3], J[3][3], w = 1.0, phi = 1.0;
      for (int m = 0; m < dim; ++m) {
        X[m] = h * (cc[m] + tab.x[qi[m]]);
        w *= tab.w[qi[m]];
        phi *= tab.V[qi[m] * 12 + ai[m]];
      }
      double det;
      if (geo.kind != 0) {
        map_geo(dim, geo, n, cc, X, x, J);
        if (dim == 3)
          det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        else
          det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      } else {
        for (int m = 0; m < dim; ++m) x[m] = X[m];
        det = 1.0;
      }
      for (int m = 0; m < dim; ++m) det *= h;
      double f = dim * pi * pi;
      for (int m = 0; m < dim; ++m) f *= sin(pi * x[m]);
      s += f * phi * w * det;
    }
    const int gx = K * cc[0] + ai[0], gy = K * cc[1] + ai[1], gz = K * cc[2] + ai[2];
    const bool bnd = gx == 0 || gx == N1 - 1 || gy == 0 || gy == N1 - 1 || (dim == 3 && (gz == 0 || gz == N1 - 1));
    if (!bnd) b[gx + (int64_t)N1 * (gy + (int64_t)N1 * gz)] += s;
  }
}

cudaError_t rhs_manufactured(int dim, int n, int K, const GeomDesc& geo, const QuadTab& tab, double* b,
                             cudaStream_t st) {
  const int N1 = K * n + 1;
  const int64_t N = dim == 3 ? (int64_t)N1 * N1 * N1 : (int64_t)N1 * N1;
  cudaError_t e = cudaMemsetAsync(b, 0, sizeof(double) * N, st);
  if (e != cudaSuccess) return e;
  const int NP = dim == 3 ? (K + 1) * (K + 1) * (K + 1) : (K + 1) * (K + 1);
  for (int colour = 0; colour < (1 << dim); ++colour) {
    const int64_t work = (dim == 3 ? (int64_t)n * n * n : (int64_t)n * n) / (1 << dim) * NP + NP * 8;
    rhs_kernel<<<grid_for(work, 128, 152 * 32), 128, 0, st>>>(dim, n, K, geo, tab, b, colour);
    g_launches += 1;
  }
  return cudaGetLastError();
}

// per-block partial of sum over cells of sum_q (u_h - u)^2 w det J
__global__ void __launch_bounds__(256) l2err_kernel(int dim, int n, int K, GeomDesc geo, QuadTab tab,
                                                    const double* __restrict__ xv, double* __restrict__ partial) {
  const int n1 = K + 1;
  const int nq = tab.nq;
  const int NQ = dim == 3 ? nq * nq * nq : nq * nq;
  const int64_t ncell = dim == 3 ? (int64_t)n * n * n : (int64_t)n * n;
  const int N1 = K * n + 1;
  const double h = 1.0 / n;
  const double pi = 3.141592653589793238462643383279502884;
  double acc = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ncell * NQ;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(t % NQ);
    const int64_t cell = t / NQ;
    const int cc[3] = {(int)(cell % n), (int)((cell / n) % n), dim == 3 ? (int)(cell / ((int64_t)n * n)) : 0};
    const int qi[3] = {q % nq, (q / nq) % nq, dim == 3 ? q / (nq * nq) : 0};
    double X[3], x[3], J[3][3], w = 1.0;
    for (int m = 0; m < dim; ++m) {
      X[m] = h * (cc[m] + tab.x[qi[m]]);
      w *= tab.w[qi[m]];
    }
    double det;
    if (geo.kind != 0) {
      map_geo(dim, geo, n, cc, X, x, J);
      if (dim == 3)
        det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
              J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
      else
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    } else {
      for (int m = 0; m < dim; ++m) x[m] = X[m];
      det = 1.0;
    }
    for (int m = 0; m < dim; ++m) det *= h;
    double uh = 0.0;
    const int NPn = dim == 3 ? n1 * n1 * n1 : n1 * n1;
    for (int a = 0; a < NPn; ++a) {
      const int ai[3] = {a % n1, (a / n1) % n1, dim == 3 ? a / (n1 * n1) : 0};
      double phi = 1.0;
      for (int m = 0; m < dim; ++m) phi *= tab.V[qi[m] * 12 + ai[m]];
      const int gx = K * cc[0] + ai[0], gy = K * cc[1] + ai[1], gz = K * cc[2] + ai[2];
      const bool bnd = gx == 0 || gx == N1 - 1 || gy == 0 || gy == N1 - 1 || (dim == 3 && (gz == 0 || gz == N1 - 1));
      if (!bnd) uh += phi * xv[gx + (int64_t)N1 * (gy + (int64_t)N1 * gz)];
    }
    double u = 1.0;
    for (int m = 0; m < dim; ++m) u *= sin(pi * x[m]);
    acc += (uh - u) * (uh - u) * w * det;
  }
  block_store_sum(acc, partial + blockIdx.x);
}

cudaError_t l2_error_partials(int dim, int n, int K, const GeomDesc& geo, const QuadTab& tab, const double* x,
                              double* partial, double* out, cudaStream_t st) {
  l2err_kernel<<<kDotBlocks, 256, 0, st>>>(dim, n, K, geo, tab, x, partial);
  sum_partials_kernel<<<1, 256, 0, st>>>(partial, kDotBlocks, out);
  g_launches += 2;
  return cudaGetLastError();
}

}  // namespace pmg
