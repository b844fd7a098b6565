// Launch wrappers for one part of the kernel library -- degree K (PMG_K),
// dimension PMG_DIM, precision PMG_PREC (0 = double, 1 = float) -- and the
// table that exposes them.  inst.cu defines the part's namespace and table
// name from those three macros and includes this file; every wrapper checks
// that the (dim, prec) it is asked for is its own.
#pragma once
#include <type_traits>

#include "kernels.cuh"
#include "kernels_def.cuh"

namespace pmg {
namespace PMG_KNS {

using TP = std::conditional_t<PMG_PREC == 0, double, float>;
constexpr int DP = PMG_DIM;

static bool mine(int dim, int prec) { return dim == DP && prec == PMG_PREC; }

static cudaError_t upload(const double* coef) {
  const int n = LAY.total;
  float tmp[kMaxCoef];
  for (int i = 0; i < n; ++i) tmp[i] = (float)coef[i];
  cudaError_t e = cudaMemcpyToSymbol(c_coef64, coef, sizeof(double) * n);
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(c_coef32, tmp, sizeof(float) * n);
}

template <int DIM, typename T>
static cudaError_t cart_apply_t(const T* x, T* y, const T* b, T* t0, T* t1, T* t2, T* t3, int n, T s,
                                cudaStream_t st) {
  const int N1 = K * n + 1;
  const int64_t work = (int64_t)(n + 1) * (DIM == 3 ? (int64_t)N1 * N1 : N1);
  const int bs = 256;
  const int g = grid_for(work, bs);
  const FastDiv dnp1(n + 1), dN1(N1);
  if constexpr (DIM == 3 && sizeof(T) == 4) {  // FP32: x and y passes fused per z plane (cart_xy_kernel)
    const int tiles = (n + CartXY<T>::CX - 1) / CartXY<T>::CX;
    cart_xy_kernel<T><<<dim3(tiles, tiles, N1), 256, 0, st>>>(x, t2, t3, n);
    if (b) cart_pass<3, 2, 2, true, T><<<g, bs, 0, st>>>(t2, t3, y, nullptr, b, n, s, dnp1, dN1);
    else cart_pass<3, 2, 2, false, T><<<g, bs, 0, st>>>(t2, t3, y, nullptr, nullptr, n, s, dnp1, dN1);
    g_launches += 2;
    (void)t0;
    (void)t1;
  } else if (DIM == 3) {
    cart_pass<3, 0, 0, false, T><<<g, bs, 0, st>>>(x, nullptr, t0, t1, nullptr, n, s, dnp1, dN1);
    cart_pass<3, 1, 1, false, T><<<g, bs, 0, st>>>(t0, t1, t2, t3, nullptr, n, s, dnp1, dN1);
    if (b) cart_pass<3, 2, 2, true, T><<<g, bs, 0, st>>>(t2, t3, y, nullptr, b, n, s, dnp1, dN1);
    else cart_pass<3, 2, 2, false, T><<<g, bs, 0, st>>>(t2, t3, y, nullptr, nullptr, n, s, dnp1, dN1);
    g_launches += 3;
  } else {
    cart_pass<2, 0, 0, false, T><<<g, bs, 0, st>>>(x, nullptr, t0, t1, nullptr, n, s, dnp1, dN1);
    if (b) cart_pass<2, 1, 2, true, T><<<g, bs, 0, st>>>(t0, t1, y, nullptr, b, n, s, dnp1, dN1);
    else cart_pass<2, 1, 2, false, T><<<g, bs, 0, st>>>(t0, t1, y, nullptr, nullptr, n, s, dnp1, dN1);
    g_launches += 2;
  }
  return cudaGetLastError();
}

static cudaError_t cart_apply(int dim, int prec, const void* x, void* y, const void* b, void* t0, void* t1,
                              void* t2, void* t3, int n, double scale, cudaStream_t s) {
  if (!mine(dim, prec)) return cudaErrorInvalidValue;
  return cart_apply_t<DP, TP>((const TP*)x, (TP*)y, (const TP*)b, (TP*)t0, (TP*)t1, (TP*)t2, (TP*)t3, n, (TP)scale,
                              s);
}

// y = A x or y = b - A x for FP64 vectors in float-float arithmetic
// (cart_pass_ff); t0..t3: FP64-sized scratch, each holding a float-pair plane
template <int DIM>
static cudaError_t cart_apply_ff_t(const double* x, double* y, const double* b, void* t0, void* t1, void* t2,
                                   void* t3, int n, double scale, cudaStream_t st) {
  const int N1 = K * n + 1;
  const int64_t work = (int64_t)(n + 1) * (DIM == 3 ? (int64_t)N1 * N1 : N1);
  const int bs = 256;
  const int g = grid_for(work, bs);
  const FastDiv dnp1(n + 1), dN1(N1);
  const float sh = (float)scale;
  const ff s{sh, (float)(scale - (double)sh)};
  float *f0 = (float*)t0, *f1 = (float*)t1, *f2 = (float*)t2, *f3 = (float*)t3;
  if (DIM == 3) {
    cart_pass_ff<3, 0, 0, false><<<g, bs, 0, st>>>(x, nullptr, f0, f1, nullptr, n, s, dnp1, dN1);
    cart_pass_ff<3, 1, 1, false><<<g, bs, 0, st>>>(f0, f1, f2, f3, nullptr, n, s, dnp1, dN1);
    if (b) cart_pass_ff<3, 2, 2, true><<<g, bs, 0, st>>>(f2, f3, y, nullptr, b, n, s, dnp1, dN1);
    else cart_pass_ff<3, 2, 2, false><<<g, bs, 0, st>>>(f2, f3, y, nullptr, nullptr, n, s, dnp1, dN1);
    g_launches += 3;
  } else {
    cart_pass_ff<2, 0, 0, false><<<g, bs, 0, st>>>(x, nullptr, f0, f1, nullptr, n, s, dnp1, dN1);
    if (b) cart_pass_ff<2, 1, 2, true><<<g, bs, 0, st>>>(f0, f1, y, nullptr, b, n, s, dnp1, dN1);
    else cart_pass_ff<2, 1, 2, false><<<g, bs, 0, st>>>(f0, f1, y, nullptr, nullptr, n, s, dnp1, dN1);
    g_launches += 2;
  }
  return cudaGetLastError();
}

static cudaError_t cart_apply_ff(int dim, const double* x, double* y, const double* b, void* t0, void* t1, void* t2,
                                 void* t3, int n, double scale, cudaStream_t s) {
  if (dim != DP) return cudaErrorInvalidValue;
  return cart_apply_ff_t<DP>(x, y, b, t0, t1, t2, t3, n, scale, s);
}

static int patch_threads(int dim) { return dim == 3 ? PatchShape<3>::TPP : PatchShape<2>::TPP; }

// shared bytes per patch of the patch-major layout
static int patch_smem(int dim, int prec, int n_iter) {
  const int es = prec == 0 ? 8 : 4;
  const int elems = dim == 3 ? (prec == 0 ? PatchShape<3>::stride<double>(n_iter) : PatchShape<3>::stride<float>(n_iter))
                             : (prec == 0 ? PatchShape<2>::stride<double>(n_iter) : PatchShape<2>::stride<float>(n_iter));
  return elems * es;
}

// shared bytes per patch of the interleaved layout (no padding)
static int patch_il_smem(int dim, int prec, int n_iter) {
  const int es = prec == 0 ? 8 : 4;
  const int elems = dim == 3 ? PatchShape<3>::ELEMS + (n_iter > 1 ? 2 * PatchShape<3>::SZT : 0)
                             : PatchShape<2>::ELEMS + (n_iter > 1 ? 2 * PatchShape<2>::SZT : 0);
  return elems * es;
}

static int dinv_len(int dim) {
  int len = 0;
  for (int l = 1; l < nlev(K); ++l) len += ipow(mp(plev(K, l)), dim);
  return len;
}

// shared memory of the block besides its patches: the inverse-diagonal tables
// when the block stages them (stage_dinv)
static int patch_cart_extra_smem(int dim, int prec) {
  const bool staged = dim == 3 ? (prec == 0 ? stage_dinv<3, double>() : stage_dinv<3, float>())
                               : (prec == 0 ? stage_dinv<2, double>() : stage_dinv<2, float>());
  return staged ? dinv_len(dim) * (prec == 0 ? 8 : 4) : 0;
}

// Grid of a persistent patch launch: every block the GPU can hold at once
// (occupancy x SMs), at most one per batch.
static unsigned persistent_grid(const void* kern, int threads, int smem, int64_t nbatch) {
  int dev = 0, sms = 152, per_sm = 1;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  const int64_t g = std::min<int64_t>(nbatch, (int64_t)sms * per_sm);
  return (unsigned)std::max<int64_t>(g, 1);
}

template <int DIM, typename T>
static cudaError_t patch_cart_t(const T* r, T* dst, int n, int ppc, int n_iter, const T* dinv,
                                const PatchParamsHost& H, int* counter, cudaStream_t st) {
  using S = PatchShape<DIM>;
  const int64_t np = patch_count(DIM, n, H.colour);
  if (np == 0) return cudaSuccess;  // no interior vertex (of this colour), no patch
  if (ppc < 1 || ppc > kMaxPatchesPerBlock) return cudaErrorInvalidValue;
  const int64_t nbatch = (np + ppc - 1) / ppc;
  // more patch lines than threads is fine: every step loops over its lines
  const int threads = std::min(kPatchMaxThreads, (ppc * S::TPP + 31) / 32 * 32);
  const int prec = sizeof(T) == 8 ? 0 : 1;
  const int smem = ppc * patch_smem(DIM, prec, n_iter) + patch_cart_extra_smem(DIM, prec);
  if (smem > kMaxDynSmem) return cudaErrorInvalidConfiguration;
  unsigned grid = (unsigned)nbatch;
  if (counter) {
    grid = persistent_grid((const void*)patch_cart_kernel<DIM, T>, threads, smem, nbatch);
    if (grid < nbatch) {  // more than one wave: persistent blocks
      cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
      if (e != cudaSuccess) return e;
    } else {
      grid = (unsigned)nbatch;
      counter = nullptr;
    }
  }
  patch_cart_kernel<DIM, T><<<grid, threads, smem, st>>>(r, dst, n, ppc, n_iter, dinv, dinv_len(DIM), to_params<T>(H),
                                                         counter, nbatch);
  g_launches += 1;
  return cudaGetLastError();
}

static cudaError_t patch_cart(int dim, int prec, const void* r, void* dst, int n, int ppc, int n_iter,
                              const void* dinv, const PatchParamsHost& P, int* counter, cudaStream_t s) {
  if (!mine(dim, prec)) return cudaErrorInvalidValue;
  return patch_cart_t<DP, TP>((const TP*)r, (TP*)dst, n, ppc, n_iter, (const TP*)dinv, P, counter, s);
}

// Interleaved layout: patches per block of this part's interleaved kernel
// for n_iter local cycles, or 0 when it has none or they do not fit.
static int patch_il_of(int dim, int prec, int n_iter) {
  if (!mine(dim, prec)) return 0;
  constexpr int il = patch_il<DP, TP>();
  if (il == 0) return 0;
  const int smem = il * patch_il_smem(dim, prec, n_iter) + patch_cart_extra_smem(dim, prec);
  return smem <= kMaxDynSmem ? il : 0;
}

template <int DIM, typename T>
static cudaError_t patch_cart_il_t(const T* r, T* dst, int n, int threads, int n_iter, const T* dinv,
                                   const PatchParamsHost& H, int* counter, cudaStream_t st) {
  const int64_t np = patch_count(DIM, n, H.colour);
  if (np == 0) return cudaSuccess;
  const int prec = sizeof(T) == 8 ? 0 : 1;
  const int il = patch_il_of(DIM, prec, n_iter);
  if (il == 0 || threads < 32 || threads > 1024 || threads % 32) return cudaErrorInvalidValue;
  const int smem = il * patch_il_smem(DIM, prec, n_iter) + patch_cart_extra_smem(DIM, prec);
  const int64_t nbatch = (np + il - 1) / il;
  unsigned grid = (unsigned)nbatch;
  if (counter) {
    grid = persistent_grid((const void*)patch_cart_il_kernel<DIM, T>, threads, smem, nbatch);
    if (grid < nbatch) {
      cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
      if (e != cudaSuccess) return e;
    } else {
      grid = (unsigned)nbatch;
      counter = nullptr;
    }
  }
  patch_cart_il_kernel<DIM, T><<<grid, threads, smem, st>>>(r, dst, n, n_iter, dinv, dinv_len(DIM), to_params<T>(H),
                                                            counter, nbatch);
  g_launches += 1;
  return cudaGetLastError();
}

static cudaError_t patch_cart_il(int dim, int prec, const void* r, void* dst, int n, int threads, int n_iter,
                                 const void* dinv, const PatchParamsHost& P, int* counter, cudaStream_t s) {
  if (!mine(dim, prec)) return cudaErrorInvalidValue;
  return patch_cart_il_t<DP, TP>((const TP*)r, (TP*)dst, n, threads, n_iter, (const TP*)dinv, P, counter, s);
}

// u (+)= the summed patch corrections held in dst (add = 0: u = sum)
template <int DIM, typename T>
static cudaError_t patch_gather_t(const T* dst, T* u, int n, int add, cudaStream_t st) {
  const int64_t N = ipow(K * n + 1, DIM);
  if (add) patch_gather_kernel<DIM, true, T><<<grid_for(N, 256), 256, 0, st>>>(dst, u, n, FastDiv(K * n + 1));
  else patch_gather_kernel<DIM, false, T><<<grid_for(N, 256), 256, 0, st>>>(dst, u, n, FastDiv(K * n + 1));
  g_launches += 1;
  return cudaGetLastError();
}

static cudaError_t patch_gather(int dim, int prec, const void* dst, void* u, int n, int add, cudaStream_t s) {
  if (!mine(dim, prec)) return cudaErrorInvalidValue;
  return patch_gather_t<DP, TP>((const TP*)dst, (TP*)u, n, add, s);
}

template <int DIM, typename T>
static cudaError_t h_prolong_t(const T* uc, T* uf, T* t0, T* t1, int nc, cudaStream_t st) {
  const int c1 = K * nc + 1, f1 = 2 * K * nc + 1;
  const int bs = 256;
  if (DIM == 3) {
    hprolong_pass<0, false, T><<<grid_for((int64_t)f1 * c1 * c1, bs), bs, 0, st>>>(uc, t0, nc, f1, c1, c1, FastDiv(f1), FastDiv(c1));
    hprolong_pass<1, false, T><<<grid_for((int64_t)f1 * f1 * c1, bs), bs, 0, st>>>(t0, t1, nc, f1, f1, c1, FastDiv(f1), FastDiv(f1));
    hprolong_pass<2, true, T><<<grid_for((int64_t)f1 * f1 * f1, bs), bs, 0, st>>>(t1, uf, nc, f1, f1, f1, FastDiv(f1), FastDiv(f1));
    g_launches += 3;
  } else {
    hprolong_pass<0, false, T><<<grid_for((int64_t)f1 * c1, bs), bs, 0, st>>>(uc, t0, nc, f1, c1, 1, FastDiv(f1), FastDiv(c1));
    hprolong_pass<1, true, T><<<grid_for((int64_t)f1 * f1, bs), bs, 0, st>>>(t0, uf, nc, f1, f1, 1, FastDiv(f1), FastDiv(f1));
    g_launches += 2;
  }
  return cudaGetLastError();
}

template <int DIM, typename T>
static cudaError_t h_restrict_t(const T* rf, T* rc, T* t0, T* t1, int nc, cudaStream_t st) {
  const int c1 = K * nc + 1, f1 = 2 * K * nc + 1;
  const int bs = 256;
  if (DIM == 3) {
    hrestrict_pass<2, T><<<grid_for((int64_t)f1 * f1 * c1, bs), bs, 0, st>>>(rf, t0, nc, f1, f1, c1, FastDiv(f1), FastDiv(f1));
    hrestrict_pass<1, T><<<grid_for((int64_t)f1 * c1 * c1, bs), bs, 0, st>>>(t0, t1, nc, f1, c1, c1, FastDiv(f1), FastDiv(c1));
    hrestrict_pass<0, T><<<grid_for((int64_t)c1 * c1 * c1, bs), bs, 0, st>>>(t1, rc, nc, c1, c1, c1, FastDiv(c1), FastDiv(c1));
    g_launches += 3;
  } else {
    hrestrict_pass<1, T><<<grid_for((int64_t)f1 * c1, bs), bs, 0, st>>>(rf, t0, nc, f1, c1, 1, FastDiv(f1), FastDiv(c1));
    hrestrict_pass<0, T><<<grid_for((int64_t)c1 * c1, bs), bs, 0, st>>>(t0, rc, nc, c1, c1, 1, FastDiv(c1), FastDiv(c1));
    g_launches += 2;
  }
  return cudaGetLastError();
}

static cudaError_t h_prolong_add(int dim, int prec, const void* uc, void* uf, void* t0, void* t1, int nc,
                                 cudaStream_t s) {
  if (!mine(dim, prec)) return cudaErrorInvalidValue;
  return h_prolong_t<DP, TP>((const TP*)uc, (TP*)uf, (TP*)t0, (TP*)t1, nc, s);
}

static cudaError_t h_restrict(int dim, int prec, const void* rf, void* rc, void* t0, void* t1, int nc,
                              cudaStream_t s) {
  if (!mine(dim, prec)) return cudaErrorInvalidValue;
  return h_restrict_t<DP, TP>((const TP*)rf, (TP*)rc, (TP*)t0, (TP*)t1, nc, s);
}

// ---------------------------------------------------------------- grouped launches
// One launch per pass for all jobs; every job's results are those of its own
// launch (each thread takes the same grid-stride slice of every job; the
// patch launch gives each batch of each job to one block).
static int64_t apply_work(int dim, int n) {
  const int64_t N1 = (int64_t)K * n + 1;
  return (int64_t)(n + 1) * (dim == 3 ? N1 * N1 : N1);
}

static bool group_ok(int count) { return count >= 1 && count <= kMaxGroup; }

template <int DIM, typename T>
static cudaError_t cart_apply_group_t(int count, const ApplyJob* jobs, cudaStream_t st) {
  GroupOf<CartPassJob<T>> g0, g1, g2;
  g0.count = g1.count = g2.count = count;
  g0.start[0] = 0;
  int64_t work = 0;
  bool resid = jobs[0].b != nullptr;
  for (int j = 0; j < count; ++j) {
    const ApplyJob& a = jobs[j];
    if ((a.b != nullptr) != resid) return cudaErrorInvalidValue;  // one pass kind per launch
    const T* x = (const T*)a.x;
    T* t0 = (T*)a.t[0];
    T* t1 = (T*)a.t[1];
    T* t2 = (T*)a.t[2];
    T* t3 = (T*)a.t[3];
    const T s = (T)a.scale;
    g0.job[j] = CartPassJob<T>{x, nullptr, t0, t1, nullptr, a.n, s, FastDiv(a.n + 1), FastDiv(K * a.n + 1)};
    if (DIM == 3) {
      g1.job[j] = CartPassJob<T>{t0, t1, t2, t3, nullptr, a.n, s, FastDiv(a.n + 1), FastDiv(K * a.n + 1)};
      g2.job[j] = CartPassJob<T>{t2, t3, (T*)a.y, nullptr, (const T*)a.b, a.n, s, FastDiv(a.n + 1), FastDiv(K * a.n + 1)};
    } else {
      g1.job[j] = CartPassJob<T>{t0, t1, (T*)a.y, nullptr, (const T*)a.b, a.n, s, FastDiv(a.n + 1), FastDiv(K * a.n + 1)};
    }
    work += apply_work(DIM, a.n);
    g0.start[j + 1] = work;
  }
  for (int j = 0; j <= count; ++j) g1.start[j] = g2.start[j] = g0.start[j];
  const int bs = 256, g = grid_for(work, bs);
  if (DIM == 3) {
    cart_pass_group<3, 0, 0, false, T><<<g, bs, 0, st>>>(g0);
    cart_pass_group<3, 1, 1, false, T><<<g, bs, 0, st>>>(g1);
    if (resid) cart_pass_group<3, 2, 2, true, T><<<g, bs, 0, st>>>(g2);
    else cart_pass_group<3, 2, 2, false, T><<<g, bs, 0, st>>>(g2);
    g_launches += 3;
  } else {
    cart_pass_group<2, 0, 0, false, T><<<g, bs, 0, st>>>(g0);
    if (resid) cart_pass_group<2, 1, 2, true, T><<<g, bs, 0, st>>>(g1);
    else cart_pass_group<2, 1, 2, false, T><<<g, bs, 0, st>>>(g1);
    g_launches += 2;
  }
  return cudaGetLastError();
}

static cudaError_t cart_apply_group(int dim, int prec, int count, const ApplyJob* jobs, cudaStream_t s) {
  if (!mine(dim, prec) || !group_ok(count)) return cudaErrorInvalidValue;
  return cart_apply_group_t<DP, TP>(count, jobs, s);
}

template <int DIM>
static cudaError_t cart_apply_ff_group_t(int count, const ApplyJob* jobs, cudaStream_t st) {
  GroupOf<CartPassFFJob> g0, g1, g2;
  g0.count = g1.count = g2.count = count;
  g0.start[0] = 0;
  int64_t work = 0;
  const bool resid = jobs[0].b != nullptr;
  for (int j = 0; j < count; ++j) {
    const ApplyJob& a = jobs[j];
    if ((a.b != nullptr) != resid) return cudaErrorInvalidValue;
    const float sh = (float)a.scale;
    const ff s{sh, (float)(a.scale - (double)sh)};
    float *f0 = (float*)a.t[0], *f1 = (float*)a.t[1], *f2 = (float*)a.t[2], *f3 = (float*)a.t[3];
    g0.job[j] = CartPassFFJob{a.x, nullptr, f0, f1, nullptr, a.n, s, FastDiv(a.n + 1), FastDiv(K * a.n + 1)};
    if (DIM == 3) {
      g1.job[j] = CartPassFFJob{f0, f1, f2, f3, nullptr, a.n, s, FastDiv(a.n + 1), FastDiv(K * a.n + 1)};
      g2.job[j] = CartPassFFJob{f2, f3, a.y, nullptr, (const double*)a.b, a.n, s, FastDiv(a.n + 1), FastDiv(K * a.n + 1)};
    } else {
      g1.job[j] = CartPassFFJob{f0, f1, a.y, nullptr, (const double*)a.b, a.n, s, FastDiv(a.n + 1), FastDiv(K * a.n + 1)};
    }
    work += apply_work(DIM, a.n);
    g0.start[j + 1] = work;
  }
  for (int j = 0; j <= count; ++j) g1.start[j] = g2.start[j] = g0.start[j];
  const int bs = 256, g = grid_for(work, bs);
  if (DIM == 3) {
    cart_pass_ff_group<3, 0, 0, false><<<g, bs, 0, st>>>(g0);
    cart_pass_ff_group<3, 1, 1, false><<<g, bs, 0, st>>>(g1);
    if (resid) cart_pass_ff_group<3, 2, 2, true><<<g, bs, 0, st>>>(g2);
    else cart_pass_ff_group<3, 2, 2, false><<<g, bs, 0, st>>>(g2);
    g_launches += 3;
  } else {
    cart_pass_ff_group<2, 0, 0, false><<<g, bs, 0, st>>>(g0);
    if (resid) cart_pass_ff_group<2, 1, 2, true><<<g, bs, 0, st>>>(g1);
    else cart_pass_ff_group<2, 1, 2, false><<<g, bs, 0, st>>>(g1);
    g_launches += 2;
  }
  return cudaGetLastError();
}

static cudaError_t cart_apply_ff_group(int dim, int count, const ApplyJob* jobs, cudaStream_t s) {
  if (dim != DP || !group_ok(count)) return cudaErrorInvalidValue;
  return cart_apply_ff_group_t<DP>(count, jobs, s);
}

template <int DIM, typename T>
static cudaError_t patch_cart_group_t(int count, const PatchSolveJob* jobs, int ppc, int n_iter, const T* dinv,
                                      int* counter, cudaStream_t st) {
  using S = PatchShape<DIM>;
  if (ppc < 1 || ppc > kMaxPatchesPerBlock) return cudaErrorInvalidValue;
  GroupOf<PatchJob<T>> G;
  G.count = 0;
  G.start[0] = 0;
  int64_t nbatch = 0;
  for (int j = 0; j < count; ++j) {
    const int64_t np = patch_count(DIM, jobs[j].n, jobs[j].P.colour);
    if (np == 0) continue;  // no patch (of this colour) on this job's level
    PatchJob<T>& J = G.job[G.count++];
    J.r = (const T*)jobs[j].r;
    J.dst = (T*)jobs[j].dst;
    J.n = jobs[j].n;
    J.P = to_params<T>(jobs[j].P);
    nbatch += (np + ppc - 1) / ppc;
    G.start[G.count] = nbatch;
  }
  if (G.count == 0) return cudaSuccess;
  const int threads = std::min(kPatchMaxThreads, (ppc * S::TPP + 31) / 32 * 32);
  const int prec = sizeof(T) == 8 ? 0 : 1;
  const int smem = ppc * patch_smem(DIM, prec, n_iter) + patch_cart_extra_smem(DIM, prec);
  if (smem > kMaxDynSmem) return cudaErrorInvalidConfiguration;
  unsigned grid = (unsigned)nbatch;
  if (counter) {
    grid = persistent_grid((const void*)patch_cart_group_kernel<DIM, T>, threads, smem, nbatch);
    if (grid < nbatch) {
      cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
      if (e != cudaSuccess) return e;
    } else {
      grid = (unsigned)nbatch;
      counter = nullptr;
    }
  }
  patch_cart_group_kernel<DIM, T><<<grid, threads, smem, st>>>(ppc, n_iter, dinv, dinv_len(DIM), counter, nbatch, G);
  g_launches += 1;
  return cudaGetLastError();
}

static cudaError_t patch_cart_group(int dim, int prec, int count, const PatchSolveJob* jobs, int ppc, int n_iter,
                                    const void* dinv, int* counter, cudaStream_t s) {
  if (!mine(dim, prec) || !group_ok(count)) return cudaErrorInvalidValue;
  return patch_cart_group_t<DP, TP>(count, jobs, ppc, n_iter, (const TP*)dinv, counter, s);
}

template <int DIM, typename T>
static cudaError_t patch_gather_group_t(int count, const GatherSolveJob* jobs, int add, cudaStream_t st) {
  GroupOf<GatherJob<T>> G;
  G.count = count;
  G.start[0] = 0;
  int64_t work = 0;
  for (int j = 0; j < count; ++j) {
    G.job[j] = GatherJob<T>{(const T*)jobs[j].dst, (T*)jobs[j].u, jobs[j].n, FastDiv(K * jobs[j].n + 1)};
    work += ipow(K * jobs[j].n + 1, DIM);
    G.start[j + 1] = work;
  }
  if (add) patch_gather_group<DIM, true, T><<<grid_for(work, 256), 256, 0, st>>>(G);
  else patch_gather_group<DIM, false, T><<<grid_for(work, 256), 256, 0, st>>>(G);
  g_launches += 1;
  return cudaGetLastError();
}

static cudaError_t patch_gather_group(int dim, int prec, int count, const GatherSolveJob* jobs, int add,
                                     cudaStream_t s) {
  if (!mine(dim, prec) || !group_ok(count)) return cudaErrorInvalidValue;
  return patch_gather_group_t<DP, TP>(count, jobs, add, s);
}

// The passes of h_prolong_t / h_restrict_t with each job's extents.
template <int DIM, typename T>
static cudaError_t h_prolong_group_t(int count, const TransferSolveJob* jobs, cudaStream_t st) {
  GroupOf<TransferJob<T>> g[3];
  int64_t work[3] = {0, 0, 0};
  for (int i = 0; i < 3; ++i) {
    g[i].count = count;
    g[i].start[0] = 0;
  }
  for (int j = 0; j < count; ++j) {
    const TransferSolveJob& a = jobs[j];
    const int nc = a.nc, c1 = K * nc + 1, f1 = 2 * K * nc + 1;
    const T* uc = (const T*)a.in;
    T *uf = (T*)a.out, *t0 = (T*)a.t0, *t1 = (T*)a.t1;
    if (DIM == 3) {
      g[0].job[j] = TransferJob<T>{uc, t0, nc, f1, c1, c1, FastDiv(f1), FastDiv(c1)};
      g[1].job[j] = TransferJob<T>{t0, t1, nc, f1, f1, c1, FastDiv(f1), FastDiv(f1)};
      g[2].job[j] = TransferJob<T>{t1, uf, nc, f1, f1, f1, FastDiv(f1), FastDiv(f1)};
      work[0] += (int64_t)f1 * c1 * c1;
      work[1] += (int64_t)f1 * f1 * c1;
      work[2] += (int64_t)f1 * f1 * f1;
    } else {
      g[0].job[j] = TransferJob<T>{uc, t0, nc, f1, c1, 1, FastDiv(f1), FastDiv(c1)};
      g[1].job[j] = TransferJob<T>{t0, uf, nc, f1, f1, 1, FastDiv(f1), FastDiv(f1)};
      work[0] += (int64_t)f1 * c1;
      work[1] += (int64_t)f1 * f1;
    }
    for (int i = 0; i < 3; ++i) g[i].start[j + 1] = work[i];
  }
  const int bs = 256;
  if (DIM == 3) {
    hprolong_group<0, false, T><<<grid_for(work[0], bs), bs, 0, st>>>(g[0]);
    hprolong_group<1, false, T><<<grid_for(work[1], bs), bs, 0, st>>>(g[1]);
    hprolong_group<2, true, T><<<grid_for(work[2], bs), bs, 0, st>>>(g[2]);
    g_launches += 3;
  } else {
    hprolong_group<0, false, T><<<grid_for(work[0], bs), bs, 0, st>>>(g[0]);
    hprolong_group<1, true, T><<<grid_for(work[1], bs), bs, 0, st>>>(g[1]);
    g_launches += 2;
  }
  return cudaGetLastError();
}

template <int DIM, typename T>
static cudaError_t h_restrict_group_t(int count, const TransferSolveJob* jobs, cudaStream_t st) {
  GroupOf<TransferJob<T>> g[3];
  int64_t work[3] = {0, 0, 0};
  for (int i = 0; i < 3; ++i) {
    g[i].count = count;
    g[i].start[0] = 0;
  }
  for (int j = 0; j < count; ++j) {
    const TransferSolveJob& a = jobs[j];
    const int nc = a.nc, c1 = K * nc + 1, f1 = 2 * K * nc + 1;
    const T* rf = (const T*)a.in;
    T *rc = (T*)a.out, *t0 = (T*)a.t0, *t1 = (T*)a.t1;
    if (DIM == 3) {
      g[0].job[j] = TransferJob<T>{rf, t0, nc, f1, f1, c1, FastDiv(f1), FastDiv(f1)};
      g[1].job[j] = TransferJob<T>{t0, t1, nc, f1, c1, c1, FastDiv(f1), FastDiv(c1)};
      g[2].job[j] = TransferJob<T>{t1, rc, nc, c1, c1, c1, FastDiv(c1), FastDiv(c1)};
      work[0] += (int64_t)f1 * f1 * c1;
      work[1] += (int64_t)f1 * c1 * c1;
      work[2] += (int64_t)c1 * c1 * c1;
    } else {
      g[0].job[j] = TransferJob<T>{rf, t0, nc, f1, c1, 1, FastDiv(f1), FastDiv(c1)};
      g[1].job[j] = TransferJob<T>{t0, rc, nc, c1, c1, 1, FastDiv(c1), FastDiv(c1)};
      work[0] += (int64_t)f1 * c1;
      work[1] += (int64_t)c1 * c1;
    }
    for (int i = 0; i < 3; ++i) g[i].start[j + 1] = work[i];
  }
  const int bs = 256;
  if (DIM == 3) {
    hrestrict_group<2, T><<<grid_for(work[0], bs), bs, 0, st>>>(g[0]);
    hrestrict_group<1, T><<<grid_for(work[1], bs), bs, 0, st>>>(g[1]);
    hrestrict_group<0, T><<<grid_for(work[2], bs), bs, 0, st>>>(g[2]);
    g_launches += 3;
  } else {
    hrestrict_group<1, T><<<grid_for(work[0], bs), bs, 0, st>>>(g[0]);
    hrestrict_group<0, T><<<grid_for(work[1], bs), bs, 0, st>>>(g[1]);
    g_launches += 2;
  }
  return cudaGetLastError();
}

static cudaError_t h_prolong_add_group(int dim, int prec, int count, const TransferSolveJob* jobs, cudaStream_t s) {
  if (!mine(dim, prec) || !group_ok(count)) return cudaErrorInvalidValue;
  return h_prolong_group_t<DP, TP>(count, jobs, s);
}

static cudaError_t h_restrict_group(int dim, int prec, int count, const TransferSolveJob* jobs, cudaStream_t s) {
  if (!mine(dim, prec) || !group_ok(count)) return cudaErrorInvalidValue;
  return h_restrict_group_t<DP, TP>(count, jobs, s);
}

// Opt every kernel of this degree into the largest dynamic shared memory the
// device allows next to the kernel's static shared memory (called once per
// device at context creation, outside any stream capture).
template <class Kern>
static cudaError_t allow_smem(Kern k, int optin) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, k);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)a.sharedSizeBytes);
  if (e != cudaSuccess) return e;
  // prefer the largest shared-memory carve-out: these kernels live in it
  return cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

static int max_threads_of(const void* k) {
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, k) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return a.maxThreadsPerBlock;
}

static int patch_max_threads(int dim, int prec, int deformed) {
  if (!mine(dim, prec)) return 0;
  return deformed ? std::min(max_threads_of((const void*)patch_def_kernel<DP, TP, float>),
                             max_threads_of((const void*)patch_def_kernel<DP, TP, double>))
                  : max_threads_of((const void*)patch_cart_kernel<DP, TP>);
}

static int patch_il_max_threads(int dim, int prec) {
  if (!mine(dim, prec) || patch_il<DP, TP>() == 0) return 0;
  return max_threads_of((const void*)patch_cart_il_kernel<DP, TP>);
}

static cudaError_t prepare() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaError_t r = cudaSuccess;
  auto acc = [&](cudaError_t x) { if (x != cudaSuccess && r == cudaSuccess) r = x; };
  acc(allow_smem(patch_cart_kernel<DP, TP>, optin));
  acc(allow_smem(patch_cart_group_kernel<DP, TP>, optin));
  if (patch_il<DP, TP>() > 0) acc(allow_smem(patch_cart_il_kernel<DP, TP>, optin));
  acc(allow_smem(patch_def_kernel<DP, TP, float>, optin));
  acc(allow_smem(patch_def_kernel<DP, TP, double>, optin));
  acc(allow_smem(def_cell_kernel<DP, TP, float>, optin));
  acc(allow_smem(def_cell_kernel<DP, TP, double>, optin));
  return r;
}

}  // namespace PMG_KNS

const KernelTable* PMG_TABLE_FN() {
  static KernelTable t = {
      PMG_K,
      PMG_DIM,
      PMG_PREC,
      PMG_KNS::prepare,
      PMG_KNS::upload,
      PMG_KNS::cart_apply,
      PMG_KNS::patch_cart,
      PMG_KNS::patch_gather,
      PMG_KNS::patch_cart_extra_smem,
      PMG_KNS::patch_threads,
      PMG_KNS::patch_smem,
      PMG_KNS::h_prolong_add,
      PMG_KNS::h_restrict,
      PMG_KNS::def_apply,
      PMG_KNS::patch_def,
      PMG_KNS::patch_def_threads,
      PMG_KNS::patch_def_smem,
      PMG_KNS::patch_max_threads,
      PMG_KNS::patch_il_of,
      PMG_KNS::patch_cart_il,
      PMG_KNS::patch_il_max_threads,
      PMG_KNS::cart_apply_ff,
      PMG_KNS::def_apply_ff,
      PMG_KNS::def_apply_candidates,
      PMG_KNS::cart_apply_group,
      PMG_KNS::cart_apply_ff_group,
      PMG_KNS::patch_cart_group,
      PMG_KNS::patch_gather_group,
      PMG_KNS::h_prolong_add_group,
      PMG_KNS::h_restrict_group,
  };
  return &t;
}

}  // namespace pmg
