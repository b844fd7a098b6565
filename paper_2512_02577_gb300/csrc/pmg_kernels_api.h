// Table of kernel launchers of one part of the library -- degree k, dimension
// d, precision -- filled by inst.cu compiled for that part.  Host code
// (pmg.cu) looks a part up through kernel_table(k, d, prec); every entry
// enqueues on the given stream and returns the launch's cudaError_t, and
// rejects (cudaErrorInvalidValue) a (dim, prec) that is not its part's.
// Precision flag: 0 = double, 1 = float (element type of every vector).
// Each part has its own constant-memory copy of the degree's coefficients:
// upload() fills that copy.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "pmg_common.cuh"

namespace pmg {

struct PatchParamsHost {
  double scale;      // h^{d-2}
  double omega_as;
  double omega[4];
  double inv_a0;     // 1 / A_{j,1} (Cartesian)
  int half;          // 1: half local V-cycle (no post-smoothing, §3.2.2)
  int colour;        // -1: every patch, additive output (omega_AS d_j per colour
                     // vector); c >= 0: only the patches of parity colour c,
                     // u += d_j added straight into dst (multiplicative sweep)
};

// Deformed-geometry arrays of one mesh level (device pointers).
struct DefLevel {
  const void* G[4];       // per p-level: per cell, ncomp x (p+1)^d points (x fastest), FP64 or FP32 (gprec)
  int gprec;              // storage precision of G: 0 double, 1 float
  const void* dinv[4];    // per p-level l >= 1: inverse diagonal on the degree-p global grid (MG precision)
  const void* dinv1;      // p = 1: inverse Q1 diagonal on the vertex grid (n+1)^d (MG precision)
};

// Jobs of grouped launches: one launch does the operation for every job (one
// level of one system each; sizes may differ between jobs, at most kMaxGroup
// jobs), with each job's results those of its own ungrouped launch.
struct ApplyJob {       // y = A x or y = b - A x (b != nullptr); t: scratch of the level's N
  const void* x;
  void* y;
  const void* b;
  void* t[4];
  int n;
  double scale;
};
struct PatchSolveJob {  // patch smoother of one level (output as patch_cart)
  const void* r;
  void* dst;
  int n;
  PatchParamsHost P;
};
struct GatherSolveJob {  // u (+)= the patch corrections in dst
  const void* dst;
  void* u;
  int n;
};
struct TransferSolveJob {  // prolongation (uf += P uc) or restriction (rc = P^T rf); t: scratch of N_f
  const void* in;
  void* out;
  void* t0;
  void* t1;
  int nc;
};

struct KernelTable {
  int K;
  int dim;
  int prec;
  cudaError_t (*prepare)();
  cudaError_t (*upload)(const double* coef);
  // y = A x (b == nullptr) or y = b - A x; Cartesian; t0..t3: scratch of N
  cudaError_t (*cart_apply)(int dim, int prec, const void* x, void* y, const void* b, void* t0, void* t1,
                            void* t2, void* t3, int n, double scale, cudaStream_t s);
  // Cartesian patch smoother, every patch of the level: omega_AS d_j written at
  // dst[c N + node] for a patch of parity colour c (N nodes of the level).
  // counter: nullptr for one block per batch of patches, else one device int
  // of scratch for a persistent launch (reset on the stream before it; used
  // only when the batches exceed one wave of resident blocks).
  cudaError_t (*patch_cart)(int dim, int prec, const void* r, void* dst, int n, int ppc, int n_iter,
                            const void* dinv, const PatchParamsHost& P, int* counter, cudaStream_t s);
  // u (+)= sum over the patches holding each node of dst (add = 0: u = sum)
  cudaError_t (*patch_gather)(int dim, int prec, const void* dst, void* u, int n, int add, cudaStream_t s);
  int (*patch_cart_extra_smem)(int dim, int prec);  // block shared bytes besides its patches
  int (*patch_threads)(int dim);                  // threads per patch
  int (*patch_smem)(int dim, int prec, int n_iter);  // shared bytes per patch
  // u_f += P u_c  /  r_c = P^T r_f  (nc = coarse cells per side); t0, t1 scratch of N_f
  cudaError_t (*h_prolong_add)(int dim, int prec, const void* uc, void* uf, void* t0, void* t1, int nc,
                               cudaStream_t s);
  cudaError_t (*h_restrict)(int dim, int prec, const void* rf, void* rc, void* t0, void* t1, int nc,
                            cudaStream_t s);
  // deformed geometry: y = A x or y = b - A x with stored G (FP64 if gprec is
  // 0, else FP32); cellbuf: n^d (K+1)^d scratch values
  // cpb: cells per block, 0 = the part's rule (def_apply_candidates lists the
  // admissible values)
  cudaError_t (*def_apply)(int dim, int prec, const void* x, void* y, const void* b, const void* G, int gprec,
                           void* cellbuf, int n, int cpb, cudaStream_t s);
  // deformed patch smoother, every patch of the level (output as patch_cart)
  cudaError_t (*patch_def)(int dim, int prec, const void* r, void* dst, int n, int ppc, int n_iter,
                           const DefLevel& lev, const PatchParamsHost& P, cudaStream_t s);
  int (*patch_def_threads)(int dim);
  int (*patch_def_smem)(int dim, int prec, int n_iter);
  // largest block the patch kernel can launch with (registers included)
  int (*patch_max_threads)(int dim, int prec, int deformed);
  // Cartesian patch smoother with the interleaved shared-memory layout (IL
  // patches per block, element-major): IL for n_iter local cycles (0: no
  // such kernel, or it does not fit); launch with `threads` per block (a
  // multiple of 32); same output as patch_cart; largest admissible threads
  int (*patch_il)(int dim, int prec, int n_iter);
  cudaError_t (*patch_cart_il)(int dim, int prec, const void* r, void* dst, int n, int threads, int n_iter,
                               const void* dinv, const PatchParamsHost& P, int* counter, cudaStream_t s);
  int (*patch_il_max_threads)(int dim, int prec);
  // y = A x (b == nullptr) or y = b - A x for FP64 x, y, b on a Cartesian
  // level, computed in float-float arithmetic; t0..t3: scratch of N doubles
  cudaError_t (*cart_apply_ff)(int dim, const double* x, double* y, const double* b, void* t0, void* t1, void* t2,
                               void* t3, int n, double scale, cudaStream_t s);
  // the same on a deformed or distorted level (3D, K <= 3, FP32-stored G)
  cudaError_t (*def_apply_ff)(int dim, const double* x, double* y, const double* b, const float* G, int n, int cpb,
                              cudaStream_t s);
  int (*def_apply_candidates)(int dim, int prec, int gprec, int* out, int max);
  // grouped launches (Cartesian); the patch launch uses the patch-major layout
  // with ppc patches per block; dinv: the part's inverse-diagonal tables
  cudaError_t (*cart_apply_group)(int dim, int prec, int count, const ApplyJob* jobs, cudaStream_t s);
  cudaError_t (*cart_apply_ff_group)(int dim, int count, const ApplyJob* jobs, cudaStream_t s);
  cudaError_t (*patch_cart_group)(int dim, int prec, int count, const PatchSolveJob* jobs, int ppc, int n_iter,
                                  const void* dinv, int* counter, cudaStream_t s);
  cudaError_t (*patch_gather_group)(int dim, int prec, int count, const GatherSolveJob* jobs, int add,
                                    cudaStream_t s);
  cudaError_t (*h_prolong_add_group)(int dim, int prec, int count, const TransferSolveJob* jobs, cudaStream_t s);
  cudaError_t (*h_restrict_group)(int dim, int prec, int count, const TransferSolveJob* jobs, cudaStream_t s);
};

// nullptr when k, dim or prec is out of range
const KernelTable* kernel_table(int K, int dim, int prec);

}  // namespace pmg
