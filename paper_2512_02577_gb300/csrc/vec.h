// Degree-independent device routines (vec.cu).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "pmg_common.cuh"

namespace pmg {

// Process-wide count of kernel launches enqueued by the library.
extern std::atomic<int64_t> g_launches;

constexpr int kDotBlocks = 304;  // fixed reduction grid: 2 x 152 SMs

// 1D tables passed by value to set-up kernels: nq points x[q], weights w[q],
// GLL basis values V[q*12 + a] and derivatives D[q*12 + a] at the points.
struct QuadTab {
  double x[12];
  double w[12];
  double V[12 * 12];
  double D[12 * 12];
  int nq;
};

cudaError_t dot(const double* x, const double* y, int64_t n, double* partial, double* out, cudaStream_t st);

// ---- grouped forms: one launch (or one per phase) for up to kMaxGroup jobs,
// each job's result bitwise that of its own call above (the reductions keep
// their fixed grid and summation order per job)
struct DotJob {
  const double* x;
  const double* y;
  int64_t n;
  double* partial;  // kDotBlocks doubles of the job's own scratch
  double* out;
};
struct CgXrJob {
  double* x;
  double* r;
  const double* p;
  const double* Ap;
  int64_t n;
  const double* s;
  int num, den;
  double* partial;
  double* rr_out;
};
struct CgPJob {
  double* p;
  const double* z;
  int64_t n;
  double* s;
  int num, den, first;
};
struct CopyJob {  // n elements from a to b
  const void* a;
  void* b;
  int64_t n;
};
struct ZeroJob {  // bytes: a multiple of 4
  void* p;
  int64_t bytes;
};
struct CoarseJob {  // as coarse_solve
  const void* Ainv;
  const int* idx;
  int nc;
  const void* b;
  void* u;
  int64_t N;
};
cudaError_t dot_group(int count, const DotJob* jobs, cudaStream_t st);
cudaError_t cg_update_xr_group(int count, const CgXrJob* jobs, cudaStream_t st);
cudaError_t cg_update_p_group(int count, const CgPJob* jobs, cudaStream_t st);
cudaError_t cast_d2f_group(int count, const CopyJob* jobs, cudaStream_t st);
cudaError_t cast_f2d_group(int count, const CopyJob* jobs, cudaStream_t st);
cudaError_t copy_group(int count, const CopyJob* jobs, int elem_bytes, cudaStream_t st);  // 4 or 8
cudaError_t zero_group(int count, const ZeroJob* jobs, cudaStream_t st);
cudaError_t coarse_solve_group(int prec, int count, const CoarseJob* jobs, cudaStream_t st);
cudaError_t cg_update_xr(double* x, double* r, const double* p, const double* Ap, int64_t n, const double* s,
                         int num, int den, double* partial, double* rr_out, cudaStream_t st);
cudaError_t cg_update_p(double* p, const double* z, int64_t n, double* s, int num, int den, int first,
                        cudaStream_t st);
// ---- flexible GMRES (outer solver for the half local V-cycle)
constexpr int kMaxKrylov = 64;  // largest restart length
// Offsets of the small GMRES state in its device array (restart length m).
struct GmresState {
  static constexpr int cs(int m) { return 0; }
  static constexpr int sn(int m) { return m; }
  static constexpr int g(int m) { return 2 * m; }            // m + 1 entries
  static constexpr int y(int m) { return 3 * m + 1; }        // m entries
  static constexpr int h2(int m) { return 4 * m + 1; }       // m + 1 entries
  static constexpr int inv(int m) { return 5 * m + 2; }
  static constexpr int est(int m) { return 5 * m + 3; }
  static constexpr int nrm2(int m) { return 5 * m + 4; }
  static constexpr int size(int m) { return 5 * m + 5; }
};
// out[i] = v_i . w for i < nv (v_i = V + i ld), deterministic two-pass;
// partial: nv * kDotBlocks doubles
cudaError_t multi_dot(const double* V, int64_t ld, int nv, const double* w, int64_t n, double* partial,
                      double* out, cudaStream_t st);
// w += sgn sum_{i < nv} c_i v_i  (c on the device)
cudaError_t multi_axpy(double* w, const double* V, int64_t ld, int nv, const double* c, double sgn, int64_t n,
                       cudaStream_t st);
// cycle start: beta = sqrt(*nrm2), g = beta e_1, v0 = r / beta
cudaError_t gmres_start(double* S, const double* nrm2, int m, const double* r, double* v0, int64_t n,
                        cudaStream_t st);
// Arnoldi step j after orthogonalisation: Givens update of H(:, j) and g,
// S[est] = |g_{j+1}|, then v = v / ||v|| (||v||^2 in *nrm2)
cudaError_t gmres_givens(double* H, double* S, const double* nrm2, int j, int m, double* v, int64_t n,
                         cudaStream_t st);
// x += Z y with y = R^{-1} g over the first k steps of the cycle
cudaError_t gmres_update(const double* H, double* S, int k, int m, const double* Z, int64_t ld, double* x, int64_t n,
                         cudaStream_t st);

cudaError_t cast_d2f(const double* a, float* b, int64_t n, cudaStream_t st);
cudaError_t cast_f2d(const float* a, double* b, int64_t n, cudaStream_t st);
cudaError_t coarse_solve(int prec, const void* Ainv, const int* idx, int nc, const void* b, void* u, int64_t N,
                         cudaStream_t st);
cudaError_t coarse_unit(double* x, int64_t N, int64_t pos, cudaStream_t st);
cudaError_t coarse_gather_row(const double* y, const int* idx, int nc, double* A, int row, cudaStream_t st);
// In-place inverse of the dense SPD matrix A (nc x nc, FP64) by Gauss-Jordan
// sweeps, stored into `out` in precision prec; *bad = 1 if a pivot is not
// positive.  row, col: nc scratch each.
cudaError_t coarse_invert(double* A, int nc, double* row, double* col, int* bad, void* out, int prec,
                          cudaStream_t st);
// Geometry of a level: kind 0 Cartesian, 1 the analytic deformation with
// amplitude amp, 2 trilinear cells spanned by displaced vertices (verts:
// device array of the finest mesh's (n_fine + 1)^d vertex positions, dim
// doubles each, x fastest; a level with n cells takes every (n_fine / n)-th).
struct GeomDesc {
  int kind;
  double amp;
  const double* verts;
  int n_fine;
};
// G_q of every cell at the (p+1)^d Gauss points, stored in FP64 (gprec 0)
// or FP32 (gprec 1); *bad |= 1 where a cell's det J <= 0 at a quadrature
// point (inverted cell)
cudaError_t compute_geometry(int dim, int n, int p, const GeomDesc& geo, const QuadTab& tab, void* G, int gprec,
                             int* bad, cudaStream_t st);
cudaError_t compute_inverse_diagonal(int dim, int n, int p, const QuadTab& tab, const void* G, int gprec,
                                     double* diag_tmp, void* inv, int prec, cudaStream_t st);
cudaError_t rhs_manufactured(int dim, int n, int K, const GeomDesc& geo, const QuadTab& tab, double* b,
                             cudaStream_t st);
cudaError_t l2_error_partials(int dim, int n, int K, const GeomDesc& geo, const QuadTab& tab, const double* x,
                              double* partial, double* out, cudaStream_t st);

}  // namespace pmg
