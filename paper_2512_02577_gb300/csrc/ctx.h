// The context of one hierarchy (pmg_ctx) and what the translation units of
// the library's host runtime share about it: error reporting, the per-level
// data, the workspace plan, the state of an incremental solve, and the
// helpers of pmg.cu that the grouped solves (group.cu) call.  Internal: not
// part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pmg.h"
#include "pmg_common.cuh"
#include "pmg_kernels_api.h"
#include "vec.h"

namespace pmg {
// records msg as the calling thread's last error; returns code
int fail(int code, const std::string& msg);
}  // namespace pmg

#define PMG_CUDA(call)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) return fail(PMG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

namespace pmg {

constexpr int kMaxCoarse = 4096;
constexpr int kNumSMs = 152;  // GB300
constexpr int64_t kAlign = 256;

enum Scal { S_RZ = 0, S_PAP = 1, S_RR = 2, S_RZN = 3, S_BB = 4, S_TMP = 5, S_COUNT = 16 };

struct LevelData {
  int n = 0, N1 = 0;
  int64_t N = 0;
  void *b = nullptr, *u = nullptr, *r = nullptr;  // MG precision
  double scale = 1.0;                             // h^{d-2}
  double inv_a0 = 0.0;                            // Cartesian 1 / A_{j,1}
  void* G[4] = {nullptr, nullptr, nullptr, nullptr};  // G_q per p-level (FP64 or FP32: geom_precision)
  void* dinv[4] = {nullptr, nullptr, nullptr, nullptr};
  void* dinv1 = nullptr;
};

// Byte layout of every device array of a context.
struct Plan {
  int dim = 3, K = 2, nlev = 1, nplev = 1, n0 = 1, mg_es = 8, g_es = 4;
  bool deformed = false, mg32 = false;
  std::vector<int> ns;
  int nc = 0;  // free DoFs on the coarsest level (0 if above the dense limit)
  bool coarse_ok = true;
  int64_t total = 0;
  // offsets
  struct LOff {
    int64_t b, u, r, G[4], dinv[4], dinv1;
  };
  std::vector<LOff> lo;
  int64_t t_mg[4], t64[4], cg[6], scal, partial, dtab64, dtab32, cidx, ainv, a64, gjrow, gjcol, gjbad, cx0, cy0;
  int64_t pbuf = -1, cellbuf = -1, counter = -1;
  int64_t verts = -1;  // distorted: positions of the finest mesh's vertices
  int64_t dtab_len = 0;
  // flexible GMRES (outer_solver GMRES): basis v_0..v_m, z_0..z_{m-1},
  // Hessenberg (m+1) x m, small state, multi-dot partials
  int m = 0;
  int64_t gv = -1, gz = -1, gh = -1, gs = -1, gpart = -1;
};

// Progress of an incremental solve (see solve_progress).
struct SolveState {
  int phase = 0;
  int it = 0, maxit = 0, status = 0;
  int gj = 0;  // GMRES: Arnoldi steps taken in the current cycle
  double rtol = 0, nb = 0, rel = 0, time_ms = 0;
  double* x_out = nullptr;
  bool x_host = false;
  const double* b_in = nullptr;  // grouped solves: the right-hand side, read at the first round
  bool b_host = false;
  int error = PMG_OK;            // grouped solves: a failure of this system's solve
};


// Phases of an incremental solve (see solve_progress).
enum SolvePhase { SP_IDLE = 0, SP_WAIT_BB = 1, SP_WAIT_RR = 2, SP_COPY_OUT = 3, SP_DONE = 4 };

struct SolveGroup;

}  // namespace pmg

struct pmg_ctx {
  pmg_config cfg{};
  pmg::Plan plan;
  int dim = 3, K = 2, L = 1, nplev = 1;
  bool deformed = false, mg32 = false;
  int mgprec = PMG_FP64;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  const pmg::KernelTable* kt[2] = {};  // kernel parts of (K, dim), by precision
  const pmg::KernelTable* km() const { return kt[mgprec]; }  // the multigrid precision's part
  std::vector<pmg::LevelData> lv;
  char* ws = nullptr;
  bool own_ws = false;
  void* t_mg[4] = {};
  double* t64[4] = {};
  double *cg_x = nullptr, *cg_r = nullptr, *cg_p = nullptr, *cg_Ap = nullptr, *cg_z = nullptr, *cg_b = nullptr;
  double* scal = nullptr;
  double* partial = nullptr;
  bool gmres = false;  // outer solver: flexible GMRES (else PCG)
  int gm = 0;          // GMRES restart length
  double *gv = nullptr, *gz = nullptr, *gh = nullptr, *gs = nullptr, *gpart = nullptr;
  int64_t gld = 0;     // stride of the GMRES basis columns
  double* host_scal = nullptr;  // pinned
  void* dtab_mg = nullptr;
  double* dtab64 = nullptr;
  float* dtab32 = nullptr;
  int* cidx = nullptr;
  void* ainv = nullptr;
  bool coarse_ready = false;
  void* pbuf = nullptr;
  void* cellbuf = nullptr;
  int* work_counter = nullptr;
  bool persistent = false;  // Cartesian patch launches as persistent grids (autotuned)
  double* verts = nullptr;  // distorted geometry: finest-mesh vertex positions
  int ppc = 1;          // patch-major layout: patches per block
  int il_threads = 0;   // > 0: interleaved layout (Cartesian), threads per block
  int def_cpb = 0;      // deformed apply: cells per block (0: the kernel part's rule)
  double omega_as = 0;
  double omega_j[4] = {1, 1, 1, 1};
  cudaGraphExec_t vgraph = nullptr;
  int64_t vgraph_launches = 0;
  cudaEvent_t ev_rr = nullptr, ev0 = nullptr, ev1 = nullptr, ev_done = nullptr;
  pmg::SolveState sv;
  pmg::SolveGroup* group = nullptr;  // the grouped solve this context is part of, if any
  uint64_t uid = 0;                   // unique over the process (a freed context's address may be reused)
};

namespace pmg {

// Smoother parameters of a level, the patch-major block shape the tuner's rule
// gives, the dense coarse level (set up on first use), a NULL check.
PatchParamsHost patch_params(const pmg_ctx* c, int level);
int rule_ppc(const pmg_ctx* c);
int ensure_coarse(pmg_ctx* c);
int check_ctx(const pmg_ctx* c);
// Advance an incremental solve (block: wait for device work); *state 1 when done.
int solve_progress(pmg_ctx* c, bool block, int* state);
void solve_info(const pmg_ctx* c, pmg_solve_info* info);

}  // namespace pmg
