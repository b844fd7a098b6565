// Grouped solves: several contexts' PCG solves advanced in lockstep, every
// launch of a round covering all of them (group.h; pmg_solve_group in the C
// ABI).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/pmg.h"
#include "ctx.h"
#include "group.h"
#include "pmg_common.cuh"
#include "pmg_kernels_api.h"
#include "vec.h"

using namespace pmg;

// Systems of the same dimension, degree and method -- MG precision,
// smoother, local cycles, smoothing steps, outer operator; Cartesian
// geometry, PCG -- on meshes of any size, solved in lockstep: each round
// launches the outer operator, the dot products and vector updates and
// every launch of the V-cycle once for all of them (grouped launches over
// per-system job tables).  V-cycles of systems with different numbers of
// levels are aligned at the finest level: descent step j smooths, forms the
// residual and restricts on level L_m - 1 - j of every system m that has
// such a level above the coarsest; the coarse solves of all systems follow
// the last descent step; the ascent mirrors the descent.  Every launch
// gives each system the arithmetic of its own pmg_solve (the same per-node
// operations; reductions with the same per-system grid and order), so each
// result is bitwise that of the system solved alone.  Systems join at the
// start of a round and leave when converged (continuous batching): a round
// enqueues the iteration of every running system and the first steps of
// every joining one, and the host reads the residual norms of the round
// while the round's preconditioner steps are still running, as pmg_solve
// does.
namespace pmg {

struct SolveGroup {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t ev = nullptr;   // after the residual norms of the last round reached the host
  bool pending = false;       // a round is enqueued and ev not yet seen
  int* counter = nullptr;     // work counter of the persistent patch launches
  std::vector<pmg_ctx*> members;  // running
  std::vector<pmg_ctx*> joining;  // start at the next round
  // The preconditioner step of a round as a CUDA graph, for the member list
  // it was captured for; captured once a member list has been seen in two
  // consecutive rounds (continuous joins and departures change it often)
  std::vector<uint64_t> last_all;   // context uids
  std::vector<uint64_t> graph_all;
  cudaGraphExec_t graph = nullptr;
  int64_t graph_launches = 0;
};

namespace {

struct GSel {
  pmg_ctx* c;
  int l;  // level of c in this launch
};

bool group_key_equal(const pmg_ctx* a, const pmg_ctx* b) {
  return a->dim == b->dim && a->K == b->K && a->mgprec == b->mgprec && a->cfg.smoother == b->cfg.smoother &&
         a->cfg.local_cycles == b->cfg.local_cycles && a->cfg.local_half == b->cfg.local_half &&
         a->cfg.smooth_steps == b->cfg.smooth_steps && a->cfg.outer_apply == b->cfg.outer_apply;
}

bool groupable(const pmg_ctx* c) { return !c->deformed && !c->gmres && c->plan.coarse_ok; }

int gcheck(cudaError_t e, const char* what) {
  return e == cudaSuccess ? PMG_OK : fail(PMG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// y = A x or y = b - A x on level l of every system, dispatched as level_apply
int g_apply(const std::vector<GSel>& S, int prec, void* const* x, void* const* y, void* const* b, cudaStream_t st) {
  ApplyJob J[kMaxGroup];
  const pmg_ctx* c0 = S[0].c;
  const bool ff = prec == PMG_FP64 && c0->cfg.outer_apply == PMG_OUTER_APPLY_FLOAT_FLOAT;
  for (size_t i = 0; i < S.size(); ++i) {
    pmg_ctx* c = S[i].c;
    const LevelData& L = c->lv[S[i].l];
    J[i].x = x[i];
    J[i].y = y[i];
    J[i].b = b ? b[i] : nullptr;
    for (int t = 0; t < 4; ++t) J[i].t[t] = (ff || prec == PMG_FP64) ? (void*)c->t64[t] : c->t_mg[t];
    J[i].n = L.n;
    J[i].scale = L.scale;
  }
  const int cnt = (int)S.size();
  if (ff) return gcheck(c0->kt[PMG_FP64]->cart_apply_ff_group(c0->dim, cnt, J, st), "grouped apply");
  return gcheck(c0->kt[prec]->cart_apply_group(c0->dim, prec, cnt, J, st), "grouped apply");
}

// r = b - A u in the MG precision on every selected level
int g_residual(const std::vector<GSel>& S, cudaStream_t st) {
  void *x[kMaxGroup], *y[kMaxGroup], *b[kMaxGroup];
  for (size_t i = 0; i < S.size(); ++i) {
    LevelData& L = S[i].c->lv[S[i].l];
    x[i] = L.u;
    y[i] = L.r;
    b[i] = L.b;
  }
  return g_apply(S, S[0].c->mgprec, x, y, b, st);
}

// patch solves of every selected level for residuals r: additive output to
// the patch buffer (colour < 0), or added to u for the patches of one colour
int g_patch_solves(const std::vector<GSel>& S, void* const* r, int colour, int* counter, cudaStream_t st) {
  PatchSolveJob J[kMaxGroup];
  for (size_t i = 0; i < S.size(); ++i) {
    pmg_ctx* c = S[i].c;
    LevelData& L = c->lv[S[i].l];
    J[i].r = r[i];
    J[i].dst = colour < 0 ? c->pbuf : L.u;
    J[i].n = L.n;
    J[i].P = patch_params(c, S[i].l);
    J[i].P.colour = colour;
  }
  pmg_ctx* c0 = S[0].c;
  return gcheck(c0->km()->patch_cart_group(c0->dim, c0->mgprec, (int)S.size(), J, rule_ppc(c0),
                                           c0->cfg.local_cycles, c0->dtab_mg, counter, st),
                "grouped patch smoother");
}

int g_patch_sweep(const std::vector<GSel>& S, bool from_b, bool add, int* counter, cudaStream_t st) {
  void* r[kMaxGroup];
  GatherSolveJob G[kMaxGroup];
  for (size_t i = 0; i < S.size(); ++i) {
    LevelData& L = S[i].c->lv[S[i].l];
    r[i] = from_b ? L.b : L.r;
    G[i] = GatherSolveJob{S[i].c->pbuf, L.u, L.n};
  }
  if (int rc = g_patch_solves(S, r, -1, counter, st)) return rc;
  pmg_ctx* c0 = S[0].c;
  return gcheck(c0->km()->patch_gather_group(c0->dim, c0->mgprec, (int)S.size(), G, add ? 1 : 0, st),
                "grouped patch gather");
}

// mult_sweep for every selected level
int g_mult_sweep(const std::vector<GSel>& S, bool forward, bool zero_guess, int* counter, cudaStream_t st) {
  pmg_ctx* c0 = S[0].c;
  const int nc = 1 << c0->dim;
  const int64_t es = c0->mg32 ? 4 : 8;
  if (zero_guess) {
    ZeroJob Z[kMaxGroup];
    for (size_t i = 0; i < S.size(); ++i) {
      LevelData& L = S[i].c->lv[S[i].l];
      Z[i] = ZeroJob{L.u, es * L.N};
    }
    if (int rc = gcheck(zero_group((int)S.size(), Z, st), "grouped zero")) return rc;
  }
  void* r[kMaxGroup];
  for (int k = 0; k < nc; ++k) {
    const int colour = forward ? k : nc - 1 - k;
    const bool first = zero_guess && k == 0;
    if (!first)
      if (int rc = g_residual(S, st)) return rc;
    for (size_t i = 0; i < S.size(); ++i) {
      LevelData& L = S[i].c->lv[S[i].l];
      r[i] = first ? L.b : L.r;
    }
    if (int rc = g_patch_solves(S, r, colour, counter, st)) return rc;
  }
  return PMG_OK;
}

int g_smooth(const std::vector<GSel>& S, int sweeps, bool forward, int* counter, cudaStream_t st) {
  const bool mult = S[0].c->cfg.smoother == PMG_SMOOTHER_MULTIPLICATIVE;
  for (int s = 0; s < sweeps; ++s) {
    if (mult) {
      if (int rc = g_mult_sweep(S, forward, false, counter, st)) return rc;
    } else {
      if (int rc = g_residual(S, st)) return rc;
      if (int rc = g_patch_sweep(S, false, true, counter, st)) return rc;
    }
  }
  return PMG_OK;
}

// the systems that have a level L - 1 - j above the coarsest
std::vector<GSel> g_depth(const std::vector<pmg_ctx*>& M, int j) {
  std::vector<GSel> S;
  for (pmg_ctx* c : M)
    if (c->L - 1 - j >= 1) S.push_back(GSel{c, c->L - 1 - j});
  return S;
}

// z_m = B_m b_m from a zero guess for every system, vectors in the finest
// level buffers (vcycle_level, level by level for all systems at once)
int g_vcycle(const std::vector<pmg_ctx*>& M, int* counter, cudaStream_t st) {
  int D = 0;
  for (pmg_ctx* c : M) D = std::max(D, c->L - 1);
  const int nu = M[0]->cfg.smooth_steps;
  const bool mult = M[0]->cfg.smoother == PMG_SMOOTHER_MULTIPLICATIVE;
  pmg_ctx* c0 = M[0];
  for (int j = 0; j < D; ++j) {
    const std::vector<GSel> S = g_depth(M, j);
    for (int s = 0; s < nu; ++s) {
      int rc;
      if (mult) rc = g_mult_sweep(S, true, s == 0, counter, st);
      else if (s == 0) rc = g_patch_sweep(S, true, false, counter, st);
      else rc = g_smooth(S, 1, true, counter, st);
      if (rc) return rc;
    }
    if (int rc = g_residual(S, st)) return rc;
    TransferSolveJob T[kMaxGroup];
    for (size_t i = 0; i < S.size(); ++i) {
      pmg_ctx* c = S[i].c;
      LevelData &L = c->lv[S[i].l], &C = c->lv[S[i].l - 1];
      T[i] = TransferSolveJob{L.r, C.b, c->t_mg[0], c->t_mg[1], C.n};
    }
    if (int rc = gcheck(c0->km()->h_restrict_group(c0->dim, c0->mgprec, (int)S.size(), T, st), "grouped restrict"))
      return rc;
  }
  CoarseJob CJ[kMaxGroup];
  for (size_t i = 0; i < M.size(); ++i) {
    pmg_ctx* c = M[i];
    LevelData& C = c->lv[0];
    CJ[i] = CoarseJob{c->ainv, c->cidx, c->plan.nc, C.b, C.u, C.N};
  }
  if (int rc = gcheck(coarse_solve_group(c0->mgprec, (int)M.size(), CJ, st), "grouped coarse solve")) return rc;
  for (int j = D - 1; j >= 0; --j) {
    const std::vector<GSel> S = g_depth(M, j);
    TransferSolveJob T[kMaxGroup];
    for (size_t i = 0; i < S.size(); ++i) {
      pmg_ctx* c = S[i].c;
      LevelData &L = c->lv[S[i].l], &C = c->lv[S[i].l - 1];
      T[i] = TransferSolveJob{C.u, L.u, c->t_mg[0], c->t_mg[1], C.n};
    }
    if (int rc = gcheck(c0->km()->h_prolong_add_group(c0->dim, c0->mgprec, (int)S.size(), T, st), "grouped prolong"))
      return rc;
    if (int rc = g_smooth(S, nu, false, counter, st)) return rc;
  }
  return PMG_OK;
}

// z = B r for every system (FP64 finest-level vectors), as precondition
int g_precondition(const std::vector<pmg_ctx*>& M, int* counter, cudaStream_t st) {
  CopyJob J[kMaxGroup];
  const bool mg32 = M[0]->mg32;
  for (size_t i = 0; i < M.size(); ++i) {
    LevelData& F = M[i]->lv[M[i]->L - 1];
    J[i] = CopyJob{M[i]->cg_r, F.b, F.N};
  }
  const int cnt = (int)M.size();
  if (int rc = gcheck(mg32 ? cast_d2f_group(cnt, J, st) : copy_group(cnt, J, 8, st), "grouped cast")) return rc;
  if (int rc = g_vcycle(M, counter, st)) return rc;
  for (size_t i = 0; i < M.size(); ++i) {
    LevelData& F = M[i]->lv[M[i]->L - 1];
    J[i] = CopyJob{F.u, M[i]->cg_z, F.N};
  }
  return gcheck(mg32 ? cast_f2d_group(cnt, J, st) : copy_group(cnt, J, 8, st), "grouped cast");
}

// g_precondition for the member list `all`, replayed from the group's graph
// when the list is the one it was captured for, captured (updating the
// instantiated graph in place when the launch sequence has the same shape)
// when the same list ran the previous round, else launched directly.
int g_precondition_round(SolveGroup* G, const std::vector<pmg_ctx*>& all) {
  cudaStream_t st = G->stream;
  std::vector<uint64_t> ids;
  for (const pmg_ctx* c : all) ids.push_back(c->uid);
  if (G->graph && G->graph_all == ids) {
    PMG_CUDA(cudaGraphLaunch(G->graph, st));
    g_launches += G->graph_launches;
    return PMG_OK;
  }
  const bool repeat = G->last_all == ids;
  G->last_all = ids;
  if (!repeat) return g_precondition(all, G->counter, st);
  cudaGraph_t g = nullptr;
  const int64_t before = g_launches.load();
  PMG_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  const int rc = g_precondition(all, G->counter, st);
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  const int64_t n = g_launches.load() - before;
  g_launches -= n;  // captured, not launched
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(PMG_ERR_CUDA, std::string("group graph capture: ") + cudaGetErrorString(e));
  bool updated = false;
  if (G->graph) {
    cudaGraphExecUpdateResultInfo info;
    updated = cudaGraphExecUpdate(G->graph, g, &info) == cudaSuccess;
    if (!updated) {
      cudaGetLastError();
      cudaGraphExecDestroy(G->graph);
      G->graph = nullptr;
    }
  }
  cudaError_t ie = cudaSuccess;
  if (!updated) ie = cudaGraphInstantiate(&G->graph, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    G->graph = nullptr;
    return fail(PMG_ERR_CUDA, std::string("group graph instantiate: ") + cudaGetErrorString(ie));
  }
  G->graph_all = ids;
  G->graph_launches = n;
  PMG_CUDA(cudaGraphLaunch(G->graph, st));
  g_launches += n;
  return PMG_OK;
}

// solve_finish on the group's stream; the context leaves the group and its
// own stream waits for the copy of its solution
int g_finish(SolveGroup* G, pmg_ctx* c, int status, int error) {
  c->sv.status = status;
  c->sv.error = error;
  const int64_t N = c->lv[c->L - 1].N;
  PMG_CUDA(cudaEventRecord(c->ev1, G->stream));
  if (c->sv.x_out)
    PMG_CUDA(cudaMemcpyAsync(c->sv.x_out, c->cg_x, 8 * N, c->sv.x_host ? cudaMemcpyDeviceToHost
                                                                        : cudaMemcpyDeviceToDevice, G->stream));
  PMG_CUDA(cudaEventRecord(c->ev_done, G->stream));
  PMG_CUDA(cudaStreamWaitEvent(c->stream, c->ev_done, 0));
  c->sv.phase = SP_COPY_OUT;
  c->group = nullptr;
  return PMG_OK;
}

// One round: decide every running system from its residual norm, start the
// joining ones, enqueue the iteration of the rest.
int g_round(SolveGroup* G) {
  cudaStream_t st = G->stream;
  std::vector<pmg_ctx*> cont;
  for (pmg_ctx* c : G->members) {
    SolveState& v = c->sv;
    bool fin = false;
    int status = PMG_OK, error = PMG_OK;
    if (v.phase == SP_WAIT_BB) {
      v.nb = std::sqrt(c->host_scal[S_BB]);
      if (!(v.nb > 0)) {
        v.rel = 0.0;
        fin = true;
      } else {
        v.rel = 1.0;
      }
    } else {
      v.rel = std::sqrt(std::max(c->host_scal[S_RR], 0.0)) / v.nb;
      if (!(v.rel == v.rel)) {
        fin = true;
        error = fail(PMG_ERR_STATE, "solver breakdown (NaN residual)");
      } else if (v.rel <= v.rtol) {
        fin = true;
      }
    }
    if (!fin && v.it >= v.maxit) {
      fin = true;
      status = PMG_NOT_CONVERGED;
    }
    if (fin) {
      if (int rc = g_finish(G, c, status, error)) return rc;
    } else {
      cont.push_back(c);
    }
  }
  std::vector<pmg_ctx*> join = G->joining;
  G->joining.clear();
  // first steps of the joining systems (solve_start)
  DotJob D[kMaxGroup];
  for (size_t i = 0; i < join.size(); ++i) {
    pmg_ctx* c = join[i];
    const int64_t N = c->lv[c->L - 1].N;
    PMG_CUDA(cudaEventRecord(c->ev0, st));
    PMG_CUDA(cudaMemcpyAsync(c->cg_r, c->sv.b_in, 8 * N,
                             c->sv.b_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st));
    PMG_CUDA(cudaMemsetAsync(c->cg_x, 0, 8 * N, st));
    D[i] = DotJob{c->cg_r, c->cg_r, N, c->partial, c->scal + S_BB};
  }
  if (!join.empty()) {
    if (int rc = gcheck(dot_group((int)join.size(), D, st), "grouped dot")) return rc;
    for (pmg_ctx* c : join)
      PMG_CUDA(cudaMemcpyAsync(c->host_scal + S_BB, c->scal + S_BB, 8, cudaMemcpyDeviceToHost, st));
  }
  // first half of the iteration of the running systems (enqueue_iteration)
  if (!cont.empty()) {
    std::vector<GSel> S;
    void *x[kMaxGroup], *y[kMaxGroup];
    CgXrJob X[kMaxGroup];
    for (size_t i = 0; i < cont.size(); ++i) {
      pmg_ctx* c = cont[i];
      const int64_t N = c->lv[c->L - 1].N;
      S.push_back(GSel{c, c->L - 1});
      x[i] = c->cg_p;
      y[i] = c->cg_Ap;
      D[i] = DotJob{c->cg_p, c->cg_Ap, N, c->partial, c->scal + S_PAP};
      X[i] = CgXrJob{c->cg_x, c->cg_r, c->cg_p, c->cg_Ap, N, c->scal, S_RZ, S_PAP, c->partial, c->scal + S_RR};
    }
    const int cnt = (int)cont.size();
    if (int rc = g_apply(S, PMG_FP64, x, y, nullptr, st)) return rc;
    if (int rc = gcheck(dot_group(cnt, D, st), "grouped dot")) return rc;
    if (int rc = gcheck(cg_update_xr_group(cnt, X, st), "grouped update")) return rc;
    for (pmg_ctx* c : cont) {
      PMG_CUDA(cudaMemcpyAsync(c->host_scal + S_RR, c->scal + S_RR, 8, cudaMemcpyDeviceToHost, st));
      ++c->sv.it;
    }
  }
  std::vector<pmg_ctx*> all = cont;
  all.insert(all.end(), join.begin(), join.end());
  G->members = all;
  if (all.empty()) {
    G->pending = false;
    return PMG_OK;
  }
  PMG_CUDA(cudaEventRecord(G->ev, st));
  G->pending = true;
  // second half: z = B r, r.z and the new direction (p = z for joining systems)
  if (int rc = g_precondition_round(G, all)) return rc;
  for (size_t i = 0; i < all.size(); ++i) {
    pmg_ctx* c = all[i];
    const bool joined = i >= cont.size();
    D[i] = DotJob{c->cg_r, c->cg_z, c->lv[c->L - 1].N, c->partial, c->scal + (joined ? S_RZ : S_RZN)};
  }
  if (int rc = gcheck(dot_group((int)all.size(), D, st), "grouped dot")) return rc;
  if (!cont.empty()) {
    CgPJob P[kMaxGroup];
    for (size_t i = 0; i < cont.size(); ++i) {
      pmg_ctx* c = cont[i];
      P[i] = CgPJob{c->cg_p, c->cg_z, c->lv[c->L - 1].N, c->scal, S_RZN, S_RZ, 0};
    }
    if (int rc = gcheck(cg_update_p_group((int)cont.size(), P, st), "grouped update")) return rc;
  }
  if (!join.empty()) {
    CopyJob C[kMaxGroup];
    for (size_t i = 0; i < join.size(); ++i) C[i] = CopyJob{join[i]->cg_z, join[i]->cg_p, join[i]->lv[join[i]->L - 1].N};
    if (int rc = gcheck(copy_group((int)join.size(), C, 8, st), "grouped copy")) return rc;
  }
  for (pmg_ctx* c : cont) c->sv.phase = SP_WAIT_RR;
  for (pmg_ctx* c : join) c->sv.phase = SP_WAIT_BB;
  return PMG_OK;
}

// every system of the group ends with `error` (a failed launch); each is
// copied out so that its context becomes usable again
void g_abort(SolveGroup* G, int error) {
  std::vector<pmg_ctx*> all = G->members;
  all.insert(all.end(), G->joining.begin(), G->joining.end());
  G->members.clear();
  G->joining.clear();
  for (pmg_ctx* c : all) {
    c->sv.x_out = nullptr;  // its contents are not a solution
    if (g_finish(G, c, PMG_OK, error) != PMG_OK) {
      c->group = nullptr;
      c->sv.phase = SP_DONE;
      c->sv.status = error;
    }
  }
  G->pending = false;
}

}  // namespace

int group_create(cudaStream_t stream, SolveGroup** out) {
  *out = nullptr;
  SolveGroup* G = new SolveGroup();
  cudaError_t e = cudaSuccess;
  if (stream) {
    G->stream = stream;
  } else {
    e = cudaStreamCreateWithFlags(&G->stream, cudaStreamNonBlocking);
    G->own_stream = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&G->ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&G->counter, 16);
  if (e != cudaSuccess) {
    if (G->ev) cudaEventDestroy(G->ev);
    if (G->own_stream) cudaStreamDestroy(G->stream);
    delete G;
    return fail(PMG_ERR_CUDA, std::string("group: ") + cudaGetErrorString(e));
  }
  *out = G;
  return PMG_OK;
}

int group_destroy(SolveGroup* G) {
  if (!G) return PMG_OK;
  if (!G->members.empty() || !G->joining.empty()) return fail(PMG_ERR_STATE, "the group has running systems");
  cudaStreamSynchronize(G->stream);
  if (G->graph) cudaGraphExecDestroy(G->graph);
  cudaFree(G->counter);
  cudaEventDestroy(G->ev);
  if (G->own_stream) cudaStreamDestroy(G->stream);
  delete G;
  return PMG_OK;
}

int group_size(const SolveGroup* G) { return (int)(G->members.size() + G->joining.size()); }

int group_cancel(SolveGroup* G) {
  g_abort(G, fail(PMG_ERR_STATE, "grouped solve cancelled"));
  const cudaError_t e = cudaStreamSynchronize(G->stream);
  return e == cudaSuccess ? PMG_OK : fail(PMG_ERR_CUDA, std::string("group: ") + cudaGetErrorString(e));
}

bool group_accepts(const SolveGroup* G, const pmg_ctx* c) {
  if (!groupable(c) || c->group || group_size(G) >= kMaxGroup) return false;
  const pmg_ctx* ref = !G->members.empty() ? G->members[0] : (!G->joining.empty() ? G->joining[0] : nullptr);
  return !ref || group_key_equal(ref, c);
}

int group_join(SolveGroup* G, pmg_ctx* c, const double* b, bool b_host, double* x, bool x_host, double rtol,
               int maxit) {
  if (!G || check_ctx(c) || !b) return fail(PMG_ERR_ARG, "NULL argument");
  if (maxit < 0 || !(rtol >= 0)) return fail(PMG_ERR_ARG, "bad rtol / maxit");
  if (c->group || (c->sv.phase != SP_IDLE && c->sv.phase != SP_DONE))
    return fail(PMG_ERR_STATE, "a solve is already in progress");
  if (!groupable(c))
    return fail(PMG_ERR_UNSUPPORTED, "grouped solves need a Cartesian mesh, PCG and a coarse level of <= 4096 DoFs");
  if (!group_accepts(G, c)) return fail(PMG_ERR_ARG, "the system's method differs from the group's, or it is full");
  if (int rc = ensure_coarse(c)) return rc;
  // the group's launches follow everything enqueued on the context so far
  PMG_CUDA(cudaEventRecord(c->ev0, c->stream));
  PMG_CUDA(cudaStreamWaitEvent(G->stream, c->ev0, 0));
  c->sv = SolveState();
  c->sv.rtol = rtol;
  c->sv.maxit = maxit;
  c->sv.b_in = b;
  c->sv.b_host = b_host;
  c->sv.x_out = x;
  c->sv.x_host = x_host;
  c->sv.phase = SP_WAIT_BB;
  c->group = G;
  G->joining.push_back(c);
  return PMG_OK;
}

// Advance the group as far as completed device work allows (block: wait
// for the round in flight).  Systems that finished have left the group;
// pmg_solve_progress on their contexts completes them.
int group_progress(SolveGroup* G, bool block) {
  if (G->pending) {
    if (block) {
      const cudaError_t e = cudaEventSynchronize(G->ev);
      if (e != cudaSuccess) {
        g_abort(G, PMG_ERR_CUDA);
        return fail(PMG_ERR_CUDA, std::string("group: ") + cudaGetErrorString(e));
      }
    } else {
      const cudaError_t q = cudaEventQuery(G->ev);
      if (q == cudaErrorNotReady) return PMG_OK;
      if (q != cudaSuccess) {
        g_abort(G, PMG_ERR_CUDA);
        return fail(PMG_ERR_CUDA, std::string("group: ") + cudaGetErrorString(q));
      }
    }
    G->pending = false;
  }
  if (G->members.empty() && G->joining.empty()) return PMG_OK;
  const int rc = g_round(G);
  if (rc != PMG_OK) g_abort(G, rc);
  return rc;
}

}  // namespace pmg

extern "C" {

int pmg_solve_group(pmg_ctx* const* ctxs, int count, const double* const* b, double* const* x, double rtol,
                    int maxit, pmg_solve_info* info) {
  if (!ctxs || !b || !x || count < 1) return fail(PMG_ERR_ARG, "NULL argument or count < 1");
  if (count > kMaxGroup) return fail(PMG_ERR_ARG, "more systems than one group holds");
  for (int i = 0; i < count; ++i) {
    if (check_ctx(ctxs[i]) || !b[i] || !x[i]) return fail(PMG_ERR_ARG, "NULL argument");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(PMG_ERR_ARG, "a context appears twice");
  }
  SolveGroup* G = nullptr;
  if (int rc = group_create(ctxs[0]->stream, &G)) return rc;
  int first_err = PMG_OK;
  int joined = 0;
  for (; joined < count; ++joined) {
    const int rc = group_join(G, ctxs[joined], b[joined], false, x[joined], false, rtol, maxit);
    if (rc != PMG_OK) {
      first_err = rc;
      break;
    }
  }
  if (first_err != PMG_OK) {
    for (int i = 0; i < joined; ++i) {  // nothing was enqueued for them yet
      ctxs[i]->group = nullptr;
      ctxs[i]->sv.phase = SP_IDLE;
    }
    G->joining.clear();
    group_destroy(G);
    return first_err;
  }
  while (group_size(G) > 0) {
    if (int rc = group_progress(G, true)) {
      first_err = rc;
      break;
    }
  }
  int status = first_err;
  for (int i = 0; i < count; ++i) {
    pmg_ctx* c = ctxs[i];
    int state = 0;
    int rc = c->sv.phase == SP_IDLE ? PMG_OK : solve_progress(c, true, &state);
    if (rc == PMG_OK && state) rc = c->sv.status;
    if (info) solve_info(c, info + i);
    c->sv.phase = SP_IDLE;
    if (status == PMG_OK || (status == PMG_NOT_CONVERGED && rc < 0)) status = rc;
  }
  group_destroy(G);
  return status;
}

}  // extern "C"
