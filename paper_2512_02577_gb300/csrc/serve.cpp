// Serving loop: many Poisson solves of different sizes and degrees resident
// on one GPU at once.
//
// A request (config, host right-hand side, host solution buffer) is queued
// by pmg_server_submit.  pmg_server_poll, which never blocks, (1) admits
// queued requests in arrival order while a slot is free and the request's
// context fits in the device-memory budget -- reusing an idle resident
// context built from the same configuration when one exists (key_of),
// evicting least-recently-used idle contexts otherwise -- (2)
// advances every running solve as far as its completed device work allows
// (pmg_solve_progress: each CG iteration enqueues its V-cycle, captured as a
// CUDA graph, before the host reads the residual), and (3) retires solves
// whose solution has reached the host.  Each slot has its own CUDA stream,
// so kernels of different requests overlap on the device, and a request that
// arrives while others run starts as soon as a slot and memory free up.
// With grouping on (pmg_server_set_grouping), small requests of one method
// instead join a group (group.h): their solves advance in lockstep with
// every launch of a round covering all members, members joining and leaving
// between rounds, so many small solves share each launch instead of each
// filling a fraction of the GPU with launches of its own.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <cstdint>
#include <deque>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/pmg.h"
#include "group.h"

namespace pmg {
void set_last_error(const std::string& msg);
}

namespace {

int fail(int code, const std::string& msg) {
  pmg::set_last_error(msg);
  return code;
}

// A resident context is reused only for a request whose configuration would
// build the same operator and preconditioner: every pmg_config field that
// pmg_create reads, with the damping as given (<= 0 means "default", so all
// non-positive values are one key), the deformation amplitude when the
// geometry uses it, and for a distorted mesh the displacement CONTENTS
// (copied at submit; compared by a 64-bit FNV-1a hash and then exactly).
struct Key {
  int dim = 0, n_cells = 0, degree = 0, mg_precision = 0, geometry = 0, n_levels = 0, local_cycles = 0,
      smooth_steps = 0, local_half = 0, outer_solver = 0, gmres_restart = 0, smoother = 0, patches_per_block = 0,
      patch_layout = 0, patch_threads = 0, outer_apply = 0, geom_precision = 0, apply_cpb = 0, persistent = 0,
      coarse_dofs = 0;
  double deform_amp = 0, omega_patch = 0, omega_jacobi[4] = {0, 0, 0, 0};
  uint64_t disp_hash = 0;
  const std::vector<double>* disp = nullptr;  // the request's own copy (distorted only)

  bool operator==(const Key& o) const {
    if (std::tie(dim, n_cells, degree, mg_precision, geometry, n_levels, local_cycles, smooth_steps, local_half,
                 outer_solver, gmres_restart, smoother, patches_per_block, patch_layout, patch_threads, outer_apply,
                 geom_precision, apply_cpb, persistent, coarse_dofs, deform_amp, omega_patch, disp_hash) !=
        std::tie(o.dim, o.n_cells, o.degree, o.mg_precision, o.geometry, o.n_levels, o.local_cycles,
                 o.smooth_steps, o.local_half, o.outer_solver, o.gmres_restart, o.smoother, o.patches_per_block,
                 o.patch_layout, o.patch_threads, o.outer_apply, o.geom_precision, o.apply_cpb, o.persistent,
                 o.coarse_dofs, o.deform_amp, o.omega_patch, o.disp_hash))
      return false;
    for (int i = 0; i < 4; ++i)
      if (omega_jacobi[i] != o.omega_jacobi[i]) return false;
    if ((disp == nullptr) != (o.disp == nullptr)) return false;
    return !disp || *disp == *o.disp;
  }
};

uint64_t fnv1a(const std::vector<double>& v) {
  uint64_t h = 1469598103934665603ull;
  const unsigned char* p = reinterpret_cast<const unsigned char*>(v.data());
  for (size_t i = 0; i < v.size() * sizeof(double); ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

// disp: the request's copy of the displacements (distorted geometry), else null
Key key_of(const pmg_config& c, const std::vector<double>* disp) {
  Key k;
  k.dim = c.dim;
  k.n_cells = c.n_cells;
  k.degree = c.degree;
  k.mg_precision = c.mg_precision;
  k.geometry = c.geometry;
  k.n_levels = c.n_levels;
  k.local_cycles = c.local_cycles;
  k.smooth_steps = c.smooth_steps;
  k.local_half = c.local_half;
  k.outer_solver = c.outer_solver;
  k.gmres_restart = c.outer_solver == PMG_OUTER_GMRES ? c.gmres_restart : 0;
  k.smoother = c.smoother;
  k.patches_per_block = c.patches_per_block;
  k.patch_layout = c.patch_layout;
  k.patch_threads = c.patch_threads;
  k.outer_apply = c.outer_apply;
  k.geom_precision = c.geometry == PMG_GEOM_CARTESIAN ? 0 : c.geom_precision;
  k.apply_cpb = c.geometry == PMG_GEOM_CARTESIAN ? 0 : c.apply_cells_per_block;
  k.persistent = c.patch_persistent;
  k.coarse_dofs = c.n_levels > 0 ? 0 : c.coarse_dofs;
  k.deform_amp = c.geometry == PMG_GEOM_DEFORMED ? c.deform_amp : 0.0;
  k.omega_patch = c.omega_patch > 0 ? c.omega_patch : 0.0;
  for (int i = 0; i < 4; ++i) k.omega_jacobi[i] = c.omega_jacobi[i] > 0 ? c.omega_jacobi[i] : 0.0;
  if (c.geometry == PMG_GEOM_DISTORTED && disp) {
    k.disp = disp;
    k.disp_hash = fnv1a(*disp);
  }
  return k;
}

struct Slot {
  pmg_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  Key key;
  std::vector<double> disp;  // the displacements the context was built from (distorted geometry)
  int64_t bytes = 0;
  bool busy = false;
  int64_t last_used = 0;
};

struct Request {
  int64_t id = 0;
  double work = 0;  // estimated cost of the solve (admission order, stream priority)
  pmg_config cfg{};
  std::vector<double> disp;  // copy of cfg.vertex_disp taken at submit (distorted geometry)
  const double* b = nullptr;
  double* x = nullptr;
  double rtol = 1e-8;
  int maxit = 500;
  int64_t bytes = 0;
  int state = 0;  // 0 queued, 1 running, 2 done, 3 failed
  int status = 0;
  double t_submit = 0, t_start = 0, t_done = 0;
  pmg_solve_info info{};
  Slot* slot = nullptr;
};

double now_s() {
  using clk = std::chrono::steady_clock;
  static const clk::time_point t0 = clk::now();
  return std::chrono::duration<double>(clk::now() - t0).count();
}

}  // namespace

struct pmg_server {
  int64_t budget = 0;
  int max_active = 8;
  int policy = PMG_SERVE_FIFO;
  double max_wait_s = 2.0;      // shortest-first: a request queued this long goes first
  double small_work = 0;        // requests below this estimated work get high-priority streams
  int prio_low = 0, prio_high = 0;
  int64_t used = 0;
  int64_t tick = 0;
  int64_t next_id = 1;
  std::deque<Request*> queue;
  std::vector<Request*> running;
  std::map<int64_t, Request*> requests;
  std::vector<Slot*> slots;
  int64_t created_contexts = 0;
  // grouped launches across requests (pmg_server_set_grouping)
  bool grouping = false;
  double group_max_work = 0;
  int max_group = 8;
  std::vector<pmg::SolveGroup*> groups;  // kept for reuse while the server lives
  std::vector<cudaStream_t> group_streams;
};

namespace {

void destroy_slot(pmg_server* s, Slot* sl) {
  pmg_destroy(sl->ctx);
  if (sl->stream) cudaStreamDestroy(sl->stream);
  s->used -= sl->bytes;
  s->slots.erase(std::find(s->slots.begin(), s->slots.end(), sl));
  delete sl;
}

// A slot for request r: an idle context with r's key, or a new one if the
// budget (after evicting idle contexts, least recently used first) and the
// device's free memory allow.  nullptr if r must wait.
Slot* acquire_slot(pmg_server* s, Request* r, int* err) {
  *err = PMG_OK;
  const Key k = key_of(r->cfg, r->cfg.geometry == PMG_GEOM_DISTORTED ? &r->disp : nullptr);
  for (Slot* sl : s->slots)
    if (!sl->busy && sl->key == k) return sl;
  while (s->used + r->bytes > s->budget) {
    Slot* victim = nullptr;
    for (Slot* sl : s->slots)
      if (!sl->busy && (!victim || sl->last_used < victim->last_used)) victim = sl;
    if (!victim) return nullptr;
    destroy_slot(s, victim);
  }
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    *err = fail(PMG_ERR_CUDA, "cudaMemGetInfo failed");
    return nullptr;
  }
  if ((int64_t)free_b < r->bytes + (int64_t)(256 << 20)) return nullptr;
  Slot* sl = new Slot();
  // small solves on high-priority streams: their kernels are scheduled ahead
  // of the pending blocks of large ones, so they are not stuck behind them
  const int prio = (s->policy == PMG_SERVE_SHORTEST_FIRST && r->work < s->small_work) ? s->prio_high : s->prio_low;
  if (cudaStreamCreateWithPriority(&sl->stream, cudaStreamNonBlocking, prio) != cudaSuccess) {
    cudaGetLastError();
    delete sl;
    *err = fail(PMG_ERR_CUDA, "cudaStreamCreate failed");
    return nullptr;
  }
  const int rc = pmg_create(&r->cfg, sl->stream, nullptr, 0, &sl->ctx);
  if (rc != PMG_OK) {
    cudaStreamDestroy(sl->stream);
    delete sl;
    *err = rc;
    return nullptr;
  }
  sl->disp = r->disp;  // the slot's key refers to its own copy
  sl->key = key_of(r->cfg, r->cfg.geometry == PMG_GEOM_DISTORTED ? &sl->disp : nullptr);
  sl->bytes = r->bytes;
  s->used += r->bytes;
  s->slots.push_back(sl);
  ++s->created_contexts;
  return sl;
}

// The queued request to admit next: the oldest (FIFO), or the one with the
// least estimated work, except that requests queued for max_wait_s or longer
// go first, oldest first (shortest-first with aging, so large requests are
// not starved).
std::deque<Request*>::iterator next_request(pmg_server* s) {
  auto it = s->queue.begin();
  if (s->policy != PMG_SERVE_SHORTEST_FIRST || s->queue.size() < 2) return it;
  const double now = now_s();
  if (now - (*it)->t_submit >= s->max_wait_s) return it;  // the oldest has waited too long
  auto best = it;
  for (; it != s->queue.end(); ++it)
    if ((*it)->work < (*best)->work) best = it;
  return best;
}

// Start r on its slot's context: in the group of running requests with the
// same method when grouping applies (a new group if none has room), else on
// its own.
int start_request(pmg_server* s, Request* r, Slot* sl) {
  if (s->grouping && r->work <= s->group_max_work) {
    pmg::SolveGroup* g = nullptr;
    for (pmg::SolveGroup* cand : s->groups)
      if (pmg::group_size(cand) < s->max_group && pmg::group_accepts(cand, sl->ctx)) {
        // a group that already holds requests of this method comes first
        if (!g || (pmg::group_size(g) == 0 && pmg::group_size(cand) > 0)) g = cand;
      }
    if (!g) {
      cudaStream_t st = nullptr;
      if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, s->prio_high) != cudaSuccess) {
        cudaGetLastError();
        st = nullptr;
      }
      if (st) {
        if (pmg::group_create(st, &g) == PMG_OK) {
          s->groups.push_back(g);
          s->group_streams.push_back(st);
        } else {
          cudaStreamDestroy(st);
          g = nullptr;
        }
      }
    }
    if (g && pmg::group_accepts(g, sl->ctx) &&
        pmg::group_join(g, sl->ctx, r->b, true, r->x, true, r->rtol, r->maxit) == PMG_OK)
      return PMG_OK;
    // not groupable (or no group could be made): on its own
  }
  return pmg_solve_start(sl->ctx, r->b, 1, r->x, 1, r->rtol, r->maxit);
}

}  // namespace

extern "C" {

int pmg_server_create(int64_t memory_budget_bytes, int max_active, pmg_server** out) {
  if (!out) return fail(PMG_ERR_ARG, "out is NULL");
  if (max_active < 1) return fail(PMG_ERR_ARG, "max_active must be >= 1");
  *out = nullptr;
  pmg_server* s = new pmg_server();
  if (memory_budget_bytes <= 0) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return fail(PMG_ERR_CUDA, "cudaMemGetInfo failed");
    }
    memory_budget_bytes = (int64_t)(0.9 * (double)free_b);
  }
  s->budget = memory_budget_bytes;
  s->max_active = max_active;
  if (cudaDeviceGetStreamPriorityRange(&s->prio_low, &s->prio_high) != cudaSuccess) {
    cudaGetLastError();
    s->prio_low = s->prio_high = 0;
  }
  now_s();
  *out = s;
  return PMG_OK;
}

int pmg_server_destroy(pmg_server* s) {
  if (!s) return PMG_OK;
  for (size_t i = 0; i < s->groups.size(); ++i) {
    if (pmg::group_size(s->groups[i]) > 0) pmg::group_cancel(s->groups[i]);
    pmg::group_destroy(s->groups[i]);
    cudaStreamDestroy(s->group_streams[i]);
  }
  s->groups.clear();
  for (Slot* sl : s->slots) {
    if (sl->stream) cudaStreamSynchronize(sl->stream);
  }
  while (!s->slots.empty()) destroy_slot(s, s->slots.back());
  for (auto& kv : s->requests) delete kv.second;
  delete s;
  return PMG_OK;
}

int pmg_server_submit(pmg_server* s, const pmg_config* cfg, const double* b_host, double* x_host, double rtol,
                      int maxit, int64_t* id) {
  if (!s || !cfg || !b_host || !x_host || !id) return fail(PMG_ERR_ARG, "NULL argument");
  if (maxit < 0 || !(rtol >= 0)) return fail(PMG_ERR_ARG, "bad rtol / maxit");
  int64_t bytes = 0;
  if (int rc = pmg_bytes_required(cfg, &bytes)) return rc;
  if (bytes > s->budget) return fail(PMG_ERR_OOM, "request needs more device memory than the server's budget");
  Request* r = new Request();
  r->id = s->next_id++;
  r->cfg = *cfg;
  if (cfg->geometry == PMG_GEOM_DISTORTED && cfg->vertex_disp) {
    // the request owns its displacements from here on: the caller's array
    // may be freed or reused before the request is admitted
    int64_t nv = 1;
    for (int d = 0; d < cfg->dim; ++d) nv *= cfg->n_cells + 1;
    r->disp.assign(cfg->vertex_disp, cfg->vertex_disp + nv * cfg->dim);
    r->cfg.vertex_disp = r->disp.data();
  }
  r->b = b_host;
  r->x = x_host;
  r->rtol = rtol;
  r->maxit = maxit;
  r->bytes = bytes;
  // estimated work: nodes of the finest grid times the degree (a local
  // p-multigrid solve costs roughly k operations per patch-interior value
  // more than a low-degree one)
  {
    double n1 = (double)cfg->degree * cfg->n_cells + 1, nodes = 1;
    for (int d = 0; d < cfg->dim; ++d) nodes *= n1;
    r->work = nodes * (cfg->degree + 2);
  }
  r->t_submit = now_s();
  s->requests[r->id] = r;
  s->queue.push_back(r);
  *id = r->id;
  return PMG_OK;
}

int pmg_server_poll(pmg_server* s, int* n_running, int* n_queued) {
  if (!s) return fail(PMG_ERR_ARG, "NULL server");
  while (!s->queue.empty() && (int)s->running.size() < s->max_active) {
    auto pos = next_request(s);
    Request* r = *pos;
    int err = PMG_OK;
    Slot* sl = acquire_slot(s, r, &err);
    if (err != PMG_OK) {
      s->queue.erase(pos);
      r->state = 3;
      r->status = err;
      r->t_done = now_s();
      continue;
    }
    if (!sl) break;  // wait for memory or a slot
    s->queue.erase(pos);
    sl->busy = true;
    r->slot = sl;
    r->t_start = now_s();
    const int rc = start_request(s, r, sl);
    if (rc != PMG_OK) {
      sl->busy = false;
      r->state = 3;
      r->status = rc;
      r->t_done = now_s();
      continue;
    }
    r->state = 1;
    s->running.push_back(r);
  }
  // advance the groups (a failed round ends its members with the error,
  // which pmg_solve_progress reports below), then every running solve
  for (pmg::SolveGroup* g : s->groups)
    if (pmg::group_size(g) > 0) pmg::group_progress(g, false);
  for (size_t i = 0; i < s->running.size();) {
    Request* r = s->running[i];
    int done = 0;
    const int rc = pmg_solve_progress(r->slot->ctx, &done, &r->info);
    if (rc < 0 || done) {
      r->state = rc < 0 ? 3 : 2;
      r->status = rc;
      r->t_done = now_s();
      r->slot->busy = false;
      r->slot->last_used = ++s->tick;
      r->slot = nullptr;
      s->running.erase(s->running.begin() + i);
      continue;
    }
    ++i;
  }
  if (n_running) *n_running = (int)s->running.size();
  if (n_queued) *n_queued = (int)s->queue.size();
  return PMG_OK;
}

int pmg_server_result(pmg_server* s, int64_t id, int* state, pmg_solve_info* info, double* t_submit,
                      double* t_start, double* t_done) {
  if (!s || !state) return fail(PMG_ERR_ARG, "NULL argument");
  auto it = s->requests.find(id);
  if (it == s->requests.end()) return fail(PMG_ERR_ARG, "unknown request id");
  Request* r = it->second;
  *state = r->state;
  if (info) *info = r->info;
  if (t_submit) *t_submit = r->t_submit;
  if (t_start) *t_start = r->t_start;
  if (t_done) *t_done = r->t_done;
  return r->state == 3 ? r->status : PMG_OK;
}

int pmg_server_set_policy(pmg_server* s, int policy, double max_wait_s, double small_work) {
  if (!s) return fail(PMG_ERR_ARG, "NULL server");
  if (policy != PMG_SERVE_FIFO && policy != PMG_SERVE_SHORTEST_FIRST) return fail(PMG_ERR_ARG, "unknown policy");
  if (!(max_wait_s > 0) || small_work < 0) return fail(PMG_ERR_ARG, "max_wait_s > 0, small_work >= 0");
  s->policy = policy;
  s->max_wait_s = max_wait_s;
  s->small_work = small_work;
  return PMG_OK;
}

int pmg_server_set_grouping(pmg_server* s, int enable, double max_work, int max_group) {
  if (!s) return fail(PMG_ERR_ARG, "NULL server");
  if (max_group < 1 || max_group > 32 || max_work < 0) return fail(PMG_ERR_ARG, "max_group in 1..32, max_work >= 0");
  s->grouping = enable != 0;
  s->group_max_work = max_work;
  s->max_group = max_group;
  return PMG_OK;
}

int pmg_server_release(pmg_server* s, int64_t id) {
  if (!s) return fail(PMG_ERR_ARG, "NULL server");
  auto it = s->requests.find(id);
  if (it == s->requests.end()) return fail(PMG_ERR_ARG, "unknown request id");
  if (it->second->state < 2) return fail(PMG_ERR_STATE, "request is still queued or running");
  delete it->second;
  s->requests.erase(it);
  return PMG_OK;
}

int pmg_server_stats(const pmg_server* s, int64_t* used_bytes, int* resident_contexts, int64_t* created_contexts) {
  if (!s) return fail(PMG_ERR_ARG, "NULL server");
  if (used_bytes) *used_bytes = s->used;
  if (resident_contexts) *resident_contexts = (int)s->slots.size();
  if (created_contexts) *created_contexts = s->created_contexts;
  return PMG_OK;
}

}  // extern "C"
