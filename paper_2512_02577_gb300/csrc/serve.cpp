// Serving loop: many Poisson solves of different sizes and degrees resident
// on one GPU at once.
//
// A request (config, host right-hand side, host solution buffer) is queued
// by pmg_server_submit.  pmg_server_poll, which never blocks, (1) admits
// queued requests in arrival order while a slot is free and the request's
// context fits in the device-memory budget -- reusing an idle resident
// context with the same (dim, n, degree, precision, geometry, levels) when
// one exists, evicting least-recently-used idle contexts otherwise -- (2)
// advances every running solve as far as its completed device work allows
// (pmg_solve_progress: each CG iteration enqueues its V-cycle, captured as a
// CUDA graph, before the host reads the residual), and (3) retires solves
// whose solution has reached the host.  Each slot has its own CUDA stream,
// so kernels of different requests overlap on the device, and a request that
// arrives while others run starts as soon as a slot and memory free up.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/pmg.h"

namespace pmg {
void set_last_error(const std::string& msg);
}

namespace {

int fail(int code, const std::string& msg) {
  pmg::set_last_error(msg);
  return code;
}

// contexts are reused only for the same configuration (a distorted mesh: the
// same displacement array, by address)
using Key = std::tuple<int, int, int, int, int, int, int, int, int, int, int, int, const double*>;

Key key_of(const pmg_config& c) {
  return Key(c.dim, c.n_cells, c.degree, c.mg_precision, c.geometry, c.n_levels, c.local_cycles, c.smooth_steps,
             c.local_half, c.outer_solver, c.outer_solver == PMG_OUTER_GMRES ? c.gmres_restart : 0, c.smoother,
             c.geometry == PMG_GEOM_DISTORTED ? c.vertex_disp : nullptr);
}

struct Slot {
  pmg_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  Key key;
  int64_t bytes = 0;
  bool busy = false;
  int64_t last_used = 0;
};

struct Request {
  int64_t id = 0;
  pmg_config cfg{};
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
  int64_t used = 0;
  int64_t tick = 0;
  int64_t next_id = 1;
  std::deque<Request*> queue;
  std::vector<Request*> running;
  std::map<int64_t, Request*> requests;
  std::vector<Slot*> slots;
  int64_t created_contexts = 0;
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
  const Key k = key_of(r->cfg);
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
  if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess) {
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
  sl->key = k;
  sl->bytes = r->bytes;
  s->used += r->bytes;
  s->slots.push_back(sl);
  ++s->created_contexts;
  return sl;
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
  now_s();
  *out = s;
  return PMG_OK;
}

int pmg_server_destroy(pmg_server* s) {
  if (!s) return PMG_OK;
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
  r->b = b_host;
  r->x = x_host;
  r->rtol = rtol;
  r->maxit = maxit;
  r->bytes = bytes;
  r->t_submit = now_s();
  s->requests[r->id] = r;
  s->queue.push_back(r);
  *id = r->id;
  return PMG_OK;
}

int pmg_server_poll(pmg_server* s, int* n_running, int* n_queued) {
  if (!s) return fail(PMG_ERR_ARG, "NULL server");
  // admit in arrival order
  while (!s->queue.empty() && (int)s->running.size() < s->max_active) {
    Request* r = s->queue.front();
    int err = PMG_OK;
    Slot* sl = acquire_slot(s, r, &err);
    if (err != PMG_OK) {
      s->queue.pop_front();
      r->state = 3;
      r->status = err;
      r->t_done = now_s();
      continue;
    }
    if (!sl) break;  // wait for memory or a slot
    s->queue.pop_front();
    sl->busy = true;
    r->slot = sl;
    r->t_start = now_s();
    const int rc = pmg_solve_start(sl->ctx, r->b, 1, r->x, 1, r->rtol, r->maxit);
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
  // advance every running solve; retire finished ones
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

int pmg_server_stats(const pmg_server* s, int64_t* used_bytes, int* resident_contexts, int64_t* created_contexts) {
  if (!s) return fail(PMG_ERR_ARG, "NULL server");
  if (used_bytes) *used_bytes = s->used;
  if (resident_contexts) *resident_contexts = (int)s->slots.size();
  if (created_contexts) *created_contexts = s->created_contexts;
  return PMG_OK;
}

}  // extern "C"
