// Grouped solves inside the library (pmg.cu): several contexts' PCG solves
// advanced in lockstep, every launch of a round covering all of them.  The
// serving loop uses these to batch the launches of concurrent requests;
// pmg_solve_group is the blocking public form.
#pragma once
#include <cuda_runtime.h>

#include "../../include/pmg.h"

namespace pmg {

struct SolveGroup;

// A group whose launches go on `stream` (nullptr: a stream of its own).
int group_create(cudaStream_t stream, SolveGroup** out);
// PMG_ERR_STATE while systems are running or joining.
int group_destroy(SolveGroup* g);
// running plus joining systems
int group_size(const SolveGroup* g);
// true if ctx can join: groupable, idle, the group's method, room left
bool group_accepts(const SolveGroup* g, const pmg_ctx* ctx);
// ctx joins at the next round (its coarse level is set up now, on its own
// stream); b / x on the host (pinned memory to overlap) or the device.
int group_join(SolveGroup* g, pmg_ctx* ctx, const double* b, bool b_host, double* x, bool x_host, double rtol,
               int maxit);
// End every system of the group with PMG_ERR_STATE (no solution copied) and
// wait for the group's stream; the contexts become usable again.
int group_cancel(SolveGroup* g);
// Advance as far as completed device work allows (block: wait for the round
// in flight).  Systems that finished have left the group; pmg_solve_progress
// on their contexts completes them (it reports "running" while a context is
// still in a group).
int group_progress(SolveGroup* g, bool block);

}  // namespace pmg
