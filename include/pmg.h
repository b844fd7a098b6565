/*
 * pmg.h -- C ABI of the GB300 matrix-free p-multigrid vertex-patch library.
 *
 * The library solves the discrete Poisson problem A_l u_l = b_l (Eq. (4) of
 * arXiv 2512.02577) for the bilinear form a(u, v) = int grad u . grad v
 * (Eq. (3)) with continuous Q_k elements (Gauss-Lobatto nodal basis, (k+1)
 * Gauss points per direction) on a structured hierarchy of nested meshes of
 * the unit square / cube (Eq. (1)), homogeneous Dirichlet conditions.
 *
 * Vectors.  Every vector argument is a contiguous array over the full
 * (k n + 1)^d nodal grid of the level, lexicographic with x fastest.
 * Boundary entries are ignored on input and written as 0 on output.  Unless
 * a function says otherwise, vectors are DEVICE pointers owned by the caller
 * (e.g. torch tensors), double for PMG_FP64 and float for PMG_FP32.
 *
 * Streams.  All device work of a context is enqueued on the stream given to
 * pmg_create and is asynchronous unless the function says it synchronises.
 * A NULL stream makes the context create its own blocking stream (ordered
 * against the legacy default stream), because the V-cycle is captured into
 * a CUDA graph and the legacy stream cannot be captured.  A context is not thread-safe; use one
 * context per thread or request.
 *
 * Errors.  Functions return PMG_OK (0), PMG_NOT_CONVERGED (+1) or a negative
 * PMG_ERR_* code; pmg_last_error() returns a message for the calling thread's
 * last error.  On an error no device work is left half-enqueued by argument
 * checks; CUDA errors are reported as PMG_ERR_CUDA.
 */
#ifndef PMG_H
#define PMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum pmg_status {
  PMG_OK = 0,
  PMG_NOT_CONVERGED = 1,
  PMG_ERR_ARG = -1,          /* invalid argument (NULL pointer, bad level, bad size) */
  PMG_ERR_UNSUPPORTED = -2,  /* dim not 2/3, degree not 1..8; V-cycle/solve on a coarse level above 4096 free DoFs;
                                pmg_create when one patch's local p-multigrid does not fit in a block's shared
                                memory (3D FP64: deformed/distorted k = 8, deformed/distorted k = 7 with
                                local_cycles >= 2, Cartesian k = 8 with local_cycles >= 2) */
  PMG_ERR_OOM = -3,          /* device workspace could not be allocated / too small */
  PMG_ERR_CUDA = -4,         /* a CUDA runtime call or kernel launch failed */
  PMG_ERR_DEVICE_TIMEOUT = -5, /* a bounded device-side wait expired (reserved: no kernel of the library waits
                                  on another block or device -- the persistent patch launches take work from
                                  an atomic counter and never spin -- so nothing returns it today) */
  PMG_ERR_STATE = -6         /* call not valid in the context's current state */
};

enum pmg_geometry {
  PMG_GEOM_CARTESIAN = 0,   /* x = X on the uniform mesh */
  PMG_GEOM_DEFORMED = 1,    /* x = X + a prod_i sin(2 pi X_i) (1,..,1), analytic */
  PMG_GEOM_DISTORTED = 2    /* randomly distorted mesh (§3.2.2, §4): the finest mesh's vertices moved by
                               vertex_disp, every cell of every level the trilinear (2D: bilinear) image
                               of its displaced corners; a coarse vertex is the fine vertex at the same
                               grid position (levels nested topologically, Eq. (2) transfers unchanged) */
};

enum pmg_precision { PMG_FP64 = 0, PMG_FP32 = 1 };

/* Vertex-patch smoother (§2.1). */
enum pmg_smoother {
  PMG_SMOOTHER_ADDITIVE = 0,       /* u += omega_patch sum_j Pi_j^T d_j, all patches from one residual */
  PMG_SMOOTHER_MULTIPLICATIVE = 1  /* Algorithm 1: patches in turn, each from the current residual; run
                                      colour by colour over the 2^d vertex-parity colours (forward in
                                      pre-smoothing and pmg_smooth, backward in post-smoothing, so the
                                      V-cycle stays symmetric); no damping */
};

/* Outer Krylov solver of pmg_solve (V-cycle as preconditioner). */
enum pmg_outer {
  PMG_OUTER_CG = 0,    /* preconditioned CG: needs the symmetric (full) local V-cycle */
  PMG_OUTER_GMRES = 1  /* flexible right-preconditioned GMRES(gmres_restart), the paper's outer solver */
};

/* Layout of the patches of one thread block in shared memory (the smoother's
 * local solves, §3.2).  Both give bitwise the same results. */
enum pmg_patch_layout {
  PMG_PATCH_AUTO = 0,         /* autotuned (or patch-major when patches_per_block > 0) */
  PMG_PATCH_MAJOR = 1,        /* each patch's vectors contiguous, patches_per_block patches per block */
  PMG_PATCH_INTERLEAVED = 2   /* Cartesian only: a fixed number of patches per block (16 where shared
                                 memory allows, fewer at high degree) stored element-major, one patch
                                 per lane group, for conflict-free shared-memory access; when it is the
                                 autotuner's choice, levels with fewer patches than one such block per
                                 SM use the patch-major layout, when the config's, every level uses it */
};

/* Arithmetic of the FP64 operator apply. */
enum pmg_outer_apply {
  PMG_OUTER_APPLY_FP64 = 0,         /* IEEE double (default) */
  PMG_OUTER_APPLY_FLOAT_FLOAT = 1   /* FP64 vectors in and out, every product and sum carried as an unevaluated
                                       pair of floats (about 48 significant bits, relative error of A x within
                                       a few 1e-14 of |A| |x|) on the FP32 pipes -- on GB300 several times
                                       faster than the FP64 pipes; the coarse-matrix assembly stays in FP64.
                                       Cartesian meshes; deformed and distorted ones in 3D with degree <= 3
                                       and geom_precision PMG_FP32 (else PMG_ERR_UNSUPPORTED) */
};

typedef struct pmg_ctx pmg_ctx;

typedef struct pmg_config {
  int dim;             /* 2 or 3 */
  int n_cells;         /* cells per side on the finest level, n >= 1 */
  int degree;          /* k in 1..8 */
  int n_levels;        /* mesh levels; 0 = coarsen while n is even (n_0 = odd part of n) */
  int geometry;        /* PMG_GEOM_CARTESIAN or PMG_GEOM_DEFORMED */
  double deform_amp;   /* a of the deformation (0.05 in the deformed benchmark) */
  int mg_precision;    /* PMG_FP64 or PMG_FP32: arithmetic of the V-cycle, smoother, transfers */
  double omega_patch;  /* additive-Schwarz damping; <= 0 selects 1.5 / 2^d */
  double omega_jacobi[4]; /* Jacobi damping per p-level (index 0 = p 1, unused);
                             <= 0 selects 4 / (3 lambda_max(D^-1 A_{j,p})) of the Cartesian patch */
  int local_cycles;    /* N_iter of the local Richardson iteration (Algorithm 2), >= 1 */
  int smooth_steps;    /* pre- and post-smoothing sweeps per level, >= 1 */
  int patches_per_block; /* patch-major layout: patches per thread block in the smoother, 0 = autotuned */
  int local_half;      /* 1: the local solver is the half V-cycle of §3.2.2 (post-smoothing dropped,
                          one fine-level patch vmult instead of two; nonsymmetric, so outer_solver must
                          be PMG_OUTER_GMRES, else PMG_ERR_UNSUPPORTED); 0: full V-cycle */
  int outer_solver;    /* PMG_OUTER_CG (default) or PMG_OUTER_GMRES */
  int gmres_restart;   /* GMRES cycle length m in 1..64 (default 30); the context then holds 2m + 1
                          extra FP64 vectors of the finest level */
  int smoother;        /* PMG_SMOOTHER_ADDITIVE (default) or PMG_SMOOTHER_MULTIPLICATIVE */
  const double* vertex_disp; /* PMG_GEOM_DISTORTED only (else ignored): HOST array of the displacements
                          of the finest mesh's (n_cells + 1)^d vertices, d doubles per vertex, vertices
                          lexicographic with x fastest; boundary vertices must have zero normal
                          displacement for the domain to stay the unit square/cube.  pmg_create
                          returns PMG_ERR_ARG if a cell is inverted (det J <= 0 at a quadrature
                          point).  Read by pmg_create only (copied); the caller keeps ownership */
  int patch_layout;    /* shared-memory layout of the smoother's patch kernel (enum pmg_patch_layout):
                          PMG_PATCH_AUTO (default) = timed at creation among the admissible layouts and
                          block shapes; PMG_PATCH_MAJOR or PMG_PATCH_INTERLEAVED to fix the layout */
  int patch_threads;   /* PMG_PATCH_INTERLEAVED: threads per block (multiple of 32), 0 = autotuned */
  int outer_apply;     /* arithmetic of every FP64 operator apply (pmg_apply / pmg_residual with PMG_FP64,
                          the outer solver's A p and residuals): enum pmg_outer_apply */
  int geom_precision;  /* deformed and distorted geometry: storage of the quadrature-point tensors G_q
                          (6 components per Gauss point in 3D): PMG_FP32 (default; the discrete operator
                          of every precision is the one of the rounded G_q) or PMG_FP64 (twice the bytes;
                          the FP64 operator then uses G_q as computed) */
  int apply_cells_per_block; /* deformed and distorted geometry: cells per thread block of the operator
                          apply, 0 = autotuned (admissible values: 4, 8, 16 for the 3D k <= 3 FP32
                          kernel, else 1, 2, 4, ... while the cell tiles fit) */
  int patch_persistent; /* Cartesian patch launches: 0 = autotuned, 1 = persistent grids (the blocks the GPU
                          holds at once take batches of patches from a counter; used on levels with more
                          than one wave of batches), -1 = one block per batch */
  int coarse_dofs;      /* with n_levels = 0: 0 = coarsen while n is even; c > 0 (<= 4096) = stop at the
                          first mesh whose free DoFs are <= c, which is then solved by the dense coarse
                          solve (fewer, larger coarse levels: the smoother launches on meshes of a few
                          patches are latency, not work) */
} pmg_config;

typedef struct pmg_solve_info {
  int iterations;      /* outer iterations taken (CG iterations or GMRES Arnoldi steps) */
  double rel_residual; /* ||b - A x||_2 / ||b||_2: CG's recursively updated residual, or GMRES's
                          Givens estimate of it */
  double time_ms;      /* wall time of the solve on the context's stream */
  int status;          /* PMG_OK or PMG_NOT_CONVERGED */
} pmg_solve_info;

/* Fill *cfg with defaults: 3D, n 8, k 2, automatic levels, Cartesian, FP64,
 * default damping, one full local V-cycle, one smoothing step, CG outer
 * solver (GMRES restart length 30 if selected). */
void pmg_config_default(pmg_config* cfg);

/* Coarsest levels with more than 4096 free DoFs are accepted: such a context
 * applies, computes residuals and smooths, while pmg_vcycle and pmg_solve
 * return PMG_ERR_UNSUPPORTED. */

/* Device bytes the context for *cfg needs (hierarchy vectors, geometry,
 * inverse diagonals, coarse inverse, scratch).  Allocates nothing; used by
 * serving admission.  Returns PMG_ERR_UNSUPPORTED / PMG_ERR_ARG for configs
 * that pmg_create would reject. */
int pmg_bytes_required(const pmg_config* cfg, int64_t* bytes);

/* Create a context: validate *cfg, lay out the level hierarchy n_l = n_0 2^l
 * (Eq. (1)), compute geometry factors and inverse diagonals for every mesh
 * level and p-level (§3.2), and factor the coarsest level.  `stream` is a
 * cudaStream_t (NULL: the context creates a blocking stream of its own).  `workspace` is a device buffer of
 * `workspace_bytes` >= pmg_bytes_required owned by the caller and used for
 * all device storage of the context; NULL makes the library cudaMalloc its
 * own (freed by pmg_destroy).  Synchronises the stream before returning. */
int pmg_create(const pmg_config* cfg, void* stream, void* workspace, int64_t workspace_bytes,
               pmg_ctx** out);

/* Destroy a context; frees what pmg_create allocated. NULL is accepted. */
int pmg_destroy(pmg_ctx* ctx);

/* Number of levels and the nodal-grid length (k n_l + 1)^d of `level`
 * (0 = coarsest, n_levels - 1 = finest). */
int pmg_num_levels(const pmg_ctx* ctx, int* n_levels);
int pmg_num_dofs(const pmg_ctx* ctx, int level, int64_t* n);

/* y = A_level x (Eq. (4)), matrix-free by sum factorisation; `prec` selects
 * the arithmetic and the element type of x and y. */
int pmg_apply(pmg_ctx* ctx, int level, int prec, const void* x, void* y);

/* r = b - A_level u (the "evaluate" step of Algorithm 1, here global). */
int pmg_residual(pmg_ctx* ctx, int level, int prec, const void* b, const void* u, void* r);

/* `sweeps` vertex-patch sweeps on `level` with the configured smoother.  The
 * level must have patches (n >= 2 cells per side) and smoother data: every
 * level but the coarsest of a deformed or distorted hierarchy (Cartesian
 * patch operators need no stored data; a single-level context is smoothable
 * on its one level); PMG_ERR_ARG otherwise.  The smoother is
 * additive,
 *   u <- u + omega_AS sum_j Pi_j^T LocalSolve_j(Pi_j (b - A u)),
 * the patch update of Algorithm 1 summed over all patches; or
 * multiplicative, Algorithm 1 itself (per parity colour: r = b - A u, then
 * u += Pi_j^T LocalSolve_j(Pi_j r) for every patch of the colour), colours in
 * increasing order.  LocalSolve = Algorithm 2 around the p-multigrid V-cycle
 * of Algorithm 3 (full, or half with local_half). */
int pmg_smooth(pmg_ctx* ctx, int level, int prec, const void* b, void* u, int sweeps);

/* One geometric V-cycle on the finest level from a zero guess: z = B r
 * (double in and out; internally FP32 when mg_precision is PMG_FP32). */
int pmg_vcycle(pmg_ctx* ctx, const double* r, double* z);

/* Outer Krylov solve, x_0 = 0, FP64 vectors and dots, the V-cycle as
 * preconditioner, until ||r||_2 <= rtol ||b||_2 or maxit iterations:
 * preconditioned CG, or with outer_solver PMG_OUTER_GMRES flexible
 * right-preconditioned GMRES(m) (Arnoldi with two classical Gram-Schmidt
 * passes, Givens rotations on the device; the paper's outer solver, §3.2.2).
 * Synchronises the stream.  Returns PMG_OK or PMG_NOT_CONVERGED; *info may
 * be NULL. */
int pmg_solve(pmg_ctx* ctx, const double* b, double* x, double rtol, int maxit, pmg_solve_info* info);

/* pmg_solve on HOST arrays: copies b to the device, solves, copies x back.
 * b and x are host pointers of length pmg_num_dofs(finest); pinned memory
 * makes the copies asynchronous. Synchronises the stream. */
int pmg_solve_host(pmg_ctx* ctx, const double* b_host, double* x_host, double rtol, int maxit,
                   pmg_solve_info* info);

/* Incremental form of pmg_solve, for drivers that interleave many contexts
 * (the serving loop): pmg_solve_start enqueues the set-up and the first
 * preconditioner step and returns; pmg_solve_progress never blocks -- it
 * advances the CG iteration as far as completed device work allows (each
 * iteration enqueues the next V-cycle before its residual norm is read) and
 * sets *done = 1 once x has been written (x on the host if x_on_host, then
 * pinned memory is required for the copy to overlap), filling *info and
 * returning the solve's status.  Same iterations and result as pmg_solve.
 * One solve per context at a time (PMG_ERR_STATE otherwise). */
int pmg_solve_start(pmg_ctx* ctx, const double* b, int b_on_host, double* x, int x_on_host, double rtol, int maxit);
int pmg_solve_progress(pmg_ctx* ctx, int* done, pmg_solve_info* info);

/* Solve count (1..32) systems at once, each on its own context, with every
 * kernel launch covering all of them (not in the paper: batching of
 * concurrent solves).  The contexts must share the dimension, degree, MG
 * precision, smoother, local cycles, half cycle, smoothing steps and outer
 * operator, and be Cartesian, PCG, with a coarse level of <= 4096 free DoFs;
 * their mesh sizes (and numbers of levels) and damping may differ.  b[i],
 * x[i]: device double vectors of context i's finest level.  The systems
 * iterate in lockstep (one CG iteration of every unconverged system per
 * round); each stops at its own tolerance or maxit, and its iterations and
 * x are bitwise those of pmg_solve on its context.  Runs on ctxs[0]'s
 * stream, after the work already enqueued on every context's stream;
 * blocks until all are done.  info: count entries (or NULL).  Returns
 * PMG_OK, PMG_NOT_CONVERGED if any system stopped at maxit, or the first
 * error (PMG_ERR_ARG for a mismatched or repeated context, PMG_ERR_UNSUPPORTED
 * for a context that cannot be grouped).  Allocates a few bytes of device
 * memory for its duration. */
int pmg_solve_group(pmg_ctx* const* ctxs, int count, const double* const* b, double* const* x, double rtol,
                    int maxit, pmg_solve_info* info);

/* b_i = int f phi_i with f = d pi^2 prod_i sin(pi x_i), the load for the
 * manufactured solution u = prod_i sin(pi x_i), (k+1)-point Gauss rule, on
 * the finest level (device, double). */
int pmg_rhs_manufactured(pmg_ctx* ctx, double* b);

/* || x - u ||_{L2} for the manufactured u, (k+3)-point Gauss rule; x is a
 * device double vector on the finest level. Synchronises the stream. */
int pmg_l2_error_manufactured(pmg_ctx* ctx, const double* x, double* err);

/* Wait for all work enqueued by the context. */
int pmg_synchronize(pmg_ctx* ctx);

/* Process-wide number of kernel launches the library has enqueued
 * (instrumentation for benchmarks; a CUDA-graph replay counts its kernel
 * nodes). */
int64_t pmg_launch_count(void);

/* Patches per thread block the smoother kernels of this context use on the
 * finest level: the config's value, or the autotuned one (layout and block
 * shape timed per dimension, degree, precision, geometry, local cycles,
 * smoother and finest n on the finest level's patch launches of one sweep;
 * cached for the process and, if the environment variable PMG_TUNE_FILE
 * names a file, in that file). */
int pmg_patches_per_block(const pmg_ctx* ctx, int* ppc);

/* 1 if the context's Cartesian patch launches run as persistent grids, else 0. */
int pmg_patch_persistent(const pmg_ctx* ctx, int* persistent);

/* Cells per thread block of a deformed or distorted context's operator
 * apply in the multigrid precision: the autotuned value (timed at creation
 * per dimension, degree, precision, geometry storage and finest n on the
 * finest level's apply; meshes below 32^3 cells use the kernel's rule and
 * report 0), 0 on Cartesian contexts. */
int pmg_apply_cells_per_block(const pmg_ctx* ctx, int* cells_per_block);

/* The patch-kernel layout of a context's finest level (enum
 * pmg_patch_layout, never AUTO), its patches per block and threads per
 * block, as chosen by the config or the autotuner. */
int pmg_patch_layout(const pmg_ctx* ctx, int* layout, int* patches_per_block, int* threads);

/* The damping a context runs with: omega_AS of the additive smoother and the
 * local Jacobi damping omega_J per p-level (omega_jacobi[4], index 0 = the
 * p = 1 level, unused and 1; entries beyond the context's p-levels are 1).
 * The config's values where it gives them (> 0), else the defaults below. */
int pmg_damping(const pmg_ctx* ctx, double* omega_patch, double* omega_jacobi);

/* Default damping for (dim, degree), without a context or a GPU (host
 * arithmetic only).  The paper gives no damping (§2.2, §3.2 name a damped
 * Jacobi smoother; its smoother is multiplicative and needs no omega_AS), so
 * these are readings: omega_AS = 1.5 / 2^d (a free DoF lies in at most 2^d
 * patch interiors), omega_J(p) = 4 / (3 lambda_max(D^-1 A_{j,p})) on the
 * Cartesian patch of degree p (scale invariant), lambda_max by Lanczos. */
int pmg_default_damping(int dim, int degree, double* omega_patch, double* omega_jacobi);

/* Instrumentation: mean device times (ms, CUDA events on the context's
 * stream) of the three phases of one smoothing step on `level`, over `reps`
 * repetitions after one warm-up, on the level's own vectors: ms[0] residual
 * r = b - A u, ms[1] the patch launch (every local solve), ms[2] the gather
 * u += sum_j Pi_j^T d_j.  Overwrites the level's work vectors. */
int pmg_smoother_phase_times(pmg_ctx* ctx, int level, int reps, double* ms);

const char* pmg_status_string(int status);
const char* pmg_last_error(void);

/* ------------------------------------------------------------------ serving
 * Many solves resident on one GPU (not in the paper: the serving layer of
 * this library).  pmg_server_submit queues a request (config, host b and x
 * of pmg_num_dofs(finest) doubles each -- pinned memory for overlapping
 * copies -- tolerance, iteration cap); pmg_server_poll never blocks: it
 * admits queued requests in arrival order while fewer than max_active run
 * and the request's pmg_bytes_required fits in the budget (in the order of
 * pmg_server_set_policy; an idle resident
 * context is reused when the request's configuration would build the same
 * operator and preconditioner: every pmg_config field pmg_create reads -- dim,
 * n, degree, levels, precision, geometry and, for the deformed geometry, its
 * amplitude, damping (all values <= 0 count as "default"), local cycles,
 * smoothing steps, half cycle, smoother, outer solver and restart, patches
 * per block -- and for a distorted mesh the same displacement values;
 * least-recently-used idle contexts are evicted to make room),
 * advances every running solve (pmg_solve_progress) and retires finished
 * ones.  Each resident context has its own stream, so the kernels of
 * concurrent requests overlap on the device.  One host thread drives a
 * server.  Budget <= 0 selects 90% of the free device memory. */
typedef struct pmg_server pmg_server;
int pmg_server_create(int64_t memory_budget_bytes, int max_active, pmg_server** out);
int pmg_server_destroy(pmg_server* server);
/* PMG_ERR_OOM if the request can never fit in the budget.  The config is
 * copied, and for a distorted mesh so are its vertex displacements: the
 * caller may free cfg and cfg->vertex_disp on return.  b_host and x_host must
 * stay valid until the request is done. */
int pmg_server_submit(pmg_server* server, const pmg_config* cfg, const double* b_host, double* x_host, double rtol,
                      int maxit, int64_t* request_id);
int pmg_server_poll(pmg_server* server, int* n_running, int* n_queued);
/* *state: 0 queued, 1 running, 2 done (x_host written, *info filled), 3
 * failed (the return value is its error).  Times in seconds on the host's
 * steady clock: submission, admission, completion. */
int pmg_server_result(pmg_server* server, int64_t request_id, int* state, pmg_solve_info* info, double* t_submit,
                      double* t_start, double* t_done);
/* Admission order of a server (default PMG_SERVE_FIFO, arrival order).
 * PMG_SERVE_SHORTEST_FIRST admits the queued request with the least
 * estimated work (finest-grid nodes x (degree + 2)) first, except that a
 * request queued for max_wait_s seconds or more goes first (oldest first),
 * and runs requests whose estimated work is below small_work on
 * high-priority CUDA streams, so that small solves are not held behind the
 * blocks of large ones.  Applies to requests admitted after the call. */
enum pmg_serve_policy { PMG_SERVE_FIFO = 0, PMG_SERVE_SHORTEST_FIRST = 1 };
int pmg_server_set_policy(pmg_server* server, int policy, double max_wait_s, double small_work);

/* Grouped launches across concurrent requests (continuous batching; off by
 * default): a running request whose estimated work is at most max_work and
 * whose method allows it (as pmg_solve_group) joins the group of running
 * requests with the same method -- any mesh size -- and is solved with them
 * in lockstep, each launch of an iteration covering every member, members
 * joining at the next round and leaving when converged, up to max_group
 * (1..32) members per group, each group on its own high-priority stream.
 * Results are bitwise those of the request solved alone.  enable = 0 turns
 * grouping off for requests admitted after the call. */
int pmg_server_set_grouping(pmg_server* server, int enable, double max_work, int max_group);

/* Forget a finished (done or failed) request: its id becomes unknown.  The
 * server keeps every request until it is released or the server destroyed,
 * so a long-running driver releases each request once it has read the
 * result.  PMG_ERR_STATE while the request is queued or running. */
int pmg_server_release(pmg_server* server, int64_t request_id);
int pmg_server_stats(const pmg_server* server, int64_t* used_bytes, int* resident_contexts,
                     int64_t* created_contexts);

/* Largest nodal grid (k n + 1)^d that pmg_apply_cartesian_noalloc accepts. */
#define PMG_NOALLOC_MAX_DOFS 2097152

/* y = A x for the Cartesian Q_k operator on the unit square/cube with
 * n_cells per side (FP64, device vectors of (k n + 1)^d entries, the layout
 * and boundary convention above), enqueued on `stream` (NULL = legacy
 * default stream), without a context and without allocating device memory.
 * The paper has no counterpart: this exists for callers that cannot
 * allocate device memory -- code running inside another framework's memory
 * pool or under a hard memory cap, and real-time loops where cudaMalloc,
 * which may synchronise the device, is not allowed.  Its scratch (four grid
 * vectors) is a file-scope device array of 4 x PMG_NOALLOC_MAX_DOFS doubles
 * (64 MiB) that every GPU loading the library holds until exit.  The first
 * call on a device (and the first for each degree) resolves that array's
 * address and loads the degree's 1D matrices into constant memory (once per
 * degree and dimension), which
 * synchronises: make it before any stream capture.  All calls share the
 * array; calls that overlap on the GPU race on it.  Grids above
 * PMG_NOALLOC_MAX_DOFS are rejected with PMG_ERR_UNSUPPORTED.  x, y and the
 * stream must belong to the calling thread's current device: the scratch
 * array, the constant-memory upload and the launch all use that device. */
int pmg_apply_cartesian_noalloc(int dim, int n_cells, int degree, const double* x, double* y, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PMG_H */
