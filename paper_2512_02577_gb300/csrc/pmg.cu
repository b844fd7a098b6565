// Host runtime of the library: context and device memory plan, hierarchy
// set-up, the geometric V-cycle (captured once as a CUDA graph), the FP64
// preconditioned CG driver, and the C ABI declared in include/pmg.h.
//
// Method: §2 of arXiv 2512.02577 -- nested meshes (Eq. (1)), embedding
// prolongation and its l2-adjoint restriction (Eq. (2)), level matrices of
// the bilinear form (Eq. (3), Eq. (4)), vertex-patch smoothing (§2.1, here
// additive), local p-multigrid (§2.2, Algorithms 2 and 3).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/pmg.h"
#include "pmg_common.cuh"
#include "ctx.h"
#include "pmg_kernels_api.h"
#include "setup.h"
#include "vec.h"

namespace pmg {
#define PMG_DECLARE_PARTS(k)                    \
  const KernelTable* kernel_table_k##k##_d2_p0(); \
  const KernelTable* kernel_table_k##k##_d2_p1(); \
  const KernelTable* kernel_table_k##k##_d3_p0(); \
  const KernelTable* kernel_table_k##k##_d3_p1();
PMG_DECLARE_PARTS(1)
PMG_DECLARE_PARTS(2)
PMG_DECLARE_PARTS(3)
PMG_DECLARE_PARTS(4)
PMG_DECLARE_PARTS(5)
PMG_DECLARE_PARTS(6)
PMG_DECLARE_PARTS(7)
PMG_DECLARE_PARTS(8)
#undef PMG_DECLARE_PARTS

const KernelTable* kernel_table(int K, int dim, int prec) {
  using Fn = const KernelTable* (*)();
#define PMG_PARTS(k) {{kernel_table_k##k##_d2_p0, kernel_table_k##k##_d2_p1}, \
                      {kernel_table_k##k##_d3_p0, kernel_table_k##k##_d3_p1}}
  static const Fn parts[8][2][2] = {PMG_PARTS(1), PMG_PARTS(2), PMG_PARTS(3), PMG_PARTS(4),
                                    PMG_PARTS(5), PMG_PARTS(6), PMG_PARTS(7), PMG_PARTS(8)};
#undef PMG_PARTS
  if (K < 1 || K > 8 || dim < 2 || dim > 3 || prec < 0 || prec > 1) return nullptr;
  return parts[K - 1][dim - 2][prec]();
}
}  // namespace pmg

using namespace pmg;

namespace {
thread_local std::string t_last_error;
}  // namespace

namespace pmg {
void set_last_error(const std::string& msg) { t_last_error = msg; }

int fail(int code, const std::string& msg) {
  t_last_error = msg;
  return code;
}
}  // namespace pmg

namespace {


int64_t ipow64(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}


int64_t bump(int64_t& cur, int64_t bytes) {
  const int64_t o = cur;
  cur += (bytes + kAlign - 1) / kAlign * kAlign;
  return o;
}

int make_plan(const pmg_config* cfg, Plan& P) {
  if (!cfg) return fail(PMG_ERR_ARG, "config is NULL");
  if (cfg->dim != 2 && cfg->dim != 3) return fail(PMG_ERR_UNSUPPORTED, "dim must be 2 or 3");
  if (cfg->degree < 1 || cfg->degree > 8) return fail(PMG_ERR_UNSUPPORTED, "degree must be in 1..8");
  if (cfg->n_cells < 1) return fail(PMG_ERR_ARG, "n_cells must be >= 1");
  if (cfg->geometry != PMG_GEOM_CARTESIAN && cfg->geometry != PMG_GEOM_DEFORMED &&
      cfg->geometry != PMG_GEOM_DISTORTED)
    return fail(PMG_ERR_ARG, "unknown geometry");
  if (cfg->geometry == PMG_GEOM_DISTORTED && !cfg->vertex_disp)
    return fail(PMG_ERR_ARG, "distorted geometry needs vertex_disp");
  if (cfg->mg_precision != PMG_FP64 && cfg->mg_precision != PMG_FP32) return fail(PMG_ERR_ARG, "unknown precision");
  if (cfg->local_cycles < 1 || cfg->smooth_steps < 1) return fail(PMG_ERR_ARG, "local_cycles, smooth_steps >= 1");
  if (cfg->local_half != 0 && cfg->local_half != 1) return fail(PMG_ERR_ARG, "local_half must be 0 or 1");
  if (cfg->outer_solver != PMG_OUTER_CG && cfg->outer_solver != PMG_OUTER_GMRES)
    return fail(PMG_ERR_ARG, "unknown outer_solver");
  if (cfg->outer_solver == PMG_OUTER_GMRES && (cfg->gmres_restart < 1 || cfg->gmres_restart > kMaxKrylov))
    return fail(PMG_ERR_ARG, "gmres_restart must be in 1..64");
  if (cfg->smoother != PMG_SMOOTHER_ADDITIVE && cfg->smoother != PMG_SMOOTHER_MULTIPLICATIVE)
    return fail(PMG_ERR_ARG, "unknown smoother");
  if (cfg->patch_layout != PMG_PATCH_AUTO && cfg->patch_layout != PMG_PATCH_MAJOR &&
      cfg->patch_layout != PMG_PATCH_INTERLEAVED)
    return fail(PMG_ERR_ARG, "unknown patch_layout");
  if (cfg->outer_apply != PMG_OUTER_APPLY_FP64 && cfg->outer_apply != PMG_OUTER_APPLY_FLOAT_FLOAT)
    return fail(PMG_ERR_ARG, "unknown outer_apply");
  if (cfg->outer_apply == PMG_OUTER_APPLY_FLOAT_FLOAT && cfg->geometry != PMG_GEOM_CARTESIAN &&
      !(cfg->dim == 3 && cfg->degree <= 3 && cfg->geom_precision == PMG_FP32))
    return fail(PMG_ERR_UNSUPPORTED,
                "the float-float operator on deformed or distorted meshes needs 3D, degree <= 3 and FP32 geometry");
  if (cfg->geom_precision != PMG_FP64 && cfg->geom_precision != PMG_FP32)
    return fail(PMG_ERR_ARG, "unknown geom_precision");
  if (cfg->patches_per_block < 0 || cfg->patch_threads < 0 || cfg->apply_cells_per_block < 0)
    return fail(PMG_ERR_ARG, "patches_per_block, patch_threads, apply_cells_per_block >= 0");
  if (cfg->patch_persistent < -1 || cfg->patch_persistent > 1) return fail(PMG_ERR_ARG, "patch_persistent in {-1, 0, 1}");
  if (cfg->coarse_dofs < 0 || cfg->coarse_dofs > kMaxCoarse) return fail(PMG_ERR_ARG, "coarse_dofs in 0..4096");
  if (cfg->local_half && cfg->outer_solver == PMG_OUTER_CG)
    return fail(PMG_ERR_UNSUPPORTED, "the half local V-cycle makes the preconditioner nonsymmetric: use GMRES");
  P.dim = cfg->dim;
  P.K = cfg->degree;
  P.deformed = cfg->geometry != PMG_GEOM_CARTESIAN;  // general geometry: stored G_q
  P.mg32 = cfg->mg_precision == PMG_FP32;
  P.mg_es = P.mg32 ? 4 : 8;
  P.g_es = cfg->geom_precision == PMG_FP64 ? 8 : 4;
  P.nplev = nlev(P.K);
  // mesh levels: n_l = n_0 2^l
  int n = cfg->n_cells, L = cfg->n_levels;
  auto free_dofs = [&](int m) { return ipow64(std::max<int64_t>((int64_t)P.K * m - 1, 0), P.dim); };
  if (L <= 0) {
    // halve while n is even; with coarse_dofs > 0, stop at the first mesh
    // whose free DoFs fit that dense coarse solve
    L = 1;
    while (n % 2 == 0 && n / 2 >= 1 && !(cfg->coarse_dofs > 0 && free_dofs(n) <= cfg->coarse_dofs)) {
      n /= 2;
      ++L;
    }
  } else {
    for (int i = 1; i < L; ++i) {
      if (n % 2) return fail(PMG_ERR_UNSUPPORTED, "n_cells must be divisible by 2^(n_levels-1)");
      n /= 2;
    }
  }
  P.n0 = n;
  P.nlev = L;
  P.ns.resize(L);
  for (int l = 0; l < L; ++l) P.ns[l] = P.n0 << l;
  const int64_t nc1 = (int64_t)P.K * P.n0 - 1;
  const int64_t nc = ipow64(std::max<int64_t>(nc1, 0), P.dim);
  // a coarse problem above the dense limit leaves apply / residual / smooth
  // usable; V-cycles and solves are then rejected
  P.coarse_ok = nc <= kMaxCoarse;
  P.nc = P.coarse_ok ? (int)nc : 0;
  const int ncomp = P.dim == 3 ? 6 : 3;
  int64_t cur = 0;
  P.lo.resize(L);
  for (int l = 0; l < L; ++l) {
    const int nl = P.ns[l];
    const int64_t N = ipow64((int64_t)P.K * nl + 1, P.dim);
    auto& o = P.lo[l];
    o.b = bump(cur, N * P.mg_es);
    o.u = bump(cur, N * P.mg_es);
    o.r = bump(cur, N * P.mg_es);
    for (int i = 0; i < 4; ++i) o.G[i] = o.dinv[i] = -1;
    o.dinv1 = -1;
    if (P.deformed) {
      // smoother data on every level that is smoothed: all but the coarsest
      // of a hierarchy, and the only level of a single-level context
      const bool smoothed = l > 0 || L == 1;
      for (int pl = 0; pl < P.nplev; ++pl) {
        const int p = plev(P.K, pl);
        const bool top = pl == P.nplev - 1;
        if (!top && !smoothed) continue;  // coarsest level: only the operator itself
        o.G[pl] = bump(cur, ipow64(nl, P.dim) * ipow64(p + 1, P.dim) * ncomp * P.g_es);
        if (smoothed && pl > 0) o.dinv[pl] = bump(cur, ipow64((int64_t)p * nl + 1, P.dim) * P.mg_es);
      }
      if (smoothed) o.dinv1 = bump(cur, ipow64(nl + 1, P.dim) * P.mg_es);
    }
  }
  const int64_t NF = ipow64((int64_t)P.K * cfg->n_cells + 1, P.dim);
  for (int i = 0; i < 4; ++i) P.t64[i] = bump(cur, NF * 8);
  for (int i = 0; i < 4; ++i) P.t_mg[i] = P.mg32 ? bump(cur, NF * 4) : P.t64[i];
  for (int i = 0; i < 6; ++i) P.cg[i] = bump(cur, NF * 8);
  if (cfg->outer_solver == PMG_OUTER_GMRES) {
    P.m = cfg->gmres_restart;
    P.gv = bump(cur, (P.m + 1) * NF * 8);
    P.gz = bump(cur, P.m * NF * 8);
    P.gh = bump(cur, (int64_t)(P.m + 1) * P.m * 8);
    P.gs = bump(cur, GmresState::size(P.m) * 8);
    P.gpart = bump(cur, (int64_t)(P.m + 1) * kDotBlocks * 8);
  }
  P.scal = bump(cur, S_COUNT * 8);
  P.counter = bump(cur, 16);  // work counter of the persistent patch launches
  P.partial = bump(cur, kDotBlocks * 8 * 2);
  P.dtab_len = 0;
  for (int pl = 1; pl < P.nplev; ++pl) P.dtab_len += ipow64(mp(plev(P.K, pl)), P.dim);
  P.dtab64 = bump(cur, std::max<int64_t>(P.dtab_len, 1) * 8);
  P.dtab32 = bump(cur, std::max<int64_t>(P.dtab_len, 1) * 4);
  P.cidx = bump(cur, std::max(P.nc, 1) * 4);
  P.ainv = bump(cur, std::max<int64_t>((int64_t)P.nc * P.nc, 1) * P.mg_es);
  P.a64 = P.mg32 ? bump(cur, std::max<int64_t>((int64_t)P.nc * P.nc, 1) * 8) : P.ainv;
  P.gjrow = bump(cur, std::max(P.nc, 1) * 8);
  P.gjcol = bump(cur, std::max(P.nc, 1) * 8);
  P.gjbad = bump(cur, 8);
  const int64_t N0 = ipow64((int64_t)P.K * P.n0 + 1, P.dim);
  P.cx0 = bump(cur, N0 * 8);  // unit vectors and operator columns of the coarse set-up
  P.cy0 = bump(cur, N0 * 8);
  // patch corrections of one smoothing step, one node-major vector per parity
  // colour (finest level; reused by the coarser ones) and, deformed, per-cell
  // operator results (FP64 for the CG)
  const int nf = cfg->n_cells;
  P.pbuf = bump(cur, (int64_t)(1 << P.dim) * ipow64((int64_t)P.K * nf + 1, P.dim) * P.mg_es);
  if (cfg->geometry == PMG_GEOM_DISTORTED) P.verts = bump(cur, ipow64(nf + 1, P.dim) * P.dim * 8);
  if (P.deformed) P.cellbuf = bump(cur, ipow64(nf, P.dim) * ipow64(P.K + 1, P.dim) * 8);
  P.total = cur;
  return PMG_OK;
}

}  // namespace

namespace {

void* at(pmg_ctx* c, int64_t off) { return off < 0 ? nullptr : (void*)(c->ws + off); }

}  // namespace

namespace pmg {
PatchParamsHost patch_params(const pmg_ctx* c, int level) {
  PatchParamsHost P;
  P.scale = c->lv[level].scale;
  P.omega_as = c->omega_as;
  for (int i = 0; i < 4; ++i) P.omega[i] = c->omega_j[i];
  P.inv_a0 = c->lv[level].inv_a0;
  P.half = c->cfg.local_half;
  P.colour = -1;
  return P;
}
}  // namespace pmg

namespace {


GeomDesc geom_desc(const pmg_ctx* c) {
  GeomDesc g{};
  g.kind = c->cfg.geometry == PMG_GEOM_DISTORTED ? 2 : (c->deformed ? 1 : 0);
  g.amp = c->cfg.deform_amp;
  g.verts = c->verts;
  g.n_fine = c->lv[c->L - 1].n;
  return g;
}

QuadTab make_tab(int p, int nq) {
  QuadTab t{};
  std::vector<double> w;
  auto x = host::gauss_points(nq, &w);
  auto nodes = host::gll_points(p);
  t.nq = nq;
  for (int q = 0; q < nq; ++q) {
    t.x[q] = x[q];
    t.w[q] = w[q];
    for (int a = 0; a <= p; ++a) {
      t.V[q * 12 + a] = host::lagrange(nodes, a, x[q]);
      t.D[q * 12 + a] = host::lagrange_deriv(nodes, a, x[q]);
    }
  }
  return t;
}

// r = b - A u (b != nullptr) or r = A u on mesh level `level`, precision prec.
// FP64 on a context with outer_apply FLOAT_FLOAT runs in float-float
// arithmetic, unless exact64 (the coarse-matrix assembly).
int level_apply(pmg_ctx* c, int level, int prec, const void* u, void* r, const void* b, bool exact64 = false) {
  LevelData& L = c->lv[level];
  cudaError_t e;
  if (prec == PMG_FP64 && !exact64 && c->cfg.outer_apply == PMG_OUTER_APPLY_FLOAT_FLOAT) {
    if (c->deformed)
      e = c->kt[PMG_FP64]->def_apply_ff(c->dim, (const double*)u, (double*)r, (const double*)b,
                                        (const float*)L.G[c->nplev - 1], L.n, c->def_cpb, c->stream);
    else
      e = c->kt[PMG_FP64]->cart_apply_ff(c->dim, (const double*)u, (double*)r, (const double*)b, c->t64[0],
                                         c->t64[1], c->t64[2], c->t64[3], L.n, L.scale, c->stream);
  } else if (c->deformed) {
    e = c->kt[prec]->def_apply(c->dim, prec, u, r, b, L.G[c->nplev - 1], c->cfg.geom_precision, c->cellbuf, L.n,
                               prec == c->mgprec ? c->def_cpb : 0, c->stream);
  } else {
    void** t = prec == PMG_FP64 ? (void**)c->t64 : c->t_mg;
    e = c->kt[prec]->cart_apply(c->dim, prec, u, r, b, t[0], t[1], t[2], t[3], L.n, L.scale, c->stream);
  }
  if (e != cudaSuccess) return fail(PMG_ERR_CUDA, std::string("apply: ") + cudaGetErrorString(e));
  return PMG_OK;
}

// The interleaved layout puts IL patches in one block: on levels with fewer
// than one such block per SM it would leave SMs idle, so when it was chosen
// by the autotuner those levels (the coarse ones) keep the patch-major
// layout with its smaller blocks.
bool use_interleaved(const pmg_ctx* c, int level, int colour) {
  if (c->il_threads <= 0) return false;
  if (c->cfg.patch_layout == PMG_PATCH_INTERLEAVED) return true;  // the caller's choice: every level
  const int il = c->km()->patch_il(c->dim, c->mgprec, c->cfg.local_cycles);
  return patch_count(c->dim, c->lv[level].n, colour) >= (int64_t)kNumSMs * il;
}

// Local solves of every patch of the level for the residual r, written to
// the patch buffer as omega_AS d_j (one launch).
int patch_solves(pmg_ctx* c, int level, const void* r, int colour = -1, void* u = nullptr) {
  LevelData& L = c->lv[level];
  PatchParamsHost P = patch_params(c, level);
  P.colour = colour;
  void* dst = colour < 0 ? c->pbuf : u;
  cudaError_t e;
  if (c->deformed) {
    DefLevel D{};
    for (int i = 0; i < 4; ++i) {
      D.G[i] = L.G[i];
      D.gprec = c->cfg.geom_precision;
      D.dinv[i] = L.dinv[i];
    }
    D.dinv1 = L.dinv1;
    e = c->km()->patch_def(c->dim, c->mgprec, r, dst, L.n, c->ppc, c->cfg.local_cycles, D, P, c->stream);
  } else if (use_interleaved(c, level, colour)) {
    e = c->km()->patch_cart_il(c->dim, c->mgprec, r, dst, L.n, c->il_threads, c->cfg.local_cycles, c->dtab_mg, P,
                               c->persistent ? c->work_counter : nullptr, c->stream);
  } else {
    e = c->km()->patch_cart(c->dim, c->mgprec, r, dst, L.n, c->ppc, c->cfg.local_cycles, c->dtab_mg, P,
                            c->persistent ? c->work_counter : nullptr, c->stream);
  }
  if (e != cudaSuccess) return fail(PMG_ERR_CUDA, std::string("patch smoother: ") + cudaGetErrorString(e));
  return PMG_OK;
}

// One additive sweep's correction: u (+)= omega_AS sum_j Pi_j^T V_j Pi_j r
// (add = false: u = that correction, the zero-initial-guess pre-smoothing).
int patch_sweep(pmg_ctx* c, int level, const void* r, void* u, bool add) {
  if (int rc = patch_solves(c, level, r)) return rc;
  cudaError_t e = c->km()->patch_gather(c->dim, c->mgprec, c->pbuf, u, c->lv[level].n, add ? 1 : 0, c->stream);
  if (e != cudaSuccess) return fail(PMG_ERR_CUDA, std::string("patch gather: ") + cudaGetErrorString(e));
  return PMG_OK;
}

// One multiplicative sweep (Algorithm 1) colour by colour: per parity colour
// the residual r = b - A u, then every patch of the colour adds its local
// solve to u (patches of a colour have disjoint interiors and none reads
// another's interior, so this is the sequential patch loop in colour-major
// order).  zero_guess: u starts at 0 and the first residual is b.
int mult_sweep(pmg_ctx* c, int level, const void* b, void* u, bool forward, bool zero_guess) {
  LevelData& L = c->lv[level];
  const int nc = 1 << c->dim;
  const size_t es = c->mg32 ? 4 : 8;
  if (zero_guess) PMG_CUDA(cudaMemsetAsync(u, 0, es * L.N, c->stream));
  for (int i = 0; i < nc; ++i) {
    const int colour = forward ? i : nc - 1 - i;
    const void* r = b;
    if (!(zero_guess && i == 0)) {
      if (int rc = level_apply(c, level, c->mgprec, u, L.r, b)) return rc;
      r = L.r;
    }
    if (int rc = patch_solves(c, level, r, colour, u)) return rc;
  }
  return PMG_OK;
}

int smooth_level(pmg_ctx* c, int level, const void* b, void* u, int sweeps, bool forward = true) {
  LevelData& L = c->lv[level];
  if (c->cfg.smoother == PMG_SMOOTHER_MULTIPLICATIVE) {
    for (int s = 0; s < sweeps; ++s)
      if (int rc = mult_sweep(c, level, b, u, forward, false)) return rc;
    return PMG_OK;
  }
  for (int s = 0; s < sweeps; ++s) {
    int rc = level_apply(c, level, c->mgprec, u, L.r, b);
    if (rc) return rc;
    rc = patch_sweep(c, level, L.r, u, true);
    if (rc) return rc;
  }
  return PMG_OK;
}

// z_l = B_l b_l from a zero guess (Eq. (1)-(4) V-cycle with additive patch
// smoothing), MG precision, vectors in the level buffers.
int vcycle_level(pmg_ctx* c, int level) {
  LevelData& L = c->lv[level];
  const size_t es = c->mg32 ? 4 : 8;
  if (level == 0) {
    cudaError_t e = coarse_solve(c->mgprec, c->ainv, c->cidx, c->plan.nc, L.b, L.u, L.N, c->stream);
    if (e != cudaSuccess) return fail(PMG_ERR_CUDA, std::string("coarse: ") + cudaGetErrorString(e));
    return PMG_OK;
  }
  (void)es;
  const int nu = c->cfg.smooth_steps;
  int rc;
  for (int s = 0; s < nu; ++s) {
    if (c->cfg.smoother == PMG_SMOOTHER_MULTIPLICATIVE) {
      rc = mult_sweep(c, level, L.b, L.u, true, s == 0);  // forward colours
    } else if (s == 0) {
      rc = patch_sweep(c, level, L.b, L.u, false);  // zero guess: the residual is b, u = S b
    } else {
      rc = smooth_level(c, level, L.b, L.u, 1);
    }
    if (rc) return rc;
  }
  if ((rc = level_apply(c, level, c->mgprec, L.u, L.r, L.b))) return rc;
  LevelData& C = c->lv[level - 1];
  cudaError_t e = c->km()->h_restrict(c->dim, c->mgprec, L.r, C.b, c->t_mg[0], c->t_mg[1], C.n, c->stream);
  if (e != cudaSuccess) return fail(PMG_ERR_CUDA, std::string("restrict: ") + cudaGetErrorString(e));
  if ((rc = vcycle_level(c, level - 1))) return rc;
  e = c->km()->h_prolong_add(c->dim, c->mgprec, C.u, L.u, c->t_mg[0], c->t_mg[1], C.n, c->stream);
  if (e != cudaSuccess) return fail(PMG_ERR_CUDA, std::string("prolongate: ") + cudaGetErrorString(e));
  // post-smoothing visits the colours backward: the V-cycle stays symmetric
  return smooth_level(c, level, L.b, L.u, nu, false);
}

// Inverses of Cartesian coarse matrices, shared by the contexts of a process:
// on the unit square/cube A_0 depends only on (dimension, degree, coarse
// cells n_0) -- not on the finest mesh -- so the set-up below runs once per
// (device, dim, degree, n_0, precision) and later contexts copy the inverse
// (the first solve of a served n_0 = 3, degree 5 request otherwise spends
// ~0.27 s assembling and inverting its 2,744 x 2,744 coarse matrix).  The
// cached buffers are device memory held until the process exits.
struct CoarseKey {
  int dev, dim, K, n0, prec;
  bool operator<(const CoarseKey& o) const {
    return std::tie(dev, dim, K, n0, prec) < std::tie(o.dev, o.dim, o.K, o.n0, o.prec);
  }
};
std::mutex g_coarse_mu;
std::map<CoarseKey, void*> g_coarse_cache;

// Coarsest level, set up before the first V-cycle: assemble A_0 on the free
// DoFs by applying the FP64 operator to unit vectors (one row per free DoF,
// A_0 being symmetric), invert it on the device (Gauss-Jordan, SPD so no
// pivoting), store the inverse in the MG precision; Cartesian inverses come
// from the process cache when an earlier context computed them.
}  // namespace

namespace pmg {
int ensure_coarse(pmg_ctx* c) {
  if (c->coarse_ready) return PMG_OK;
  if (!c->plan.coarse_ok)
    return fail(PMG_ERR_UNSUPPORTED, "coarsest level has more than 4096 free DoFs: no V-cycle or solve");
  LevelData& C = c->lv[0];
  const int N1 = C.N1;
  std::vector<int> idx;
  for (int64_t g = 0; g < C.N; ++g) {
    const int x = (int)(g % N1), y = (int)((g / N1) % N1), z = c->dim == 3 ? (int)(g / ((int64_t)N1 * N1)) : 1;
    if (x > 0 && x < N1 - 1 && y > 0 && y < N1 - 1 && (c->dim == 2 || (z > 0 && z < N1 - 1))) idx.push_back((int)g);
  }
  const int nc = (int)idx.size();
  if (nc != c->plan.nc) return fail(PMG_ERR_STATE, "coarse size mismatch");
  const size_t inv_bytes = (size_t)nc * nc * (c->mg32 ? 4 : 8);
  int dev = 0;
  PMG_CUDA(cudaGetDevice(&dev));
  const CoarseKey ckey{dev, c->dim, c->K, c->plan.n0, c->mgprec};
  if (!c->deformed && nc > 0) {
    std::lock_guard<std::mutex> g(g_coarse_mu);
    auto it = g_coarse_cache.find(ckey);
    if (it != g_coarse_cache.end()) {
      PMG_CUDA(cudaMemcpyAsync(c->cidx, idx.data(), 4 * nc, cudaMemcpyHostToDevice, c->stream));
      PMG_CUDA(cudaMemcpyAsync(c->ainv, it->second, inv_bytes, cudaMemcpyDeviceToDevice, c->stream));
      PMG_CUDA(cudaStreamSynchronize(c->stream));  // idx is a host temporary
      c->coarse_ready = true;
      return PMG_OK;
    }
  }
  if (nc > 0) {
    double* A = (double*)at(c, c->plan.a64);
    double* xd = (double*)at(c, c->plan.cx0);  // dedicated: the CG vectors may be live here
    double* yd = (double*)at(c, c->plan.cy0);
    int* bad = (int*)at(c, c->plan.gjbad);
    PMG_CUDA(cudaMemcpyAsync(c->cidx, idx.data(), 4 * nc, cudaMemcpyHostToDevice, c->stream));
    PMG_CUDA(cudaMemsetAsync(bad, 0, 4, c->stream));
    for (int j = 0; j < nc; ++j) {
      PMG_CUDA(coarse_unit(xd, C.N, idx[j], c->stream));
      int rc = level_apply(c, 0, PMG_FP64, xd, yd, nullptr, true);
      if (rc) return rc;
      PMG_CUDA(coarse_gather_row(yd, c->cidx, nc, A, j, c->stream));
    }
    PMG_CUDA(coarse_invert(A, nc, (double*)at(c, c->plan.gjrow), (double*)at(c, c->plan.gjcol), bad, c->ainv,
                           c->mgprec, c->stream));
    int hbad = 0;
    PMG_CUDA(cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, c->stream));
    PMG_CUDA(cudaStreamSynchronize(c->stream));
    if (hbad) return fail(PMG_ERR_STATE, "coarse matrix is not positive definite");
    if (!c->deformed) {
      std::lock_guard<std::mutex> g(g_coarse_mu);
      if (!g_coarse_cache.count(ckey)) {
        void* buf = nullptr;
        if (cudaMalloc(&buf, inv_bytes) == cudaSuccess) {
          cudaError_t e = cudaMemcpyAsync(buf, c->ainv, inv_bytes, cudaMemcpyDeviceToDevice, c->stream);
          if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
          if (e == cudaSuccess) g_coarse_cache[ckey] = buf;
          else cudaFree(buf);
        }
        cudaGetLastError();  // a failed cache insertion leaves this context correct
      }
    }
  }
  c->coarse_ready = true;
  return PMG_OK;
}
}  // namespace pmg

namespace {


// Capture the finest-level V-cycle once as a CUDA graph.
int ensure_vgraph(pmg_ctx* c) {
  if (c->vgraph) return PMG_OK;
  if (int rc = ensure_coarse(c)) return rc;
  cudaGraph_t g = nullptr;
  const int64_t before = g_launches.load();
  PMG_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  int rc = vcycle_level(c, c->L - 1);
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  const int64_t n = g_launches.load() - before;
  g_launches -= n;  // captured, not launched
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(PMG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&c->vgraph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(PMG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  c->vgraph_launches = n;
  return PMG_OK;
}

// z = B r for FP64 device vectors r, z on the finest level.
int precondition(pmg_ctx* c, const double* r, double* z) {
  LevelData& F = c->lv[c->L - 1];
  int rc = ensure_vgraph(c);
  if (rc) return rc;
  if (c->mg32) {
    PMG_CUDA(cast_d2f(r, (float*)F.b, F.N, c->stream));
  } else {
    PMG_CUDA(cudaMemcpyAsync(F.b, r, 8 * F.N, cudaMemcpyDeviceToDevice, c->stream));
  }
  PMG_CUDA(cudaGraphLaunch(c->vgraph, c->stream));
  g_launches += c->vgraph_launches;
  if (c->mg32) {
    PMG_CUDA(cast_f2d((const float*)F.u, z, F.N, c->stream));
  } else {
    PMG_CUDA(cudaMemcpyAsync(z, F.u, 8 * F.N, cudaMemcpyDeviceToDevice, c->stream));
  }
  return PMG_OK;
}

// ---------------------------------------------------------------- autotuner
// Shared-memory layout and block shape of the smoother's patch kernel, per
// (dim, degree, MG precision, geometry, local cycles, smoother, finest n):
// the patch-major layout with 1..64 patches per block, and (Cartesian) the
// interleaved layout with 128..1024 threads per block.  Every admissible
// candidate is timed on the patch launches of one finest-level sweep -- the
// one launch over all patches (additive) or the 2^d colour launches
// (multiplicative, each over an eighth of the patches in 3D, where the last
// wave matters) -- with CUDA events, best of 3 after a warm-up (fewer for
// long or clearly slower launches, see time_of), and the fastest is kept
// for the process; with PMG_TUNE_FILE set, results are also
// read from and appended to that file ("dim k prec geom cycles smoother n
// layout ppc threads persistent" per line).  The fastest candidate is then
// timed once more as a persistent grid (Cartesian), kept if faster.  Small meshes, whose launches are too short
// to time, use a rule (interleaved with 256 threads where available, else
// about 256 threads of patch-major patches) without caching it.
struct TuneKey {
  int dim, K, prec, geom, cycles, smoother, n;
  bool operator<(const TuneKey& o) const {
    return std::tie(dim, K, prec, geom, cycles, smoother, n) <
           std::tie(o.dim, o.K, o.prec, o.geom, o.cycles, o.smoother, o.n);
  }
};
struct TuneVal {
  int layout, ppc, threads, persistent;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;
bool g_tune_file_read = false;

void tune_file_read_locked() {
  if (g_tune_file_read) return;
  g_tune_file_read = true;
  const char* path = std::getenv("PMG_TUNE_FILE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[256];
  while (std::fgets(line, sizeof(line), f)) {
    TuneKey k{};
    TuneVal v{};
    if (std::sscanf(line, "%d %d %d %d %d %d %d %d %d %d %d", &k.dim, &k.K, &k.prec, &k.geom, &k.cycles,
                    &k.smoother, &k.n, &v.layout, &v.ppc, &v.threads, &v.persistent) == 11)
      g_tune[k] = v;
  }
  std::fclose(f);
}

void tune_file_append_locked(const TuneKey& k, const TuneVal& v) {
  const char* path = std::getenv("PMG_TUNE_FILE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%d %d %d %d %d %d %d %d %d %d %d\n", k.dim, k.K, k.prec, k.geom, k.cycles, k.smoother, k.n,
               v.layout, v.ppc, v.threads, v.persistent);
  std::fclose(f);
}

int admissible_ppc(const pmg_ctx* c, int ppc) {
  const int tpp = c->deformed ? c->km()->patch_def_threads(c->dim) : c->km()->patch_threads(c->dim);
  const int smem = c->deformed ? c->km()->patch_def_smem(c->dim, c->mgprec, c->cfg.local_cycles)
                               : c->km()->patch_smem(c->dim, c->mgprec, c->cfg.local_cycles);
  const int maxt = c->km()->patch_max_threads(c->dim, c->mgprec, c->deformed ? 1 : 0);
  const int extra = c->deformed ? 0 : c->km()->patch_cart_extra_smem(c->dim, c->mgprec);
  return ppc >= 1 && ppc <= 64 && (ppc * tpp + 31) / 32 * 32 <= std::min(1024, maxt) &&
         ppc * smem + extra <= kMaxDynSmem;
}

// the interleaved layout exists for this context and admits `threads`
int admissible_il(const pmg_ctx* c, int threads) {
  if (c->deformed || c->km()->patch_il(c->dim, c->mgprec, c->cfg.local_cycles) == 0) return 0;
  return threads >= 32 && threads % 32 == 0 && threads <= c->km()->patch_il_max_threads(c->dim, c->mgprec);
}

}  // namespace

namespace pmg {
int rule_ppc(const pmg_ctx* c) {
  const int tpp = c->deformed ? c->km()->patch_def_threads(c->dim) : c->km()->patch_threads(c->dim);
  int ppc = std::max(1, 256 / tpp);
  while (ppc > 1 && !admissible_ppc(c, ppc)) --ppc;
  return ppc;
}
}  // namespace pmg

namespace {


void set_layout(pmg_ctx* c, const TuneVal& v) {
  c->ppc = v.ppc;
  c->il_threads = v.layout == PMG_PATCH_INTERLEAVED ? v.threads : 0;
  c->persistent = v.persistent != 0;
}

int choose_patch_layout(pmg_ctx* c) {
  const pmg_config& cf = c->cfg;
  if (!admissible_ppc(c, 1)) return fail(PMG_ERR_UNSUPPORTED, "patch does not fit in shared memory for this degree");
  int layout = cf.patch_layout;
  if (layout == PMG_PATCH_AUTO && cf.patches_per_block > 0) layout = PMG_PATCH_MAJOR;
  if (layout == PMG_PATCH_INTERLEAVED && !admissible_il(c, 32))
    return fail(PMG_ERR_UNSUPPORTED, "no interleaved patch layout for this configuration (deformed geometry, or "
                                     "the interleaved patches do not fit in shared memory)");
  c->ppc = rule_ppc(c);
  c->il_threads = 0;
  c->persistent = cf.patch_persistent > 0 && !c->deformed;
  if (layout == PMG_PATCH_MAJOR && cf.patches_per_block > 0) {
    if (!admissible_ppc(c, cf.patches_per_block)) return fail(PMG_ERR_ARG, "patches_per_block not admissible");
    c->ppc = cf.patches_per_block;
    return PMG_OK;
  }
  if (layout == PMG_PATCH_INTERLEAVED && cf.patch_threads > 0) {
    if (!admissible_il(c, cf.patch_threads)) return fail(PMG_ERR_ARG, "patch_threads not admissible");
    c->il_threads = cf.patch_threads;
    return PMG_OK;
  }
  const bool try_major = layout != PMG_PATCH_INTERLEAVED;
  const bool try_il = layout != PMG_PATCH_MAJOR && admissible_il(c, 256);
  if (try_il) c->il_threads = 256;  // rule for meshes too small to time
  LevelData& F = c->lv[c->L - 1];
  const int64_t patches = ipow64(std::max(F.n - 1, 0), c->dim);
  if (c->K == 1 || patches < 4096) return PMG_OK;
  const bool mult = cf.smoother == PMG_SMOOTHER_MULTIPLICATIVE;
  const TuneKey key{c->dim, c->K, c->mgprec, c->deformed ? 1 : 0, cf.local_cycles, mult ? 1 : 0, F.n};
  auto valid = [&](const TuneVal& v) {
    return v.layout == PMG_PATCH_INTERLEAVED ? try_il && admissible_il(c, v.threads)
                                             : try_major && admissible_ppc(c, v.ppc);
  };
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_file_read_locked();
    auto it = g_tune.find(key);
    if (it != g_tune.end() && valid(it->second)) {
      TuneVal v = it->second;
      if (cf.patch_persistent != 0) v.persistent = cf.patch_persistent > 0 && !c->deformed;
      set_layout(c, v);
      return PMG_OK;
    }
  }
  std::vector<TuneVal> cand;
  const int tpp = c->deformed ? c->km()->patch_def_threads(c->dim) : c->km()->patch_threads(c->dim);
  if (try_major)
    for (int ppc = 1; ppc <= 64; ++ppc) {
      if (!admissible_ppc(c, ppc)) continue;
      const int thr = ppc * tpp, padded = (thr + 31) / 32 * 32;
      if (ppc > 2 && thr < 0.85 * padded) continue;  // warps with many idle lanes: not worth timing
      cand.push_back({PMG_PATCH_MAJOR, ppc, 0, 0});
    }
  if (try_il)
    for (int t : {128, 192, 256, 320, 384, 448, 512, 640, 768, 896, 1024})
      if (admissible_il(c, t)) cand.push_back({PMG_PATCH_INTERLEAVED, c->ppc, t, 0});
  const size_t es = c->mg32 ? 4 : 8;
  PMG_CUDA(cudaMemsetAsync(F.r, 0, es * F.N, c->stream));
  PMG_CUDA(cudaMemsetAsync(F.u, 0, es * F.N, c->stream));
  cudaEvent_t e0, e1;
  PMG_CUDA(cudaEventCreate(&e0));
  PMG_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  TuneVal best_v{c->il_threads > 0 ? PMG_PATCH_INTERLEAVED : PMG_PATCH_MAJOR, c->ppc, c->il_threads, 0};
  const int64_t before = g_launches.load();
  // best of 3 timed repetitions after a warm-up (one when the warm-up took
  // over 2 ms: launches that long time reproducibly, and the set-up of a
  // large context is on its first request's critical path; none when the
  // warm-up took 1.5x the best time so far); 1e30 if the device rejects a
  // launch (resources): not a candidate
  auto time_of = [&](const TuneVal& v) -> float {
    set_layout(c, v);
    float tmin = 1e30f;
    int reps = 4;
    for (int rep = 0; rep < reps; ++rep) {
      cudaEventRecord(e0, c->stream);
      int rc = PMG_OK;
      if (mult) {
        for (int col = 0; col < (1 << c->dim) && !rc; ++col) rc = patch_solves(c, c->L - 1, F.r, col, F.u);
      } else {
        rc = patch_solves(c, c->L - 1, F.r);
      }
      cudaEventRecord(e1, c->stream);
      if (rc) {
        cudaGetLastError();
        return 1e30f;
      }
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tmin = std::min(tmin, ms);
      else if (ms > 1.5f * best) return ms;  // far behind the best so far: not timed further
      else if (ms > 2.f) reps = 2;
    }
    return tmin;
  };
  for (const TuneVal& v : cand) {
    const float t = time_of(v);
    if (t < best * 0.995f) {
      best = t;
      best_v = v;
    }
  }
  if (!c->deformed && cf.patch_persistent == 0) {  // the winner as a persistent grid, kept if faster
    TuneVal pv = best_v;
    pv.persistent = 1;
    if (time_of(pv) < best * 0.995f) best_v = pv;
  }
  g_launches -= g_launches.load() - before;  // tuning launches are not the caller's work
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cf.patch_persistent != 0) best_v.persistent = cf.patch_persistent > 0 && !c->deformed;
  set_layout(c, best_v);
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_tune[key] = best_v;
  tune_file_append_locked(key, best_v);
  return PMG_OK;
}

// Cells per block of the deformed operator apply in the multigrid precision
// (the residuals of every smoothing step), per (dim, degree, precision,
// geometry storage, finest n): each admissible value is timed on the finest
// level's apply, best of 3 after a warm-up, and kept for the process; meshes
// below 32^3 cells (2D: 256^2) use the kernel part's rule.  The float-float
// outer operator uses the same value.
struct DefTuneKey {
  int dim, K, prec, gprec, n;
  bool operator<(const DefTuneKey& o) const {
    return std::tie(dim, K, prec, gprec, n) < std::tie(o.dim, o.K, o.prec, o.gprec, o.n);
  }
};
std::map<DefTuneKey, int> g_def_tune;

int choose_def_cpb(pmg_ctx* c) {
  c->def_cpb = 0;
  if (!c->deformed) return PMG_OK;
  if (c->cfg.apply_cells_per_block > 0) {  // the caller's value, if the part admits it
    int cand[16];
    const int nc = c->km()->def_apply_candidates(c->dim, c->mgprec, c->cfg.geom_precision, cand, 16);
    for (int i = 0; i < nc; ++i)
      if (cand[i] == c->cfg.apply_cells_per_block) {
        c->def_cpb = cand[i];
        return PMG_OK;
      }
    return fail(PMG_ERR_ARG, "apply_cells_per_block not admissible for this configuration");
  }
  LevelData& F = c->lv[c->L - 1];
  const int64_t cells = ipow64(F.n, c->dim);
  if (cells < (c->dim == 3 ? 32768 : 65536)) return PMG_OK;
  const DefTuneKey key{c->dim, c->K, c->mgprec, c->cfg.geom_precision, F.n};
  {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_def_tune.find(key);
    if (it != g_def_tune.end()) {
      c->def_cpb = it->second;
      return PMG_OK;
    }
  }
  int cand[16];
  const int nc = c->km()->def_apply_candidates(c->dim, c->mgprec, c->cfg.geom_precision, cand, 16);
  cudaEvent_t e0, e1;
  PMG_CUDA(cudaEventCreate(&e0));
  PMG_CUDA(cudaEventCreate(&e1));
  const size_t es = c->mg32 ? 4 : 8;
  PMG_CUDA(cudaMemsetAsync(F.u, 0, es * F.N, c->stream));
  const int64_t before = g_launches.load();
  float best = 1e30f;
  int best_cpb = 0;
  for (int i = 0; i < nc; ++i) {
    c->def_cpb = cand[i];
    float tmin = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(e0, c->stream);
      const int rc = level_apply(c, c->L - 1, c->mgprec, F.u, F.r, nullptr);
      cudaEventRecord(e1, c->stream);
      if (rc) {
        cudaGetLastError();
        tmin = 1e30f;
        break;
      }
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tmin = std::min(tmin, ms);
    }
    if (tmin < best * 0.995f) {
      best = tmin;
      best_cpb = cand[i];
    }
  }
  g_launches -= g_launches.load() - before;  // tuning launches are not the caller's work
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->def_cpb = best_cpb;
  std::lock_guard<std::mutex> g(g_tune_mu);
  g_def_tune[key] = best_cpb;
  return PMG_OK;
}

}  // namespace

namespace pmg {
int check_ctx(const pmg_ctx* c) { return c ? PMG_OK : fail(PMG_ERR_ARG, "context is NULL"); }
}  // namespace pmg

namespace {


// omega_AS reading: theta / 2^d with theta = 1.5 (every free DoF lies in at
// most 2^d patch interiors)
double default_omega_patch(int dim) { return 1.5 / (1 << dim); }

// Pinned host copies of the solver scalars (S_COUNT doubles per context),
// carved from page-locked slabs that live for the process: cudaMallocHost
// and cudaFreeHost per context would cost more than the rest of a small
// context's set-up.
std::mutex g_pin_mu;
std::vector<double*> g_pin_free;

double* pinned_scalars_get() {
  std::lock_guard<std::mutex> g(g_pin_mu);
  if (g_pin_free.empty()) {
    constexpr int kPerSlab = 256;
    double* slab = nullptr;
    if (cudaMallocHost((void**)&slab, sizeof(double) * S_COUNT * kPerSlab) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    for (int i = kPerSlab - 1; i >= 0; --i) g_pin_free.push_back(slab + (size_t)i * S_COUNT);
  }
  double* p = g_pin_free.back();
  g_pin_free.pop_back();
  return p;
}

void pinned_scalars_put(double* p) {
  std::lock_guard<std::mutex> g(g_pin_mu);
  g_pin_free.push_back(p);
}

int setup_context(pmg_ctx* c) {
  const Plan& P = c->plan;
  c->lv.resize(c->L);
  for (int l = 0; l < c->L; ++l) {
    LevelData& D = c->lv[l];
    D.n = P.ns[l];
    D.N1 = c->K * D.n + 1;
    D.N = ipow64(D.N1, c->dim);
    D.b = at(c, P.lo[l].b);
    D.u = at(c, P.lo[l].u);
    D.r = at(c, P.lo[l].r);
    const double h = 1.0 / D.n;
    D.scale = std::pow(h, c->dim - 2);
    // Cartesian A_{j,1} = h^{d-2} d (2) (2/3)^{d-1}
    D.inv_a0 = 1.0 / (D.scale * c->dim * 2.0 * std::pow(2.0 / 3.0, c->dim - 1));
    for (int i = 0; i < 4; ++i) {
      D.G[i] = at(c, P.lo[l].G[i]);
      D.dinv[i] = at(c, P.lo[l].dinv[i]);
    }
    D.dinv1 = at(c, P.lo[l].dinv1);
  }
  for (int i = 0; i < 4; ++i) {
    c->t64[i] = (double*)at(c, P.t64[i]);
    c->t_mg[i] = at(c, P.t_mg[i]);
  }
  if (P.m > 0) {
    c->gmres = true;
    c->gm = P.m;
    c->gld = c->lv[c->L - 1].N;
    c->gv = (double*)at(c, P.gv);
    c->gz = (double*)at(c, P.gz);
    c->gh = (double*)at(c, P.gh);
    c->gs = (double*)at(c, P.gs);
    c->gpart = (double*)at(c, P.gpart);
  }
  double** cg[6] = {&c->cg_x, &c->cg_r, &c->cg_p, &c->cg_Ap, &c->cg_z, &c->cg_b};
  for (int i = 0; i < 6; ++i) *cg[i] = (double*)at(c, P.cg[i]);
  c->scal = (double*)at(c, P.scal);
  c->partial = (double*)at(c, P.partial);
  c->dtab64 = (double*)at(c, P.dtab64);
  c->dtab32 = (float*)at(c, P.dtab32);
  c->dtab_mg = c->mg32 ? (void*)c->dtab32 : (void*)c->dtab64;
  c->cidx = (int*)at(c, P.cidx);
  c->ainv = at(c, P.ainv);
  c->pbuf = at(c, P.pbuf);
  c->work_counter = (int*)at(c, P.counter);
  c->cellbuf = at(c, P.cellbuf);
  c->verts = (double*)at(c, P.verts);

  // coefficients and kernel attributes: once per device and kernel part
  // (module state that every context of the part shares)
  std::vector<double> coef(kMaxCoef, 0.0);
  host::fill_coefficients(c->K, coef.data());
  {
    static std::mutex mu;
    static std::set<std::pair<int, const KernelTable*>> ready;
    int dev = 0;
    PMG_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> g(mu);
    for (const KernelTable* t : c->kt) {
      if (ready.count({dev, t})) continue;
      PMG_CUDA(t->prepare());
      PMG_CUDA(t->upload(coef.data()));
      ready.insert({dev, t});
    }
  }

  // damping
  const pmg_config& cf = c->cfg;
  c->omega_as = cf.omega_patch > 0 ? cf.omega_patch : default_omega_patch(c->dim);
  for (int l = 0; l < 4; ++l) {
    if (l < c->nplev && l > 0)
      c->omega_j[l] = cf.omega_jacobi[l] > 0 ? cf.omega_jacobi[l]
                                             : host::default_omega_jacobi(c->dim, plev(c->K, l));
    else
      c->omega_j[l] = 1.0;
  }

  // Cartesian scale-free inverse diagonal tables of the patch operators
  {
    const CoefLayout LA = coef_layout(c->K);
    std::vector<double> t64;
    for (int pl = 1; pl < c->nplev; ++pl) {
      const int m = mp(plev(c->K, pl));
      const int64_t S = ipow64(m, c->dim);
      for (int64_t i = 0; i < S; ++i) {
        const int ii[3] = {(int)(i % m), (int)((i / m) % m), c->dim == 3 ? (int)(i / (m * m)) : 0};
        double s = 0.0;
        for (int dir = 0; dir < c->dim; ++dir) {
          double t = 1.0;
          for (int dd = 0; dd < c->dim; ++dd)
            t *= dd == dir ? coef[LA.dK[pl] + ii[dd]] : coef[LA.dM[pl] + ii[dd]];
          s += t;
        }
        t64.push_back(1.0 / s);
      }
    }
    if (!t64.empty()) {
      std::vector<float> t32(t64.begin(), t64.end());
      PMG_CUDA(cudaMemcpyAsync(c->dtab64, t64.data(), 8 * t64.size(), cudaMemcpyHostToDevice, c->stream));
      PMG_CUDA(cudaMemcpyAsync(c->dtab32, t32.data(), 4 * t32.size(), cudaMemcpyHostToDevice, c->stream));
      PMG_CUDA(cudaStreamSynchronize(c->stream));
    }
  }

  // deformed geometry: G_q per level and p-level, inverse diagonals
  if (c->deformed) {
    int* geobad = (int*)at(c, c->plan.gjbad);  // free until the coarse set-up
    PMG_CUDA(cudaMemsetAsync(geobad, 0, sizeof(int), c->stream));
    if (c->verts) {
      // vertex positions of the finest mesh: reference position + displacement
      const int nf = c->lv[c->L - 1].n, nv = nf + 1;
      const int64_t NV = ipow64(nv, c->dim);
      std::vector<double> pos((size_t)(NV * c->dim));
      for (int64_t v = 0; v < NV; ++v) {
        int64_t t = v;
        for (int m = 0; m < c->dim; ++m) {
          pos[v * c->dim + m] = (double)(t % nv) / nf + cf.vertex_disp[v * c->dim + m];
          t /= nv;
        }
      }
      PMG_CUDA(cudaMemcpyAsync(c->verts, pos.data(), 8 * pos.size(), cudaMemcpyHostToDevice, c->stream));
      PMG_CUDA(cudaStreamSynchronize(c->stream));
    }
    for (int l = 0; l < c->L; ++l) {
      LevelData& D = c->lv[l];
      for (int pl = 0; pl < c->nplev; ++pl) {
        if (!D.G[pl]) continue;
        const int p = plev(c->K, pl);
        PMG_CUDA(compute_geometry(c->dim, D.n, p, geom_desc(c), make_tab(p, p + 1), D.G[pl], c->cfg.geom_precision,
                                  geobad, c->stream));
        if (D.dinv[pl])
          PMG_CUDA(compute_inverse_diagonal(c->dim, D.n, p, make_tab(p, p + 1), D.G[pl], c->cfg.geom_precision,
                                            c->t64[0], D.dinv[pl],
                                            c->mgprec, c->stream));
      }
      if (D.dinv1)
        PMG_CUDA(compute_inverse_diagonal(c->dim, D.n, 1, make_tab(1, 2), D.G[0], c->cfg.geom_precision, c->t64[0],
                                          D.dinv1, c->mgprec,
                                          c->stream));
    }
    int bad = 0;
    PMG_CUDA(cudaMemcpyAsync(&bad, geobad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PMG_CUDA(cudaStreamSynchronize(c->stream));
    if (bad) return fail(PMG_ERR_ARG, "inverted cell: det J <= 0 at a quadrature point of the mesh");
  }

  // patch-kernel layout and block shape: the autotuned choice (or the caller's)
  if (int rc = choose_patch_layout(c)) return rc;
  if (int rc = choose_def_cpb(c)) return rc;

  c->host_scal = pinned_scalars_get();
  if (!c->host_scal) return fail(PMG_ERR_OOM, "cudaMallocHost failed");
  PMG_CUDA(cudaEventCreateWithFlags(&c->ev_rr, cudaEventDisableTiming));
  PMG_CUDA(cudaEventCreate(&c->ev0));
  PMG_CUDA(cudaEventCreate(&c->ev1));
  PMG_CUDA(cudaEventCreateWithFlags(&c->ev_done, cudaEventDisableTiming));
  PMG_CUDA(cudaStreamSynchronize(c->stream));
  return PMG_OK;
}

}  // namespace

extern "C" {

void pmg_config_default(pmg_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->dim = 3;
  cfg->n_cells = 8;
  cfg->degree = 2;
  cfg->n_levels = 0;
  cfg->geometry = PMG_GEOM_CARTESIAN;
  cfg->deform_amp = 0.05;
  cfg->mg_precision = PMG_FP64;
  cfg->omega_patch = 0;
  cfg->local_cycles = 1;
  cfg->smooth_steps = 1;
  cfg->patches_per_block = 0;
  cfg->local_half = 0;
  cfg->outer_solver = PMG_OUTER_CG;
  cfg->gmres_restart = 30;
  cfg->smoother = PMG_SMOOTHER_ADDITIVE;
  cfg->vertex_disp = nullptr;
  cfg->patch_layout = PMG_PATCH_AUTO;
  cfg->patch_threads = 0;
  cfg->outer_apply = PMG_OUTER_APPLY_FP64;
  cfg->geom_precision = PMG_FP32;
  cfg->apply_cells_per_block = 0;
  cfg->patch_persistent = 0;
  cfg->coarse_dofs = 0;
}

int pmg_bytes_required(const pmg_config* cfg, int64_t* bytes) {
  if (!bytes) return fail(PMG_ERR_ARG, "bytes is NULL");
  Plan P;
  int rc = make_plan(cfg, P);
  if (rc) return rc;
  *bytes = P.total;
  return PMG_OK;
}

int pmg_create(const pmg_config* cfg, void* stream, void* workspace, int64_t workspace_bytes, pmg_ctx** out) {
  if (!out) return fail(PMG_ERR_ARG, "out is NULL");
  *out = nullptr;
  static std::atomic<uint64_t> next_uid{1};
  pmg_ctx* c = new pmg_ctx();
  c->uid = next_uid++;
  int rc = make_plan(cfg, c->plan);
  if (rc) {
    delete c;
    return rc;
  }
  c->cfg = *cfg;
  c->dim = cfg->dim;
  c->K = cfg->degree;
  c->L = c->plan.nlev;
  c->nplev = c->plan.nplev;
  c->deformed = c->plan.deformed;
  c->mg32 = c->plan.mg32;
  c->mgprec = cfg->mg_precision;
  c->stream = (cudaStream_t)stream;
  if (!c->stream) {
    // the legacy default stream cannot be captured into a CUDA graph: use a
    // blocking stream of our own, which still orders against it
    cudaError_t e = cudaStreamCreate(&c->stream);
    if (e != cudaSuccess) {
      delete c;
      return fail(PMG_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    c->own_stream = true;
  }
  c->kt[0] = kernel_table(c->K, c->dim, PMG_FP64);
  c->kt[1] = kernel_table(c->K, c->dim, PMG_FP32);
  if (workspace) {
    if (workspace_bytes < c->plan.total) {
      delete c;
      return fail(PMG_ERR_OOM, "workspace smaller than pmg_bytes_required");
    }
    if ((uintptr_t)workspace % kAlign) {
      delete c;
      return fail(PMG_ERR_ARG, "workspace must be 256-byte aligned");
    }
    c->ws = (char*)workspace;
  } else {
    cudaError_t e = cudaMalloc((void**)&c->ws, c->plan.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return fail(PMG_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    c->own_ws = true;
  }
  rc = setup_context(c);
  if (rc) {
    pmg_destroy(c);
    return rc;
  }
  *out = c;
  return PMG_OK;
}

int pmg_destroy(pmg_ctx* c) {
  if (!c) return PMG_OK;
  if (c->group) return fail(PMG_ERR_STATE, "the context is part of a grouped solve");
  if (c->vgraph) cudaGraphExecDestroy(c->vgraph);
  if (c->ev_rr) cudaEventDestroy(c->ev_rr);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->ev_done) cudaEventDestroy(c->ev_done);
  if (c->host_scal) pinned_scalars_put(c->host_scal);
  if (c->own_ws && c->ws) cudaFree(c->ws);
  if (c->own_stream && c->stream) {
    cudaStreamSynchronize(c->stream);
    cudaStreamDestroy(c->stream);
  }
  delete c;
  return PMG_OK;
}

int pmg_num_levels(const pmg_ctx* c, int* n) {
  if (check_ctx(c) || !n) return fail(PMG_ERR_ARG, "NULL argument");
  *n = c->L;
  return PMG_OK;
}

int pmg_num_dofs(const pmg_ctx* c, int level, int64_t* n) {
  if (check_ctx(c) || !n) return fail(PMG_ERR_ARG, "NULL argument");
  if (level < 0 || level >= c->L) return fail(PMG_ERR_ARG, "level out of range");
  *n = c->lv[level].N;
  return PMG_OK;
}

static int check_prec(const pmg_ctx* c, int prec) {
  if (prec != PMG_FP64 && prec != PMG_FP32) return fail(PMG_ERR_ARG, "unknown precision");
  if (prec == PMG_FP32 && !c->mg32) return fail(PMG_ERR_ARG, "FP32 calls need a context with mg_precision FP32");
  return PMG_OK;
}

int pmg_apply(pmg_ctx* c, int level, int prec, const void* x, void* y) {
  if (check_ctx(c) || !x || !y) return fail(PMG_ERR_ARG, "NULL argument");
  if (level < 0 || level >= c->L) return fail(PMG_ERR_ARG, "level out of range");
  if (int rc = check_prec(c, prec)) return rc;
  return level_apply(c, level, prec, x, y, nullptr);
}

int pmg_residual(pmg_ctx* c, int level, int prec, const void* b, const void* u, void* r) {
  if (check_ctx(c) || !b || !u || !r) return fail(PMG_ERR_ARG, "NULL argument");
  if (level < 0 || level >= c->L) return fail(PMG_ERR_ARG, "level out of range");
  if (int rc = check_prec(c, prec)) return rc;
  return level_apply(c, level, prec, u, r, b);
}

// A level can be smoothed when it has patches (n >= 2) and its smoother
// data: every level but the coarsest of a hierarchy, the coarsest too when
// Cartesian (the patch operators need no stored data), and the only level of
// a single-level context.
static int check_smooth_level(const pmg_ctx* c, int level) {
  if (level < 0 || level >= c->L) return fail(PMG_ERR_ARG, "level out of range");
  if (c->lv[level].n < 2) return fail(PMG_ERR_ARG, "level has no interior vertex (n < 2): no patches to smooth");
  if (level == 0 && c->L > 1 && c->deformed)
    return fail(PMG_ERR_ARG, "the coarsest level of a deformed hierarchy holds no smoother data");
  return PMG_OK;
}

int pmg_smooth(pmg_ctx* c, int level, int prec, const void* b, void* u, int sweeps) {
  if (check_ctx(c) || !b || !u) return fail(PMG_ERR_ARG, "NULL argument");
  if (int rc = check_smooth_level(c, level)) return rc;
  if (prec != c->mgprec) return fail(PMG_ERR_ARG, "smoother precision must equal mg_precision");
  if (sweeps < 0) return fail(PMG_ERR_ARG, "sweeps < 0");
  return smooth_level(c, level, b, u, sweeps);
}

int pmg_vcycle(pmg_ctx* c, const double* r, double* z) {
  if (check_ctx(c) || !r || !z) return fail(PMG_ERR_ARG, "NULL argument");
  return precondition(c, r, z);
}

// ---------------------------------------------------------------- PCG
}  // extern "C"

namespace pmg {

// The solve is a state machine so that a server can interleave many
// contexts: every step enqueues device work and records an event; the host
// only reads ||r||^2 once the event has completed, while the preconditioner
// of the next iteration is already enqueued behind it.

static int enqueue_iteration(pmg_ctx* c) {
  const int64_t N = c->lv[c->L - 1].N;
  cudaStream_t s = c->stream;
  if (int rc = level_apply(c, c->L - 1, PMG_FP64, c->cg_p, c->cg_Ap, nullptr)) return rc;
  PMG_CUDA(dot(c->cg_p, c->cg_Ap, N, c->partial, c->scal + S_PAP, s));
  PMG_CUDA(cg_update_xr(c->cg_x, c->cg_r, c->cg_p, c->cg_Ap, N, c->scal, S_RZ, S_PAP, c->partial, c->scal + S_RR, s));
  PMG_CUDA(cudaMemcpyAsync(c->host_scal + S_RR, c->scal + S_RR, 8, cudaMemcpyDeviceToHost, s));
  PMG_CUDA(cudaEventRecord(c->ev_rr, s));
  ++c->sv.it;
  // the next preconditioner step goes in before the host looks at ||r||
  if (int rc = precondition(c, c->cg_r, c->cg_z)) return rc;
  PMG_CUDA(dot(c->cg_r, c->cg_z, N, c->partial, c->scal + S_RZN, s));
  PMG_CUDA(cg_update_p(c->cg_p, c->cg_z, N, c->scal, S_RZN, S_RZ, 0, s));
  return PMG_OK;
}

// ---------------------------------------------------------------- GMRES
// Flexible right-preconditioned GMRES(m) (the paper's outer solver, needed
// with the half local V-cycle, §3.2.2): each step z_j = B v_j (V-cycle),
// w = A z_j, two classical Gram-Schmidt passes against v_0..v_j (one
// multi-dot and one multi-axpy each), ||w||, the Givens update of the
// Hessenberg column on the device, v_{j+1} = w / ||w||; the host reads only
// the residual estimate |g_{j+1}| while the next step's V-cycle is already
// enqueued.  At convergence, maxit or the end of a cycle, x += Z y; a new
// cycle restarts from the true residual b - A x.

// v_0 = r / ||r|| (r: first cycle b, else b - A x) and z_0 = B v_0
static int gmres_cycle_start(pmg_ctx* c, bool first) {
  const int64_t N = c->lv[c->L - 1].N;
  cudaStream_t s = c->stream;
  double* nrm2 = c->gs + GmresState::nrm2(c->gm);
  if (first) {
    PMG_CUDA(cudaMemcpyAsync(nrm2, c->scal + S_BB, 8, cudaMemcpyDeviceToDevice, s));
  } else {
    if (int rc = level_apply(c, c->L - 1, PMG_FP64, c->cg_x, c->cg_r, c->cg_b)) return rc;
    PMG_CUDA(dot(c->cg_r, c->cg_r, N, c->partial, nrm2, s));
  }
  PMG_CUDA(gmres_start(c->gs, nrm2, c->gm, c->cg_r, c->gv, N, s));
  c->sv.gj = 0;
  return precondition(c, c->gv, c->gz);
}

// Arnoldi step j = sv.gj (z_j already enqueued); records ev_rr after the
// residual estimate's copy, then enqueues z_{j+1} if the cycle has room.
static int gmres_enqueue_step(pmg_ctx* c) {
  const int64_t N = c->lv[c->L - 1].N, ld = c->gld;
  cudaStream_t s = c->stream;
  const int j = c->sv.gj, m = c->gm;
  double* w = c->gv + (j + 1) * ld;
  double* hcol = c->gh + (int64_t)j * (m + 1);
  double* h2 = c->gs + GmresState::h2(m);
  double* nrm2 = c->gs + GmresState::nrm2(m);
  if (int rc = level_apply(c, c->L - 1, PMG_FP64, c->gz + j * ld, w, nullptr)) return rc;
  PMG_CUDA(multi_dot(c->gv, ld, j + 1, w, N, c->gpart, hcol, s));
  PMG_CUDA(multi_axpy(w, c->gv, ld, j + 1, hcol, -1.0, N, s));
  PMG_CUDA(multi_dot(c->gv, ld, j + 1, w, N, c->gpart, h2, s));
  PMG_CUDA(multi_axpy(w, c->gv, ld, j + 1, h2, -1.0, N, s));
  PMG_CUDA(dot(w, w, N, c->partial, nrm2, s));
  PMG_CUDA(gmres_givens(c->gh, c->gs, nrm2, j, m, w, N, s));
  PMG_CUDA(cudaMemcpyAsync(c->host_scal + S_RR, c->gs + GmresState::est(m), 8, cudaMemcpyDeviceToHost, s));
  PMG_CUDA(cudaEventRecord(c->ev_rr, s));
  ++c->sv.it;
  c->sv.gj = j + 1;
  if (j + 1 < m) return precondition(c, w, c->gz + (j + 1) * ld);
  return PMG_OK;
}

// x += Z y over the steps of the current cycle
static int gmres_update_x(pmg_ctx* c) {
  const int64_t N = c->lv[c->L - 1].N;
  PMG_CUDA(gmres_update(c->gh, c->gs, c->sv.gj, c->gm, c->gz, c->gld, c->cg_x, N, c->stream));
  return PMG_OK;
}

static int solve_start(pmg_ctx* c, const double* b, bool b_host, double rtol, int maxit) {
  const int64_t N = c->lv[c->L - 1].N;
  cudaStream_t s = c->stream;
  c->sv = SolveState();
  c->sv.rtol = rtol;
  c->sv.maxit = maxit;
  PMG_CUDA(cudaEventRecord(c->ev0, s));
  if (b_host) PMG_CUDA(cudaMemcpyAsync(c->cg_r, b, 8 * N, cudaMemcpyHostToDevice, s));
  else PMG_CUDA(cudaMemcpyAsync(c->cg_r, b, 8 * N, cudaMemcpyDeviceToDevice, s));
  PMG_CUDA(cudaMemsetAsync(c->cg_x, 0, 8 * N, s));
  PMG_CUDA(dot(c->cg_r, c->cg_r, N, c->partial, c->scal + S_BB, s));
  PMG_CUDA(cudaMemcpyAsync(c->host_scal + S_BB, c->scal + S_BB, 8, cudaMemcpyDeviceToHost, s));
  PMG_CUDA(cudaEventRecord(c->ev_rr, s));
  if (c->gmres) {
    // b is kept for the residuals of restarted cycles
    PMG_CUDA(cudaMemcpyAsync(c->cg_b, c->cg_r, 8 * N, cudaMemcpyDeviceToDevice, s));
    if (int rc = gmres_cycle_start(c, true)) return rc;
    c->sv.phase = SP_WAIT_BB;
    return PMG_OK;
  }
  if (int rc = precondition(c, c->cg_r, c->cg_z)) return rc;
  PMG_CUDA(dot(c->cg_r, c->cg_z, N, c->partial, c->scal + S_RZ, s));
  PMG_CUDA(cudaMemcpyAsync(c->cg_p, c->cg_z, 8 * N, cudaMemcpyDeviceToDevice, s));
  c->sv.phase = SP_WAIT_BB;
  return PMG_OK;
}

static int solve_finish(pmg_ctx* c, int status) {
  const int64_t N = c->lv[c->L - 1].N;
  c->sv.status = status;
  if (c->gmres && c->sv.gj > 0) {
    if (int rc = gmres_update_x(c)) return rc;
  }
  PMG_CUDA(cudaEventRecord(c->ev1, c->stream));
  if (c->sv.x_out) {
    PMG_CUDA(cudaMemcpyAsync(c->sv.x_out, c->cg_x, 8 * N,
                             c->sv.x_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream));
  }
  PMG_CUDA(cudaEventRecord(c->ev_done, c->stream));
  c->sv.phase = SP_COPY_OUT;
  return PMG_OK;
}

// Advance the solve as far as completed device work allows; with `block`,
// wait for each pending event.  *state: 0 running, 1 done.
int solve_progress(pmg_ctx* c, bool block, int* state) {
  *state = 0;
  if (c->group) return PMG_OK;  // advanced by its group until its solution is copied out
  for (;;) {
    if (c->sv.phase == SP_IDLE) return fail(PMG_ERR_STATE, "no solve in progress");
    if (c->sv.phase == SP_DONE) {
      *state = 1;
      return PMG_OK;
    }
    cudaEvent_t ev = c->sv.phase == SP_COPY_OUT ? c->ev_done : c->ev_rr;
    if (block) {
      PMG_CUDA(cudaEventSynchronize(ev));
    } else {
      const cudaError_t q = cudaEventQuery(ev);
      if (q == cudaErrorNotReady) return PMG_OK;
      if (q != cudaSuccess) return fail(PMG_ERR_CUDA, std::string("solve: ") + cudaGetErrorString(q));
    }
    if (c->sv.phase == SP_COPY_OUT) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, c->ev0, c->ev1);
      c->sv.time_ms = ms;
      c->sv.phase = SP_DONE;
      if (c->sv.error != PMG_OK) c->sv.status = c->sv.error;
      continue;
    }
    if (c->sv.phase == SP_WAIT_BB) {
      c->sv.nb = std::sqrt(c->host_scal[S_BB]);
      if (!(c->sv.nb > 0)) {
        c->sv.rel = 0.0;
        if (int rc = solve_finish(c, PMG_OK)) return rc;
        continue;
      }
      c->sv.rel = 1.0;
    } else {
      c->sv.rel = c->gmres ? c->host_scal[S_RR] / c->sv.nb
                           : std::sqrt(std::max(c->host_scal[S_RR], 0.0)) / c->sv.nb;
      if (!(c->sv.rel == c->sv.rel)) return fail(PMG_ERR_STATE, "solver breakdown (NaN residual)");
      if (c->sv.rel <= c->sv.rtol) {
        if (int rc = solve_finish(c, PMG_OK)) return rc;
        continue;
      }
    }
    if (c->sv.it >= c->sv.maxit) {
      if (int rc = solve_finish(c, PMG_NOT_CONVERGED)) return rc;
      continue;
    }
    if (c->gmres) {
      if (c->sv.gj == c->gm) {  // end of a cycle: update x and restart
        if (int rc = gmres_update_x(c)) return rc;
        if (int rc = gmres_cycle_start(c, false)) return rc;
      }
      if (int rc = gmres_enqueue_step(c)) return rc;
    } else {
      if (int rc = enqueue_iteration(c)) return rc;
    }
    c->sv.phase = SP_WAIT_RR;
  }
}

void solve_info(const pmg_ctx* c, pmg_solve_info* info) {
  if (!info) return;
  info->iterations = c->sv.it;
  info->rel_residual = c->sv.rel;
  info->time_ms = c->sv.time_ms;
  info->status = c->sv.status;
}

static int solve_blocking(pmg_ctx* c, const double* b, bool b_host, double* x, bool x_host, double rtol, int maxit,
                          pmg_solve_info* info) {
  if (check_ctx(c) || !b || !x) return fail(PMG_ERR_ARG, "NULL argument");
  if (maxit < 0 || !(rtol >= 0)) return fail(PMG_ERR_ARG, "bad rtol / maxit");
  if (c->group) return fail(PMG_ERR_STATE, "the context is part of a grouped solve");
  if (int rc = solve_start(c, b, b_host, rtol, maxit)) return rc;
  c->sv.x_out = x;
  c->sv.x_host = x_host;
  int state = 0;
  if (int rc = solve_progress(c, true, &state)) return rc;
  solve_info(c, info);
  const int status = c->sv.status;
  c->sv.phase = SP_IDLE;
  return status;
}

}  // namespace pmg

extern "C" {

int pmg_solve(pmg_ctx* c, const double* b, double* x, double rtol, int maxit, pmg_solve_info* info) {
  return solve_blocking(c, b, false, x, false, rtol, maxit, info);
}

int pmg_solve_host(pmg_ctx* c, const double* b_host, double* x_host, double rtol, int maxit, pmg_solve_info* info) {
  return solve_blocking(c, b_host, true, x_host, true, rtol, maxit, info);
}

int pmg_solve_start(pmg_ctx* c, const double* b, int b_on_host, double* x, int x_on_host, double rtol, int maxit) {
  if (check_ctx(c) || !b || !x) return fail(PMG_ERR_ARG, "NULL argument");
  if (maxit < 0 || !(rtol >= 0)) return fail(PMG_ERR_ARG, "bad rtol / maxit");
  if (c->group || (c->sv.phase != SP_IDLE && c->sv.phase != SP_DONE))
    return fail(PMG_ERR_STATE, "a solve is already in progress");
  if (int rc = solve_start(c, b, b_on_host != 0, rtol, maxit)) return rc;
  c->sv.x_out = x;
  c->sv.x_host = x_on_host != 0;
  return PMG_OK;
}

int pmg_solve_progress(pmg_ctx* c, int* done, pmg_solve_info* info) {
  if (check_ctx(c) || !done) return fail(PMG_ERR_ARG, "NULL argument");
  int state = 0;
  if (int rc = solve_progress(c, false, &state)) return rc;
  *done = state;
  if (state) {
    solve_info(c, info);
    c->sv.phase = SP_IDLE;
    return c->sv.status;
  }
  return PMG_OK;
}

int pmg_rhs_manufactured(pmg_ctx* c, double* b) {
  if (check_ctx(c) || !b) return fail(PMG_ERR_ARG, "NULL argument");
  LevelData& F = c->lv[c->L - 1];
  PMG_CUDA(rhs_manufactured(c->dim, F.n, c->K, geom_desc(c), make_tab(c->K, c->K + 1), b,
                            c->stream));
  return PMG_OK;
}

int pmg_l2_error_manufactured(pmg_ctx* c, const double* x, double* err) {
  if (check_ctx(c) || !x || !err) return fail(PMG_ERR_ARG, "NULL argument");
  LevelData& F = c->lv[c->L - 1];
  PMG_CUDA(l2_error_partials(c->dim, F.n, c->K, geom_desc(c), make_tab(c->K, c->K + 3), x,
                             c->partial, c->scal + S_TMP, c->stream));
  PMG_CUDA(cudaMemcpyAsync(c->host_scal + S_TMP, c->scal + S_TMP, 8, cudaMemcpyDeviceToHost, c->stream));
  PMG_CUDA(cudaStreamSynchronize(c->stream));
  *err = std::sqrt(std::max(c->host_scal[S_TMP], 0.0));
  return PMG_OK;
}

int pmg_synchronize(pmg_ctx* c) {
  if (check_ctx(c)) return PMG_ERR_ARG;
  PMG_CUDA(cudaStreamSynchronize(c->stream));
  return PMG_OK;
}

int64_t pmg_launch_count(void) { return g_launches.load(); }

int pmg_smoother_phase_times(pmg_ctx* c, int level, int reps, double* ms) {
  if (check_ctx(c) || !ms) return fail(PMG_ERR_ARG, "NULL argument");
  if (int rc = check_smooth_level(c, level)) return rc;
  if (reps < 1) return fail(PMG_ERR_ARG, "reps < 1");
  LevelData& L = c->lv[level];
  cudaEvent_t ev[4];
  for (auto& e : ev) PMG_CUDA(cudaEventCreate(&e));
  double acc[3] = {0, 0, 0};
  int rc = PMG_OK;
  for (int it = 0; it <= reps && rc == PMG_OK; ++it) {  // iteration 0 warms up
    cudaEventRecord(ev[0], c->stream);
    rc = level_apply(c, level, c->mgprec, L.u, L.r, L.b);
    cudaEventRecord(ev[1], c->stream);
    if (!rc) rc = patch_solves(c, level, L.r);
    cudaEventRecord(ev[2], c->stream);
    if (!rc) {
      cudaError_t e = c->km()->patch_gather(c->dim, c->mgprec, c->pbuf, L.u, L.n, 1, c->stream);
      if (e != cudaSuccess) rc = fail(PMG_ERR_CUDA, cudaGetErrorString(e));
    }
    cudaEventRecord(ev[3], c->stream);
    cudaEventSynchronize(ev[3]);
    if (it > 0)
      for (int k = 0; k < 3; ++k) {
        float t = 0.f;
        cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
        acc[k] += t;
      }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (rc) return rc;
  for (int k = 0; k < 3; ++k) ms[k] = acc[k] / reps;
  return PMG_OK;
}

int pmg_default_damping(int dim, int degree, double* omega_patch, double* omega_jacobi) {
  if (dim != 2 && dim != 3) return fail(PMG_ERR_UNSUPPORTED, "dim must be 2 or 3");
  if (degree < 1 || degree > 8) return fail(PMG_ERR_UNSUPPORTED, "degree must be in 1..8");
  if (!omega_patch || !omega_jacobi) return fail(PMG_ERR_ARG, "NULL argument");
  *omega_patch = default_omega_patch(dim);
  const int np = nlev(degree);
  for (int l = 0; l < 4; ++l)
    omega_jacobi[l] = (l > 0 && l < np) ? host::default_omega_jacobi(dim, plev(degree, l)) : 1.0;
  return PMG_OK;
}

int pmg_damping(const pmg_ctx* c, double* omega_patch, double* omega_jacobi) {
  if (check_ctx(c) || !omega_patch || !omega_jacobi) return fail(PMG_ERR_ARG, "NULL argument");
  *omega_patch = c->omega_as;
  for (int l = 0; l < 4; ++l) omega_jacobi[l] = c->omega_j[l];
  return PMG_OK;
}

int pmg_patches_per_block(const pmg_ctx* c, int* ppc) {
  if (check_ctx(c) || !ppc) return fail(PMG_ERR_ARG, "NULL argument");
  *ppc = c->il_threads > 0 ? c->km()->patch_il(c->dim, c->mgprec, c->cfg.local_cycles) : c->ppc;
  return PMG_OK;
}

int pmg_patch_persistent(const pmg_ctx* c, int* persistent) {
  if (check_ctx(c) || !persistent) return fail(PMG_ERR_ARG, "NULL argument");
  *persistent = c->persistent ? 1 : 0;
  return PMG_OK;
}

int pmg_apply_cells_per_block(const pmg_ctx* c, int* cpb) {
  if (check_ctx(c) || !cpb) return fail(PMG_ERR_ARG, "NULL argument");
  *cpb = c->def_cpb;
  return PMG_OK;
}

int pmg_patch_layout(const pmg_ctx* c, int* layout, int* patches_per_block, int* threads) {
  if (check_ctx(c) || !layout || !patches_per_block || !threads) return fail(PMG_ERR_ARG, "NULL argument");
  if (c->il_threads > 0) {
    *layout = PMG_PATCH_INTERLEAVED;
    *patches_per_block = c->km()->patch_il(c->dim, c->mgprec, c->cfg.local_cycles);
    *threads = c->il_threads;
  } else {
    const int tpp = c->deformed ? c->km()->patch_def_threads(c->dim) : c->km()->patch_threads(c->dim);
    *layout = PMG_PATCH_MAJOR;
    *patches_per_block = c->ppc;
    *threads = std::min(1024, (c->ppc * tpp + 31) / 32 * 32);
  }
  return PMG_OK;
}

const char* pmg_status_string(int s) {
  switch (s) {
    case PMG_OK: return "ok";
    case PMG_NOT_CONVERGED: return "not converged";
    case PMG_ERR_ARG: return "invalid argument";
    case PMG_ERR_UNSUPPORTED: return "unsupported configuration";
    case PMG_ERR_OOM: return "out of device memory";
    case PMG_ERR_CUDA: return "CUDA error";
    case PMG_ERR_DEVICE_TIMEOUT: return "device wait timed out";
    case PMG_ERR_STATE: return "invalid state";
    default: return "unknown status";
  }
}

const char* pmg_last_error(void) { return t_last_error.c_str(); }

}  // extern "C"

