// Deformed-geometry kernels for one degree K (included by inst_k.cuh after
// kernels.cuh).  The operator is the general sum-factorised form of Eq. (3):
// per cell, interpolate the nodal values from the Gauss-Lobatto nodes to the
// (p+1)^d Gauss points (d 1D contractions with S), take reference gradients
// by collocation derivatives at the Gauss points (Dq), multiply by the stored
// symmetric tensor G_q = w_q det J J^{-1} J^{-T} (float32, §3's
// quadrature-point "evaluation kernel"), and apply the transposed steps.
// Cells of one parity colour share no node, so colour-by-colour launches
// accumulate without atomics and in a fixed order.
#pragma once

namespace pmg {
namespace PMG_KNS {

template <int DIM>
__host__ __device__ constexpr int ncomp() { return DIM == 3 ? 6 : 3; }

// y = C x (TR = false) or y = C^T x (TR = true) for an n x n row-major C.
template <int n, bool TR, typename T>
__device__ __forceinline__ void mvn(const T* C, const T* x, T* y) {
#pragma unroll
  for (int i = 0; i < n; ++i) {
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < n; ++j) acc += (TR ? C[j * n + i] : C[i * n + j]) * x[j];
    y[i] = acc;
  }
}

// Contract one axis of an n^DIM tile: dst = C src along AX (ACC: dst += ...).
template <int DIM, int n, int AX, bool TR, bool ACC, typename T>
__device__ __forceinline__ void tile_axis(const T* C, const T* src, T* dst, int lane, int tpc) {
  constexpr int EZ = DIM == 3 ? n : 1;
  constexpr int nl = n * EZ;
  constexpr int st = AX == 0 ? 1 : (AX == 1 ? n : n * n);
  for (int L = lane; L < nl; L += tpc) {
    const int b = line_base<AX, n, n, EZ>(L);
    T x[n], y[n];
#pragma unroll
    for (int j = 0; j < n; ++j) x[j] = src[b + j * st];
    mvn<n, TR>(C, x, y);
#pragma unroll
    for (int i = 0; i < n; ++i) {
      if (ACC) dst[b + i * st] += y[i];
      else dst[b + i * st] = y[i];
    }
  }
}

// Cell operator of p-level l on a (p+1)^DIM tile: A0 (nodal values in) ->
// A0 (cell contribution out); A1, B0..B2 are work tiles; Gc points at the
// cell's tensor block [comp][point].  All threads of the block must call it.
template <int DIM, int l, typename T>
__device__ __forceinline__ void cell_op(T* A0, T* A1, T* B0, T* B1, T* B2, const float* __restrict__ Gc,
                                        int lane, int tpc) {
  constexpr int p = plev(K, l);
  constexpr int n1 = p + 1;
  constexpr int NP = ipow(n1, DIM);
  const T* Sm = coef<T>() + LAY.S[l];
  const T* Dm = coef<T>() + LAY.Dq[l];
  // values at Gauss points
  if constexpr (DIM == 3) {
    tile_axis<3, n1, 0, false, false>(Sm, A0, A1, lane, tpc);
    __syncthreads();
    tile_axis<3, n1, 1, false, false>(Sm, A1, A0, lane, tpc);
    __syncthreads();
    tile_axis<3, n1, 2, false, false>(Sm, A0, A1, lane, tpc);
    __syncthreads();
    tile_axis<3, n1, 0, false, false>(Dm, A1, B0, lane, tpc);
    tile_axis<3, n1, 1, false, false>(Dm, A1, B1, lane, tpc);
    tile_axis<3, n1, 2, false, false>(Dm, A1, B2, lane, tpc);
    __syncthreads();
    for (int q = lane; q < NP; q += tpc) {
      const T g0 = B0[q], g1 = B1[q], g2 = B2[q];
      const T G00 = (T)Gc[0 * NP + q], G01 = (T)Gc[1 * NP + q], G02 = (T)Gc[2 * NP + q];
      const T G11 = (T)Gc[3 * NP + q], G12 = (T)Gc[4 * NP + q], G22 = (T)Gc[5 * NP + q];
      B0[q] = G00 * g0 + G01 * g1 + G02 * g2;
      B1[q] = G01 * g0 + G11 * g1 + G12 * g2;
      B2[q] = G02 * g0 + G12 * g1 + G22 * g2;
    }
    __syncthreads();
    tile_axis<3, n1, 0, true, false>(Dm, B0, A1, lane, tpc);
    __syncthreads();
    tile_axis<3, n1, 1, true, true>(Dm, B1, A1, lane, tpc);
    __syncthreads();
    tile_axis<3, n1, 2, true, true>(Dm, B2, A1, lane, tpc);
    __syncthreads();
    tile_axis<3, n1, 2, true, false>(Sm, A1, A0, lane, tpc);
    __syncthreads();
    tile_axis<3, n1, 1, true, false>(Sm, A0, A1, lane, tpc);
    __syncthreads();
    tile_axis<3, n1, 0, true, false>(Sm, A1, A0, lane, tpc);
    __syncthreads();
  } else {
    tile_axis<2, n1, 0, false, false>(Sm, A0, A1, lane, tpc);
    __syncthreads();
    tile_axis<2, n1, 1, false, false>(Sm, A1, A0, lane, tpc);
    __syncthreads();
    tile_axis<2, n1, 0, false, false>(Dm, A0, B0, lane, tpc);
    tile_axis<2, n1, 1, false, false>(Dm, A0, B1, lane, tpc);
    __syncthreads();
    for (int q = lane; q < NP; q += tpc) {
      const T g0 = B0[q], g1 = B1[q];
      const T G00 = (T)Gc[0 * NP + q], G01 = (T)Gc[1 * NP + q], G11 = (T)Gc[2 * NP + q];
      B0[q] = G00 * g0 + G01 * g1;
      B1[q] = G01 * g0 + G11 * g1;
    }
    __syncthreads();
    tile_axis<2, n1, 0, true, false>(Dm, B0, A1, lane, tpc);
    __syncthreads();
    tile_axis<2, n1, 1, true, true>(Dm, B1, A1, lane, tpc);
    __syncthreads();
    tile_axis<2, n1, 1, true, false>(Sm, A1, A0, lane, tpc);
    __syncthreads();
    tile_axis<2, n1, 0, true, false>(Sm, A0, A1, lane, tpc);
    __syncthreads();
    for (int q = lane; q < NP; q += tpc) A0[q] = A1[q];
    __syncthreads();
  }
}

// Global deformed apply, one parity colour of cells: y += SIGN * A_cell x.
// Boundary nodes of y are written as 0.
template <int DIM, int SIGN, typename T>
__global__ void def_cell_kernel(const T* __restrict__ x, T* __restrict__ y, const float* __restrict__ G, int n,
                                int colour, int cpb) {
  constexpr int l = nlev(K) - 1;
  constexpr int n1 = K + 1;
  constexpr int NP = ipow(n1, DIM);
  constexpr int TPC = ipow(n1, DIM - 1);
  extern __shared__ __align__(16) unsigned char smraw[];
  const int grp = threadIdx.x / TPC, lane = threadIdx.x % TPC;
  T* A0 = reinterpret_cast<T*>(smraw) + (int64_t)grp * 5 * NP;
  T *A1 = A0 + NP, *B0 = A1 + NP, *B1 = B0 + NP, *B2 = B1 + NP;
  const int cx = (colour & 1) ? n / 2 : (n + 1) / 2, cy = ((colour >> 1) & 1) ? n / 2 : (n + 1) / 2;
  const int cz = DIM == 3 ? (((colour >> 2) & 1) ? n / 2 : (n + 1) / 2) : 1;
  const int64_t ncell = (int64_t)cx * cy * cz;
  const int64_t cid = (int64_t)blockIdx.x * cpb + grp;
  const bool active = cid < ncell;
  int c[3] = {0, 0, 0};
  if (active) {
    int64_t t = cid;
    c[0] = 2 * (int)(t % cx) + (colour & 1); t /= cx;
    c[1] = 2 * (int)(t % cy) + ((colour >> 1) & 1); t /= cy;
    c[2] = DIM == 3 ? 2 * (int)t + ((colour >> 2) & 1) : 0;
  }
  const int N1 = K * n + 1;
  for (int i = lane; i < NP; i += TPC) {
    T v = T(0);
    if (active) {
      const int ax = i % n1, ay = (i / n1) % n1, az = DIM == 3 ? i / (n1 * n1) : 0;
      const int gx = K * c[0] + ax, gy = K * c[1] + ay, gz = K * c[2] + az;
      const bool bnd = gx == 0 || gx == N1 - 1 || gy == 0 || gy == N1 - 1 ||
                       (DIM == 3 && (gz == 0 || gz == N1 - 1));
      if (!bnd) v = x[gx + (int64_t)N1 * (gy + (int64_t)N1 * gz)];
    }
    A0[i] = v;
  }
  __syncthreads();
  const int64_t cell = active ? c[0] + (int64_t)n * (c[1] + (int64_t)n * c[2]) : 0;
  cell_op<DIM, l, T>(A0, A1, B0, B1, B2, G + cell * ncomp<DIM>() * NP, lane, TPC);
  if (active) {
    for (int i = lane; i < NP; i += TPC) {
      const int ax = i % n1, ay = (i / n1) % n1, az = DIM == 3 ? i / (n1 * n1) : 0;
      const int gx = K * c[0] + ax, gy = K * c[1] + ay, gz = K * c[2] + az;
      const bool bnd = gx == 0 || gx == N1 - 1 || gy == 0 || gy == N1 - 1 ||
                       (DIM == 3 && (gz == 0 || gz == N1 - 1));
      const int64_t g = gx + (int64_t)N1 * (gy + (int64_t)N1 * gz);
      if (bnd) y[g] = T(0);
      else y[g] += (SIGN > 0 ? A0[i] : -A0[i]);
    }
  }
}

template <int DIM, typename T>
static cudaError_t def_apply_t(const T* x, T* y, const T* b, const float* G, int n, cudaStream_t st) {
  constexpr int n1 = K + 1;
  constexpr int NP = ipow(n1, DIM);
  constexpr int TPC = ipow(n1, DIM - 1);
  int cpb = 128 / TPC;
  if (cpb < 1) cpb = 1;
  const int smem = cpb * 5 * NP * (int)sizeof(T);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e;
  if (b) e = cudaMemcpyAsync(y, b, sizeof(T) * (size_t)ipow(K * n + 1, DIM), cudaMemcpyDeviceToDevice, st);
  else e = cudaMemsetAsync(y, 0, sizeof(T) * (size_t)ipow(K * n + 1, DIM), st);
  if (e != cudaSuccess) return e;
  for (int colour = 0; colour < (1 << DIM); ++colour) {
    const int cx = (colour & 1) ? n / 2 : (n + 1) / 2, cy = ((colour >> 1) & 1) ? n / 2 : (n + 1) / 2;
    const int cz = DIM == 3 ? (((colour >> 2) & 1) ? n / 2 : (n + 1) / 2) : 1;
    const int64_t nc = (int64_t)cx * cy * cz;
    if (nc == 0) continue;
    const unsigned blocks = (unsigned)((nc + cpb - 1) / cpb);
    if (b) def_cell_kernel<DIM, -1, T><<<blocks, cpb * TPC, smem, st>>>(x, y, G, n, colour, cpb);
    else def_cell_kernel<DIM, 1, T><<<blocks, cpb * TPC, smem, st>>>(x, y, G, n, colour, cpb);
    g_launches += 1;
  }
  return cudaGetLastError();
}

static cudaError_t def_apply(int dim, int prec, const void* x, void* y, const void* b, const float* G, int n,
                             cudaStream_t s) {
  if (prec == 0) {
    if (dim == 3) return def_apply_t<3, double>((const double*)x, (double*)y, (const double*)b, G, n, s);
    return def_apply_t<2, double>((const double*)x, (double*)y, (const double*)b, G, n, s);
  }
  if (dim == 3) return def_apply_t<3, float>((const float*)x, (float*)y, (const float*)b, G, n, s);
  return def_apply_t<2, float>((const float*)x, (float*)y, (const float*)b, G, n, s);
}

// ---------------------------------------------------------------------------
// Deformed vertex-patch smoother.  The patch vmult (§3.2.1) distributes the
// patch-interior vector to the 2^d cells of the patch (zero on the patch
// boundary), applies the cell operator with each cell's stored G, and sums
// the cell results back onto the interior nodes.  Inverse diagonals come
// from the global degree-p diagonal of the level (a patch-interior DoF has
// its whole support inside the patch, so diag(A_{j,p}) is that diagonal).
// ---------------------------------------------------------------------------
template <int DIM>
struct DefShape {
  using PS = PatchShape<DIM>;
  static constexpr int NCELL = 1 << DIM;
  static constexpr int n1T = K + 1;
  static constexpr int NPT = ipow(n1T, DIM);
  static constexpr int XSZ = ipow(2 * K + 1, DIM);
  static constexpr int TPC = ipow(n1T, DIM - 1);
  static constexpr int TPP = NCELL * TPC;
  static constexpr int WORK = XSZ + NCELL * 5 * NPT;
  static constexpr int ELEMS = PS::ELEMS + WORK;
};

template <typename T>
struct DefLevelT {
  const float* G[4];
  const T* dinv[4];
};

template <int DIM, typename T>
struct DefGeo {
  DefLevelT<T> lev;
  int v[3];
  int n;
  T* work;

  __device__ __forceinline__ T dinv_at(int l, int i) const {
    const int p = l == nlev(K) - 1 ? K : plev(K, l);
    const int m = 2 * p - 1, N1 = p * n + 1;
    const int ix = i % m, iy = (i / m) % m, iz = DIM == 3 ? i / (m * m) : 0;
    const int gx = p * (v[0] - 1) + 1 + ix, gy = p * (v[1] - 1) + 1 + iy;
    const int gz = DIM == 3 ? p * (v[2] - 1) + 1 + iz : 0;
    return lev.dinv[l][gx + (int64_t)N1 * (gy + (int64_t)N1 * gz)];
  }

  template <int l>
  __device__ __forceinline__ void resid(const T* d, const T* r, T* out, T* t0, T* t1, int lane, int tpp) const {
    constexpr int p = plev(K, l);
    constexpr int m = mp(p), mf = 2 * p + 1, n1 = p + 1;
    constexpr int NP = ipow(n1, DIM);
    constexpr int XS = ipow(mf, DIM);
    constexpr int TPC = ipow(n1, DIM - 1);
    constexpr int NCELL = 1 << DIM;
    T* X = work;
    T* cb = work + DefShape<DIM>::XSZ;
    // expand d to the full patch grid, zero on the patch boundary
    for (int i = lane; i < XS; i += tpp) {
      const int fx = i % mf, fy = (i / mf) % mf, fz = DIM == 3 ? i / (mf * mf) : 1;
      const bool in = fx > 0 && fx < mf - 1 && fy > 0 && fy < mf - 1 && (DIM == 2 || (fz > 0 && fz < mf - 1));
      X[i] = in ? d[(fx - 1) + m * ((fy - 1) + m * (DIM == 3 ? fz - 1 : 0))] : T(0);
    }
    __syncthreads();
    int cg = lane / TPC, cl = lane % TPC;
    const bool cell_active = cg < NCELL;
    if (!cell_active) { cg = 0; cl = TPC; }  // idle threads still reach every barrier
    const int ox = cg & 1, oy = (cg >> 1) & 1, oz = DIM == 3 ? (cg >> 2) & 1 : 0;
    T* A0 = cb + (int64_t)cg * 5 * NP;
    T *A1 = A0 + NP, *B0 = A1 + NP, *B1 = B0 + NP, *B2 = B1 + NP;
    for (int i = cl; i < NP; i += TPC) {
      const int ax = i % n1, ay = (i / n1) % n1, az = DIM == 3 ? i / (n1 * n1) : 0;
      A0[i] = X[(p * ox + ax) + mf * ((p * oy + ay) + mf * (DIM == 3 ? p * oz + az : 0))];
    }
    __syncthreads();
    const int cx = v[0] - 1 + ox, cy = v[1] - 1 + oy, cz = DIM == 3 ? v[2] - 1 + oz : 0;
    const int64_t cell = cx + (int64_t)n * (cy + (int64_t)n * cz);
    cell_op<DIM, l, T>(A0, A1, B0, B1, B2, lev.G[l] + cell * ncomp<DIM>() * NP, cl, TPC);
    // sum the cell results back onto the interior nodes: out = r - A d
    for (int i = lane; i < ipow(m, DIM); i += tpp) {
      const int fx = i % m + 1, fy = (i / m) % m + 1, fz = DIM == 3 ? i / (m * m) + 1 : 0;
      T acc = T(0);
#pragma unroll
      for (int c = 0; c < NCELL; ++c) {
        const int qx = c & 1, qy = (c >> 1) & 1, qz = DIM == 3 ? (c >> 2) & 1 : 0;
        const int ax = fx - p * qx, ay = fy - p * qy, az = DIM == 3 ? fz - p * qz : 0;
        if (ax < 0 || ax > p || ay < 0 || ay > p || az < 0 || az > p) continue;
        acc += cb[(int64_t)c * 5 * NP + ax + n1 * (ay + n1 * az)];
      }
      out[i] = r[i] - acc;
    }
    __syncthreads();
  }
};

template <int DIM, typename T>
__global__ void patch_def_kernel(const T* __restrict__ r, T* __restrict__ u, int n, int colour, int ppc,
                                 int n_iter, DefLevelT<T> lev, const T* __restrict__ dinv1, PatchParams<T> P) {
  using S = PatchShape<DIM>;
  using DS = DefShape<DIM>;
  constexpr int TPP = DS::TPP;
  constexpr int MT = S::MT;
  constexpr int L = S::L;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int grp = threadIdx.x / TPP, lane = threadIdx.x % TPP;
  const int gstride = DS::ELEMS + (n_iter > 1 ? 2 * S::SZT : 0);
  T* sm = reinterpret_cast<T*>(smraw) + (int64_t)grp * gstride;
  const int cx = colour_count(n, colour & 1), cy = colour_count(n, (colour >> 1) & 1);
  const int cz = DIM == 3 ? colour_count(n, (colour >> 2) & 1) : 1;
  const int64_t npatch = (int64_t)cx * cy * cz;
  const int64_t pid = (int64_t)blockIdx.x * ppc + grp;
  const bool active = pid < npatch;
  DefGeo<DIM, T> geo;
  geo.lev = lev;
  geo.n = n;
  geo.work = sm + S::ELEMS;
  geo.v[0] = geo.v[1] = 1;
  geo.v[2] = DIM == 3 ? 1 : 0;
  if (active) {
    int64_t t = pid;
    const int ix = (int)(t % cx); t /= cx;
    const int iy = (int)(t % cy); t /= cy;
    const int iz = (int)t;
    geo.v[0] = 2 * ix + ((colour & 1) ? 1 : 2);
    geo.v[1] = 2 * iy + (((colour >> 1) & 1) ? 1 : 2);
    geo.v[2] = DIM == 3 ? 2 * iz + (((colour >> 2) & 1) ? 1 : 2) : 0;
  }
  const int N1 = K * n + 1;
  const int g0x = K * (geo.v[0] - 1) + 1, g0y = K * (geo.v[1] - 1) + 1;
  const int g0z = DIM == 3 ? K * (geo.v[2] - 1) + 1 : 0;
  T* rt = sm + S::off_r(L - 1);
  T* dt = sm + S::off_d(L - 1);
  for (int i = lane; i < S::SZT; i += TPP) {
    T val = T(0);
    if (active) {
      const int ix = i % MT, iy = (i / MT) % MT, iz = DIM == 3 ? i / (MT * MT) : 0;
      val = r[(int64_t)(g0x + ix) + (int64_t)N1 * ((g0y + iy) + (int64_t)N1 * (DIM == 3 ? g0z + iz : 0))];
    }
    rt[i] = val;
  }
  // p = 1 coarse solve: the vertex's inverse Q1 diagonal
  const int64_t vid = geo.v[0] + (int64_t)(n + 1) * (geo.v[1] + (int64_t)(n + 1) * geo.v[2]);
  const T inv_a0 = dinv1[vid];
  __syncthreads();
  if (n_iter > 1) {
    T* rj = sm + DS::ELEMS;
    T* ds = rj + S::SZT;
    for (int i = lane; i < S::SZT; i += TPP) rj[i] = rt[i];
    __syncthreads();
    pvcycle<DIM, L - 1, T>(sm, geo, P, inv_a0, lane, TPP);
    for (int i = lane; i < S::SZT; i += TPP) ds[i] = dt[i];
    __syncthreads();
    for (int it = 1; it < n_iter; ++it) {
      geo.template resid<L - 1>(ds, rj, rt, sm, sm + S::SZT, lane, TPP);
      pvcycle<DIM, L - 1, T>(sm, geo, P, inv_a0, lane, TPP);
      for (int i = lane; i < S::SZT; i += TPP) ds[i] += dt[i];
      __syncthreads();
    }
    for (int i = lane; i < S::SZT; i += TPP) dt[i] = ds[i];
    __syncthreads();
  } else {
    pvcycle<DIM, L - 1, T>(sm, geo, P, inv_a0, lane, TPP);
  }
  if (active) {
    for (int i = lane; i < S::SZT; i += TPP) {
      const int ix = i % MT, iy = (i / MT) % MT, iz = DIM == 3 ? i / (MT * MT) : 0;
      u[(int64_t)(g0x + ix) + (int64_t)N1 * ((g0y + iy) + (int64_t)N1 * (DIM == 3 ? g0z + iz : 0))] +=
          P.omega_as * dt[i];
    }
  }
}

static int patch_def_threads(int dim) { return dim == 3 ? DefShape<3>::TPP : DefShape<2>::TPP; }

static int patch_def_smem(int dim, int prec, int n_iter) {
  const int es = prec == 0 ? 8 : 4;
  const int elems = dim == 3 ? DefShape<3>::ELEMS + (n_iter > 1 ? 2 * PatchShape<3>::SZT : 0)
                             : DefShape<2>::ELEMS + (n_iter > 1 ? 2 * PatchShape<2>::SZT : 0);
  return elems * es;
}

template <int DIM, typename T>
static cudaError_t patch_def_t(const T* r, T* u, int n, int colour, int ppc, int n_iter, const DefLevel& L,
                               const PatchParamsHost& H, cudaStream_t st) {
  if (n < 2) return cudaSuccess;
  const int cx = (colour & 1) ? n / 2 : (n - 1) / 2;
  const int cy = ((colour >> 1) & 1) ? n / 2 : (n - 1) / 2;
  const int cz = DIM == 3 ? (((colour >> 2) & 1) ? n / 2 : (n - 1) / 2) : 1;
  const int64_t np = (int64_t)cx * cy * cz;
  if (np == 0) return cudaSuccess;
  const int smem = ppc * patch_def_smem(DIM, sizeof(T) == 8 ? 0 : 1, n_iter);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  DefLevelT<T> lev;
  for (int i = 0; i < 4; ++i) {
    lev.G[i] = L.G[i];
    lev.dinv[i] = (const T*)L.dinv[i];
  }
  const unsigned blocks = (unsigned)((np + ppc - 1) / ppc);
  patch_def_kernel<DIM, T><<<blocks, ppc * DefShape<DIM>::TPP, smem, st>>>(r, u, n, colour, ppc, n_iter, lev,
                                                                          (const T*)L.dinv1, to_params<T>(H));
  g_launches += 1;
  return cudaGetLastError();
}

static cudaError_t patch_def(int dim, int prec, const void* r, void* u, int n, int colour, int ppc, int n_iter,
                             const DefLevel& L, const PatchParamsHost& P, cudaStream_t s) {
  if (prec == 0) {
    if (dim == 3) return patch_def_t<3, double>((const double*)r, (double*)u, n, colour, ppc, n_iter, L, P, s);
    return patch_def_t<2, double>((const double*)r, (double*)u, n, colour, ppc, n_iter, L, P, s);
  }
  if (dim == 3) return patch_def_t<3, float>((const float*)r, (float*)u, n, colour, ppc, n_iter, L, P, s);
  return patch_def_t<2, float>((const float*)r, (float*)u, n, colour, ppc, n_iter, L, P, s);
}

}  // namespace PMG_KNS
}  // namespace pmg
