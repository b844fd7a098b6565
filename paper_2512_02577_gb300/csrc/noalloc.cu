// Allocation-free entry point: the Cartesian operator apply y = A x without
// a context and without allocating device memory.
//
// Some callers cannot allocate device memory: code that runs inside another
// framework's memory pool or under a hard device-memory cap, and real-time
// loops where cudaMalloc (which may synchronise the device) is not allowed.
// This variant of the three-pass Cartesian apply keeps its four intermediate
// grid vectors in a file-scope __device__ array instead of context scratch.
// The array (PMG_NOALLOC_MAX_DOFS doubles x 4 = 64 MiB) is part of the
// library's device image: every GPU that loads the library holds it until
// the process exits.  Every call shares it and it keeps the last call's
// contents; each call writes every scratch element it later reads, so
// nothing needs clearing, but calls that overlap on the GPU (different
// streams, or different host threads) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pmg.h"
#include "pmg_common.cuh"
#include "pmg_kernels_api.h"
#include "setup.h"

namespace pmg {
const KernelTable* kernel_table(int K, int dim, int prec);
void set_last_error(const std::string& msg);
}  // namespace pmg

namespace {

constexpr int64_t kMaxDofs = PMG_NOALLOC_MAX_DOFS;

static __device__ __align__(256) double g_apply_scratch[4 * kMaxDofs];

struct DeviceState {
  bool ready = false;
  double* scratch = nullptr;  // device address of g_apply_scratch on this device
  bool coef[9][2] = {};  // by degree and dimension
};

constexpr int kMaxDevices = 64;
std::mutex g_mu;
DeviceState g_state[kMaxDevices];

int fail(int code, const std::string& msg) {
  pmg::set_last_error(msg);
  return code;
}

}  // namespace

extern "C" int pmg_apply_cartesian_noalloc(int dim, int n_cells, int degree, const double* x, double* y,
                                           void* stream) {
  if (dim != 2 && dim != 3) return fail(PMG_ERR_UNSUPPORTED, "dim must be 2 or 3");
  if (degree < 1 || degree > 8) return fail(PMG_ERR_UNSUPPORTED, "degree must be in 1..8");
  if (n_cells < 1) return fail(PMG_ERR_ARG, "n_cells must be >= 1");
  if (!x || !y) return fail(PMG_ERR_ARG, "NULL vector");
  const int64_t n1 = (int64_t)degree * n_cells + 1;
  const int64_t N = dim == 3 ? n1 * n1 * n1 : n1 * n1;
  if (N > kMaxDofs)
    return fail(PMG_ERR_UNSUPPORTED, "grid of " + std::to_string(N) + " nodes exceeds the allocation-free limit of " +
                                         std::to_string(kMaxDofs) + " ((k n + 1)^d)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(PMG_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(PMG_ERR_UNSUPPORTED, "device ordinal above 63");
  // the vectors must live on this device (a pointer of another device, or a
  // host pointer, would be dereferenced by kernels running here)
  for (const void* v : {(const void*)x, (const void*)y}) {
    cudaPointerAttributes a{};
    e = cudaPointerGetAttributes(&a, v);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(PMG_ERR_ARG, std::string("cudaPointerGetAttributes: ") + cudaGetErrorString(e));
    }
    if ((a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != dev)
      return fail(PMG_ERR_ARG, "x and y must be device memory of the current device (" + std::to_string(dev) + ")");
  }
  const pmg::KernelTable* kt = pmg::kernel_table(degree, dim, 0);
  double* scratch = nullptr;
  {
    // first call on this device (and first call for this degree): resolve the
    // scratch address and load the degree's 1D matrices into constant memory
    std::lock_guard<std::mutex> g(g_mu);
    DeviceState& s = g_state[dev];
    if (!s.ready) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_apply_scratch);
      if (e != cudaSuccess) return fail(PMG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      s.scratch = (double*)ptr;
      s.ready = true;
    }
    if (!s.coef[degree][dim - 2]) {
      std::vector<double> coef(pmg::kMaxCoef, 0.0);
      pmg::host::fill_coefficients(degree, coef.data());
      e = kt->prepare();
      if (e == cudaSuccess) e = kt->upload(coef.data());
      if (e != cudaSuccess) return fail(PMG_ERR_CUDA, std::string("coefficient upload: ") + cudaGetErrorString(e));
      s.coef[degree][dim - 2] = true;
    }
    scratch = s.scratch;
  }
  const double scale = std::pow(1.0 / n_cells, dim - 2);
  e = kt->cart_apply(dim, 0, x, y, nullptr, scratch, scratch + N, scratch + 2 * N, scratch + 3 * N, n_cells, scale,
                     (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(PMG_ERR_CUDA, std::string("apply: ") + cudaGetErrorString(e));
  return PMG_OK;
}
