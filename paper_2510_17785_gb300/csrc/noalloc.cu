// pmg_lanczos_bounds_noalloc: the per-patch Lanczos eigenvalue estimates of
// pmg_compute_bounds for a range of patches, for callers that must not
// allocate device memory.
//
// Who cannot allocate: code that runs while a CUDA graph is being captured
// (cudaMalloc is not capturable), code inside a framework that owns the
// device memory budget through its own caching allocator and forbids raw
// cudaMalloc/cudaFree (which also synchronise the device), and long-running
// or latency-critical solvers that recompute Chebyshev bounds mid-run and must
// not stall on, or fail in, an allocation.  pmg_compute_bounds needs a
// device buffer for the Lanczos basis; this entry point uses a fixed
// file-scope device array instead.
//
// The array (kScratchBytes = 16 MiB) is part of the library image: every GPU
// that loads the library holds it until the process exits.  All calls share
// it and it keeps whatever the last call wrote.  The Lanczos kernel writes
// every basis vector before reading it, so nothing needs clearing.  Calls
// whose kernels overlap on the GPU (different streams, or different contexts
// on one device) race on the array: serialise them.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/pmg.h"
#include "basis.h"
#include "lanczos_view.h"
#include "patch.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;
static __device__ __align__(256) double g_lanczos_scratch[kScratchBytes / sizeof(double)];

constexpr int kMaxDevices = 64;
struct DeviceState {
  bool ready = false;
  double* scratch = nullptr;   // device address of g_lanczos_scratch on this device
};
DeviceState g_dev[kMaxDevices];
std::mutex g_mu;

template <int DIM, int Q>
cudaError_t set_smem_attr() {
  constexpr size_t smem = pmg::lanczos_smem<DIM, Q, double>();
  if constexpr (smem > 227 * 1024) {
    return cudaSuccess;
  } else {
    return cudaFuncSetAttribute(pmg::k_lanczos<DIM, Q, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  }
}

// Once per device, with that device current: upload this file's constant
// tables, set the kernels' shared-memory limits and take the device address
// of the scratch array (its name is only a host-side stand-in in host code).
cudaError_t setup_device(int dev) {
  pmg::Tables<double> t64;
  pmg::Tables<float> t32;
  pmg::Rules r;
  pmg::build_tables(t64, t32, r);
  cudaError_t e = (cudaError_t)pmg::upload_tables_tu(t64, t32, r);
  if (e != cudaSuccess) return e;
  cudaError_t a[] = {set_smem_attr<2, 2>(), set_smem_attr<2, 3>(), set_smem_attr<2, 4>(), set_smem_attr<2, 5>(),
                     set_smem_attr<2, 6>(), set_smem_attr<2, 7>(), set_smem_attr<2, 8>(), set_smem_attr<3, 2>(),
                     set_smem_attr<3, 3>(), set_smem_attr<3, 4>(), set_smem_attr<3, 5>(), set_smem_attr<3, 6>(),
                     set_smem_attr<3, 7>(), set_smem_attr<3, 8>()};
  for (cudaError_t x : a)
    if (x != cudaSuccess) return x;
  double* ptr = nullptr;
  e = cudaGetSymbolAddress((void**)&ptr, g_lanczos_scratch);
  if (e != cudaSuccess) return e;
  g_dev[dev].scratch = ptr;
  g_dev[dev].ready = true;
  return cudaSuccess;
}

template <int DIM, int Q>
int launch(const pmg::LanczosArgs<double>& a, cudaStream_t s) {
  constexpr size_t smem = pmg::lanczos_smem<DIM, Q, double>();
  if constexpr (smem > 227 * 1024) {
    return PMG_ERR_UNSUPPORTED;
  } else {
    pmg::k_lanczos<DIM, Q, double><<<a.n_items, 256, smem, s>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? PMG_OK : PMG_ERR_CUDA;
  }
}

template <int DIM>
int launch_q(int q, const pmg::LanczosArgs<double>& a, cudaStream_t s) {
  switch (q) {
    case 2: return launch<DIM, 2>(a, s);
    case 3: return launch<DIM, 3>(a, s);
    case 4: return launch<DIM, 4>(a, s);
    case 5: return launch<DIM, 5>(a, s);
    case 6: return launch<DIM, 6>(a, s);
    case 7: return launch<DIM, 7>(a, s);
    case 8: return launch<DIM, 8>(a, s);
    default: return PMG_ERR_UNSUPPORTED;
  }
}

}  // namespace

extern "C" int pmg_lanczos_bounds_noalloc(pmg_ctx* ctx, int level, int k, int64_t first_patch, int64_t n_patches,
                                          double* ritz_dev, double* bounds_dev, void* stream) {
  if (!ctx) return PMG_ERR_ARG;
  pmg::LanczosView v;
  if (pmg::lanczos_view(ctx, level, k, &v) != PMG_OK)
    return pmg::set_last_error(ctx, PMG_ERR_ARG, "noalloc Lanczos: context not set up, or level / p-level out of range");
  if (v.q < 2) return pmg::set_last_error(ctx, PMG_ERR_ARG, "noalloc Lanczos: the p = 1 level has no interval");
  if (first_patch < 0 || n_patches < 0 || first_patch + n_patches > v.npatch)
    return pmg::set_last_error(ctx, PMG_ERR_ARG, "noalloc Lanczos: patch range outside the level");
  if (n_patches > 0 && (!ritz_dev || !bounds_dev))
    return pmg::set_last_error(ctx, PMG_ERR_ARG, "noalloc Lanczos: null output pointer");
  size_t ni = 1;
  for (int ax = 0; ax < v.dim; ++ax) ni *= (size_t)(2 * v.q - 1);
  const size_t need = (size_t)n_patches * (size_t)v.ksteps * ni * sizeof(double);
  if (need > kScratchBytes)
    return pmg::set_last_error(ctx, PMG_ERR_ARG,
                               "noalloc Lanczos: n_patches * lanczos_steps * (2q-1)^d doubles exceed the fixed "
                               "16 MiB scratch array; split the patch range into smaller calls");
  if (v.ksteps > 64) return pmg::set_last_error(ctx, PMG_ERR_ARG, "noalloc Lanczos: more than 64 Lanczos steps");
  if (v.device < 0 || v.device >= kMaxDevices) return pmg::set_last_error(ctx, PMG_ERR_ARG, "device index too large");
  if (cudaSetDevice(v.device) != cudaSuccess)
    return pmg::set_last_error(ctx, PMG_ERR_CUDA, "noalloc Lanczos: cudaSetDevice failed");
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev[v.device].ready) {
      cudaError_t e = setup_device(v.device);
      if (e != cudaSuccess) return pmg::set_last_error(ctx, PMG_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  if (n_patches == 0) return PMG_OK;
  pmg::LanczosArgs<double> a;
  a.N = v.N;
  a.n_items = (int)n_patches;
  a.first_patch = (int)first_patch;
  a.G = v.G64;
  a.dinv = v.dinv64;
  a.V = g_dev[v.device].scratch;
  a.ksteps = v.ksteps;
  a.seed = v.seed;
  a.safety = v.safety;
  a.ratio = v.ratio;
  // the kernel indexes its outputs by global patch id; shift so that patch
  // first_patch lands in entry 0 of the caller's arrays
  a.ritz = ritz_dev - 2 * first_patch;
  a.bounds = bounds_dev - 2 * first_patch;
  const int st = v.dim == 2 ? launch_q<2>(v.q, a, (cudaStream_t)stream) : launch_q<3>(v.q, a, (cudaStream_t)stream);
  if (st == PMG_ERR_UNSUPPORTED)
    return pmg::set_last_error(ctx, st, "noalloc Lanczos: the FP64 working set of this degree exceeds shared memory");
  if (st != PMG_OK) return pmg::set_last_error(ctx, st, cudaGetErrorString(cudaGetLastError()));
  return PMG_OK;
}
