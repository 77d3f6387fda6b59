// pmg_lanczos_bounds_noalloc: the per-patch Lanczos eigenvalue estimates of
// pmg_compute_bounds for a range of patches, for callers that must not
// allocate device memory.
//
// Who cannot allocate: code inside a framework that owns the device memory
// budget through its own caching allocator and forbids raw cudaMalloc/cudaFree
// (which also synchronise the device), and long-running or latency-critical
// solvers that recompute Chebyshev bounds mid-run and must not stall on, or
// fail in, an allocation.  pmg_compute_bounds needs a device buffer for the
// Lanczos basis; this entry point uses a fixed file-scope device array
// instead.
//
// The array (kScratchBytes = 16 MiB) is part of the library image: every GPU
// that loads the library holds it until the process exits.  All calls share
// it and it keeps whatever the last call wrote.  The Lanczos kernel writes
// every basis vector before reading it, so nothing needs clearing.  Calls
// whose kernels overlap on the GPU (different streams, or different contexts
// on one device) race on the array: serialise them.
//
// Degrees whose FP64 working set does not fit in shared memory (3D q >= 7)
// use the FP32 operator with FP64 Lanczos vectors, as pmg_compute_bounds
// does; that needs the context's FP32 geometry, which mixed-precision
// contexts always hold and FP64 contexts hold once pmg_compute_bounds has
// taken that fallback.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/pmg.h"
#include "basis.h"
#include "device_guard.h"
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

template <int DIM, int Q, typename T>
cudaError_t set_smem_attr() {
  constexpr size_t smem = pmg::lanczos_smem<DIM, Q, T>();
  if constexpr (smem > 227 * 1024) {
    return cudaSuccess;
  } else {
    return cudaFuncSetAttribute(pmg::k_lanczos<DIM, Q, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
}

template <typename T>
cudaError_t set_smem_attrs() {
  cudaError_t a[] = {set_smem_attr<2, 2, T>(), set_smem_attr<2, 3, T>(), set_smem_attr<2, 4, T>(),
                     set_smem_attr<2, 5, T>(), set_smem_attr<2, 6, T>(), set_smem_attr<2, 7, T>(),
                     set_smem_attr<2, 8, T>(), set_smem_attr<3, 2, T>(), set_smem_attr<3, 3, T>(),
                     set_smem_attr<3, 4, T>(), set_smem_attr<3, 5, T>(), set_smem_attr<3, 6, T>(),
                     set_smem_attr<3, 7, T>(), set_smem_attr<3, 8, T>()};
  for (cudaError_t x : a)
    if (x != cudaSuccess) return x;
  return cudaSuccess;
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
  e = set_smem_attrs<double>();
  if (e != cudaSuccess) return e;
  e = set_smem_attrs<float>();
  if (e != cudaSuccess) return e;
  double* ptr = nullptr;
  e = cudaGetSymbolAddress((void**)&ptr, g_lanczos_scratch);
  if (e != cudaSuccess) return e;
  g_dev[dev].scratch = ptr;
  g_dev[dev].ready = true;
  return cudaSuccess;
}

template <int DIM, int Q, typename T>
int launch(const pmg::LanczosArgs<T>& a, cudaStream_t s) {
  constexpr size_t smem = pmg::lanczos_smem<DIM, Q, T>();
  if constexpr (smem > 227 * 1024) {
    return PMG_ERR_UNSUPPORTED;
  } else {
    pmg::k_lanczos<DIM, Q, T><<<a.n_items, 256, smem, s>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? PMG_OK : PMG_ERR_CUDA;
  }
}

template <int DIM, typename T>
int launch_q(int q, const pmg::LanczosArgs<T>& a, cudaStream_t s) {
  switch (q) {
    case 2: return launch<DIM, 2, T>(a, s);
    case 3: return launch<DIM, 3, T>(a, s);
    case 4: return launch<DIM, 4, T>(a, s);
    case 5: return launch<DIM, 5, T>(a, s);
    case 6: return launch<DIM, 6, T>(a, s);
    case 7: return launch<DIM, 7, T>(a, s);
    case 8: return launch<DIM, 8, T>(a, s);
    default: return PMG_ERR_UNSUPPORTED;
  }
}

template <typename T>
void fill_args(pmg::LanczosArgs<T>& a, const pmg::LanczosView& v, int64_t first_patch, int64_t n_patches,
               double* scratch, double* ritz_dev, double* bounds_dev) {
  a.N = v.N;
  a.n_items = (int)n_patches;
  a.first_patch = (int)first_patch;
  a.V = scratch;
  a.ksteps = v.ksteps;
  a.seed = v.seed;
  a.safety = v.safety;
  a.ratio = v.ratio;
  a.ritz = ritz_dev;
  a.bounds = nullptr;
  a.bounds_f64 = bounds_dev;
  a.out_offset = first_patch;      // patch first_patch lands in entry 0 of the caller's arrays
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
  pmg::DeviceGuard guard(v.device);
  if (guard.err != cudaSuccess)
    return pmg::set_last_error(ctx, PMG_ERR_CUDA, "noalloc Lanczos: cudaGetDevice/cudaSetDevice failed");
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev[v.device].ready) {
      cudaError_t e = setup_device(v.device);
      if (e != cudaSuccess) return pmg::set_last_error(ctx, PMG_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  if (n_patches == 0) return PMG_OK;
  cudaStream_t s = (cudaStream_t)stream;
  double* scratch = g_dev[v.device].scratch;
  pmg::LanczosArgs<double> a;
  fill_args(a, v, first_patch, n_patches, scratch, ritz_dev, bounds_dev);
  a.G = v.G64;
  a.dinv = v.dinv64;
  int st = v.dim == 2 ? launch_q<2, double>(v.q, a, s) : launch_q<3, double>(v.q, a, s);
  if (st == PMG_ERR_UNSUPPORTED) {
    // the FP64 working set does not fit: FP32 operator, FP64 Lanczos vectors
    if (!v.G32 || !v.dinv32)
      return pmg::set_last_error(ctx, PMG_ERR_UNSUPPORTED,
                                 "noalloc Lanczos: this degree needs the FP32 geometry copy, which this FP64 context "
                                 "has not made (pmg_compute_bounds with Lanczos bounds makes it)");
    pmg::LanczosArgs<float> b;
    fill_args(b, v, first_patch, n_patches, scratch, ritz_dev, bounds_dev);
    b.G = v.G32;
    b.dinv = v.dinv32;
    st = v.dim == 2 ? launch_q<2, float>(v.q, b, s) : launch_q<3, float>(v.q, b, s);
  }
  if (st == PMG_ERR_UNSUPPORTED)
    return pmg::set_last_error(ctx, st, "noalloc Lanczos: the working set of this degree exceeds shared memory");
  if (st != PMG_OK) return pmg::set_last_error(ctx, st, cudaGetErrorString(cudaGetLastError()));
  return PMG_OK;
}
