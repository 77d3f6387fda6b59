// Definitions of the launchers declared in launch.h.  Included by the four
// kern_<d>d_<prec>.cu translation units, each of which instantiates them for
// its own dimension and precision (and owns its own constant tables).
#pragma once
#include "global.cuh"
#include "launch.h"

namespace pmg {

// index of the current device for per-device caches (-1 on failure)
inline int current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
  return dev;
}

inline int grid_for(size_t work, int threads) {
  size_t g = (work + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  return (int)g;
}

#define PMG_CHECK_LAUNCH()                              \
  do {                                                  \
    if (cudaPeekAtLastError() != cudaSuccess) return ST_CUDA; \
  } while (0)


template <int DIM, int P, typename T, int V>
int launch_patch_PV(int mode, const PatchArgs<T>& a, cudaStream_t s) {
  using C = Config<DIM, P, T, V>;
  if constexpr (!C::exists) {
    return ST_UNSUPPORTED;
  } else {
    if (a.n_items <= 0) return ST_OK;
    const int grid = (a.n_items + C::PPB - 1) / C::PPB;
    const int dev = current_device();
    if (dev < 0) return ST_CUDA;
    if (mode == MODE_SWEEP) {
      static bool attr[64] = {};                 // the attribute is per device
      if (!attr[dev]) {
        if (cudaFuncSetAttribute(k_patch<DIM, P, T, MODE_SWEEP, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)C::smem) != cudaSuccess)
          return ST_CUDA;
        attr[dev] = true;
      }
      k_patch<DIM, P, T, MODE_SWEEP, V><<<grid, C::NT, C::smem, s>>>(a);
    } else {
      if constexpr (V != 0 && V != VARIANT_PAPER_LEVELS) return ST_UNSUPPORTED;
      static bool attr[64] = {};
      if (!attr[dev]) {
        if (cudaFuncSetAttribute(k_patch<DIM, P, T, MODE_LOCAL, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)C::smem) != cudaSuccess)
          return ST_CUDA;
        attr[dev] = true;
      }
      k_patch<DIM, P, T, MODE_LOCAL, V><<<grid, C::NT, C::smem, s>>>(a);
    }
    PMG_CHECK_LAUNCH();
    return ST_OK;
  }
}

// variants > 0 exist for 3D degrees 3..8 (sweep mode only)
template <int DIM, int P, typename T>
int launch_patch_P(int mode, int variant, const PatchArgs<T>& a, cudaStream_t s) {
  if (variant == 0) return launch_patch_PV<DIM, P, T, 0>(mode, a, s);
  if (variant == VARIANT_PAPER_LEVELS) return launch_patch_PV<DIM, P, T, VARIANT_PAPER_LEVELS>(mode, a, s);
  if constexpr (DIM == 3 && P >= 3) {
    switch (variant) {
      case 1: return launch_patch_PV<DIM, P, T, 1>(mode, a, s);
      case 2: return launch_patch_PV<DIM, P, T, 2>(mode, a, s);
      case 3: return launch_patch_PV<DIM, P, T, 3>(mode, a, s);
      case 4: return launch_patch_PV<DIM, P, T, 4>(mode, a, s);
      case 5: return launch_patch_PV<DIM, P, T, 5>(mode, a, s);
      case 6: return launch_patch_PV<DIM, P, T, 6>(mode, a, s);
      case 7: return launch_patch_PV<DIM, P, T, 7>(mode, a, s);
      case 8: return launch_patch_PV<DIM, P, T, 8>(mode, a, s);
      case 9: return launch_patch_PV<DIM, P, T, 9>(mode, a, s);
      case 10: return launch_patch_PV<DIM, P, T, 10>(mode, a, s);
      case 11: return launch_patch_PV<DIM, P, T, 11>(mode, a, s);
      case 12: return launch_patch_PV<DIM, P, T, 12>(mode, a, s);
      case 13: return launch_patch_PV<DIM, P, T, 13>(mode, a, s);
      case 14: return launch_patch_PV<DIM, P, T, 14>(mode, a, s);
      case 15: return launch_patch_PV<DIM, P, T, 15>(mode, a, s);
      default: return ST_UNSUPPORTED;
    }
  }
  return ST_UNSUPPORTED;
}

// Launch shape of the persistent sweep: the one-patch-per-CTA shape with
// geometry staged in shared memory where it exists (3D, FP32, degree >= 3),
// else the default shape.
template <int DIM, int P, typename T>
constexpr int persist_variant() {
  if constexpr (DIM == 3 && P >= 3 && sizeof(T) == 4) {
    if constexpr (Config<DIM, P, T, 3>::exists) return 3;
  }
  return 0;
}

template <int DIM, int P, typename T>
int launch_patch_persist_P(const PersistArgs<T>& pa, int* grid_out, cudaStream_t s) {
  constexpr int V = persist_variant<DIM, P, T>();
  using C = Config<DIM, P, T, V>;
  if constexpr (!C::exists) {
    return ST_UNSUPPORTED;
  } else {
    const int dev = current_device();
    if (dev < 0) return ST_CUDA;
    static int cap[64] = {};                     // co-resident CTAs of this kernel on the device
    if (!cap[dev]) {
      if (cudaFuncSetAttribute(k_patch_persist<DIM, P, T, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)C::smem) != cudaSuccess)
        return ST_CUDA;
      int per_sm = 0, nsm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_patch_persist<DIM, P, T, V>, C::NT, C::smem) !=
              cudaSuccess ||
          cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return ST_CUDA;
      if (per_sm * nsm <= 0) return ST_UNSUPPORTED;
      cap[dev] = per_sm * nsm;
    }
    int need = 1;
    for (int c = 0; c < pa.n_colours; ++c) need = std::max(need, (pa.counts[c] + C::PPB - 1) / C::PPB);
    const int grid = std::min(need, cap[dev]);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(C::NT);
    cfg.dynamicSmemBytes = C::smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_patch_persist<DIM, P, T, V>, pa) != cudaSuccess) return ST_CUDA;
    if (grid_out) *grid_out = grid;
    return ST_OK;
  }
}

template <int DIM, typename T>
int launch_patch_persist(int P, const PersistArgs<T>& pa, int* grid_out, cudaStream_t s) {
  switch (P) {
    case 1: return launch_patch_persist_P<DIM, 1, T>(pa, grid_out, s);
    case 2: return launch_patch_persist_P<DIM, 2, T>(pa, grid_out, s);
    case 3: return launch_patch_persist_P<DIM, 3, T>(pa, grid_out, s);
    case 4: return launch_patch_persist_P<DIM, 4, T>(pa, grid_out, s);
    case 5: return launch_patch_persist_P<DIM, 5, T>(pa, grid_out, s);
    case 6: return launch_patch_persist_P<DIM, 6, T>(pa, grid_out, s);
    case 7: return launch_patch_persist_P<DIM, 7, T>(pa, grid_out, s);
    case 8: return launch_patch_persist_P<DIM, 8, T>(pa, grid_out, s);
    default: return ST_UNSUPPORTED;
  }
}

template <int DIM, typename T>
int launch_patch(int P, int mode, int variant, const PatchArgs<T>& a, cudaStream_t s) {
  switch (P) {
    case 1: return launch_patch_P<DIM, 1, T>(mode, variant, a, s);
    case 2: return launch_patch_P<DIM, 2, T>(mode, variant, a, s);
    case 3: return launch_patch_P<DIM, 3, T>(mode, variant, a, s);
    case 4: return launch_patch_P<DIM, 4, T>(mode, variant, a, s);
    case 5: return launch_patch_P<DIM, 5, T>(mode, variant, a, s);
    case 6: return launch_patch_P<DIM, 6, T>(mode, variant, a, s);
    case 7: return launch_patch_P<DIM, 7, T>(mode, variant, a, s);
    case 8: return launch_patch_P<DIM, 8, T>(mode, variant, a, s);
    default: return ST_UNSUPPORTED;
  }
}

template <int DIM, int P, typename T, int V>
void patch_config_PV(size_t* smem, int* ppb, int* nt) {
  using C = Config<DIM, P, T, V>;
  const bool ok = C::exists && (V == 0 || V == VARIANT_PAPER_LEVELS || (DIM == 3 && P >= 3));
  *smem = ok ? C::smem : 0;
  *ppb = ok ? C::PPB : 0;
  *nt = ok ? C::NT : 0;
}

template <int DIM, int P, typename T>
void patch_config_P(int variant, size_t* smem, int* ppb, int* nt) {
  if (variant == VARIANT_PAPER_LEVELS) return patch_config_PV<DIM, P, T, VARIANT_PAPER_LEVELS>(smem, ppb, nt);
  switch (variant) {
    case 0: return patch_config_PV<DIM, P, T, 0>(smem, ppb, nt);
    case 1: return patch_config_PV<DIM, P, T, 1>(smem, ppb, nt);
    case 2: return patch_config_PV<DIM, P, T, 2>(smem, ppb, nt);
    case 3: return patch_config_PV<DIM, P, T, 3>(smem, ppb, nt);
    case 4: return patch_config_PV<DIM, P, T, 4>(smem, ppb, nt);
    case 5: return patch_config_PV<DIM, P, T, 5>(smem, ppb, nt);
    case 6: return patch_config_PV<DIM, P, T, 6>(smem, ppb, nt);
    case 7: return patch_config_PV<DIM, P, T, 7>(smem, ppb, nt);
    case 8: return patch_config_PV<DIM, P, T, 8>(smem, ppb, nt);
    case 9: return patch_config_PV<DIM, P, T, 9>(smem, ppb, nt);
    case 10: return patch_config_PV<DIM, P, T, 10>(smem, ppb, nt);
    case 11: return patch_config_PV<DIM, P, T, 11>(smem, ppb, nt);
    case 12: return patch_config_PV<DIM, P, T, 12>(smem, ppb, nt);
    case 13: return patch_config_PV<DIM, P, T, 13>(smem, ppb, nt);
    case 14: return patch_config_PV<DIM, P, T, 14>(smem, ppb, nt);
    case 15: return patch_config_PV<DIM, P, T, 15>(smem, ppb, nt);
    default: *smem = 0; *ppb = 0; *nt = 0;
  }
}

template <int DIM, typename T>
void patch_config(int P, int variant, size_t* smem, int* ppb, int* nt) {
  switch (P) {
    case 1: return patch_config_P<DIM, 1, T>(variant, smem, ppb, nt);
    case 2: return patch_config_P<DIM, 2, T>(variant, smem, ppb, nt);
    case 3: return patch_config_P<DIM, 3, T>(variant, smem, ppb, nt);
    case 4: return patch_config_P<DIM, 4, T>(variant, smem, ppb, nt);
    case 5: return patch_config_P<DIM, 5, T>(variant, smem, ppb, nt);
    case 6: return patch_config_P<DIM, 6, T>(variant, smem, ppb, nt);
    case 7: return patch_config_P<DIM, 7, T>(variant, smem, ppb, nt);
    case 8: return patch_config_P<DIM, 8, T>(variant, smem, ppb, nt);
    default: *smem = 0; *ppb = 0; *nt = 0;
  }
}

template <int DIM, int Q, typename T>
int launch_lanczos_Q(const LanczosArgs<T>& a, cudaStream_t s) {
  constexpr size_t smem = lanczos_smem<DIM, Q, T>();
  if constexpr (smem > 227 * 1024) {
    return ST_UNSUPPORTED;
  } else {
    if (a.n_items <= 0) return ST_OK;
    if (a.ksteps > 64) return ST_ARG;
    static bool attr[64] = {};                   // the attribute is per device
    const int dev = current_device();
    if (dev < 0) return ST_CUDA;
    if (!attr[dev]) {
      if (cudaFuncSetAttribute(k_lanczos<DIM, Q, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
        return ST_CUDA;
      attr[dev] = true;
    }
    k_lanczos<DIM, Q, T><<<a.n_items, 256, smem, s>>>(a);
    PMG_CHECK_LAUNCH();
    return ST_OK;
  }
}

template <int DIM, typename T>
int launch_lanczos(int q, const LanczosArgs<T>& a, cudaStream_t s) {
  switch (q) {
    case 2: return launch_lanczos_Q<DIM, 2, T>(a, s);
    case 3: return launch_lanczos_Q<DIM, 3, T>(a, s);
    case 4: return launch_lanczos_Q<DIM, 4, T>(a, s);
    case 5: return launch_lanczos_Q<DIM, 5, T>(a, s);
    case 6: return launch_lanczos_Q<DIM, 6, T>(a, s);
    case 7: return launch_lanczos_Q<DIM, 7, T>(a, s);
    case 8: return launch_lanczos_Q<DIM, 8, T>(a, s);
    default: return ST_UNSUPPORTED;
  }
}

template <int DIM>
int launch_dense_patch(int q, const double* G64, int N, int first, int n, double* A, cudaStream_t s) {
  if (n <= 0) return ST_OK;
  switch (q) {
    case 2: k_dense_patch<DIM, 2><<<n, 128, dense_patch_smem<DIM, 2>(), s>>>(G64, N, first, n, A); break;
    case 3:
      if constexpr (DIM == 2) { k_dense_patch<DIM, 3><<<n, 128, dense_patch_smem<DIM, 3>(), s>>>(G64, N, first, n, A); break; }
      return ST_UNSUPPORTED;
    case 4:
      if constexpr (DIM == 2) { k_dense_patch<DIM, 4><<<n, 128, dense_patch_smem<DIM, 4>(), s>>>(G64, N, first, n, A); break; }
      return ST_UNSUPPORTED;
    default: return ST_UNSUPPORTED;
  }
  PMG_CHECK_LAUNCH();
  return ST_OK;
}

template <int DIM, int Q, typename T>
int launch_cell_apply_Q(const T* u, T* out, const T* G, int N, cudaStream_t s) {
  constexpr int NT = DIM == 3 ? 128 : 64;
  constexpr int CPB = DIM == 3 ? (Q <= 2 ? 4 : (Q <= 5 ? 2 : 1)) : (Q <= 4 ? 8 : 4);
  using CA = CellApply<DIM, Q, T, NT, CPB>;
  static bool attr[64] = {};                     // the attribute is per device
  const int dev = current_device();
  if (dev < 0) return ST_CUDA;
  if (!attr[dev]) {
    if (cudaFuncSetAttribute(k_cell_apply<DIM, Q, T, NT, CPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)CA::smem) != cudaSuccess)
      return ST_CUDA;
    attr[dev] = true;
  }
  size_t M = (size_t)Q * N + 1, total = 1;
  for (int ax = 0; ax < DIM; ++ax) total *= M;
  k_fill<T><<<grid_for(total, 256), 256, 0, s>>>(out, total, T(0));
  const int Nh = (N + 1) / 2;
  int nclass = 1;
  for (int ax = 0; ax < DIM; ++ax) nclass *= Nh;
  const int grid = (nclass + CPB - 1) / CPB;
  for (int par = 0; par < (1 << DIM); ++par)
    k_cell_apply<DIM, Q, T, NT, CPB><<<grid, NT, CA::smem, s>>>(u, out, G, N, par);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}

template <int DIM, typename T>
int launch_cell_apply(int q, const T* u, T* out, const T* G, int N, cudaStream_t s) {
  switch (q) {
    case 1: return launch_cell_apply_Q<DIM, 1, T>(u, out, G, N, s);
    case 2: return launch_cell_apply_Q<DIM, 2, T>(u, out, G, N, s);
    case 3: return launch_cell_apply_Q<DIM, 3, T>(u, out, G, N, s);
    case 4: return launch_cell_apply_Q<DIM, 4, T>(u, out, G, N, s);
    case 5: return launch_cell_apply_Q<DIM, 5, T>(u, out, G, N, s);
    case 6: return launch_cell_apply_Q<DIM, 6, T>(u, out, G, N, s);
    case 7: return launch_cell_apply_Q<DIM, 7, T>(u, out, G, N, s);
    case 8: return launch_cell_apply_Q<DIM, 8, T>(u, out, G, N, s);
    default: return ST_UNSUPPORTED;
  }
}

template <int DIM, typename T>
int launch_geometry(const double* coords, const double* kappa, int N, int q, T* G, int* err, cudaStream_t s) {
  size_t ncell = 1, ngc = 1;
  for (int ax = 0; ax < DIM; ++ax) { ncell *= N; ngc *= (q + 1); }
  k_geometry<DIM, T><<<grid_for(ncell * ngc, 256), 256, 0, s>>>(coords, kappa, N, q, G, err);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}

template <int DIM, typename T>
int launch_additive_update(T* u, const T* corr, double theta, int weighted, int q, int N, cudaStream_t s) {
  size_t nd = 1;
  for (int ax = 0; ax < DIM; ++ax) nd *= (size_t)q * N + 1;
  k_additive_update<DIM, T><<<grid_for(nd, 256), 256, 0, s>>>(u, corr, T(theta), weighted, q, N);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}

template <int DIM>
int launch_diag(const double* G64, int N, int q, double* diag, double* dinv64, float* dinv32, cudaStream_t s) {
  const size_t M = (size_t)q * N + 1;
  size_t total = 1, ngc = 1;
  for (int ax = 0; ax < DIM; ++ax) { total *= M; ngc *= (q + 1); }
  k_fill<double><<<grid_for(total, 256), 256, 0, s>>>(diag, total, 0.0);
  const int Nh = (N + 1) / 2;
  size_t nclass = 1;
  for (int ax = 0; ax < DIM; ++ax) nclass *= Nh;
  for (int par = 0; par < (1 << DIM); ++par)
    k_diag<DIM><<<grid_for(nclass * ngc, 128), 128, 0, s>>>(G64, N, q, par, diag);
  k_invert_diag<DIM, float><<<grid_for(total, 256), 256, 0, s>>>(diag, (int)M, dinv64, dinv32);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}

template <int DIM>
int launch_rhs_manufactured(const double* coords, int N, int q, double* b, cudaStream_t s) {
  const size_t M = (size_t)q * N + 1;
  size_t total = 1, nn = 1;
  for (int ax = 0; ax < DIM; ++ax) { total *= M; nn *= (q + 1); }
  k_fill<double><<<grid_for(total, 256), 256, 0, s>>>(b, total, 0.0);
  const int Nh = (N + 1) / 2;
  size_t nclass = 1;
  for (int ax = 0; ax < DIM; ++ax) nclass *= Nh;
  for (int par = 0; par < (1 << DIM); ++par)
    k_rhs_manufactured<DIM><<<grid_for(nclass * nn, 128), 128, 0, s>>>(coords, N, q, par, b);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}

template <typename T>
int launch_band_sweep(const T* in, T* out, const double* W, const int* start, int width, int Lin, int Lout, size_t O,
                      size_t I, int mask, cudaStream_t s) {
  const size_t total = O * (size_t)Lout * I;
  k_band_sweep<T><<<grid_for(total, 256), 256, 0, s>>>(in, out, W, start, width, Lin, Lout, O, I, mask);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}

template <typename T>
int launch_fill(T* x, size_t n, T v, cudaStream_t s) {
  k_fill<T><<<grid_for(n, 256), 256, 0, s>>>(x, n, v);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}
template <typename T>
int launch_sub_from(const T* x, T* y, size_t n, cudaStream_t s) {
  k_sub_from<T><<<grid_for(n, 256), 256, 0, s>>>(x, y, n);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}
template <typename T>
int launch_add_to(const T* x, T* y, size_t n, cudaStream_t s) {
  k_add_to<T><<<grid_for(n, 256), 256, 0, s>>>(x, y, n);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}
template <int DIM, typename T>
int launch_mask_boundary(T* x, int M, cudaStream_t s) {
  size_t total = 1;
  for (int ax = 0; ax < DIM; ++ax) total *= M;
  k_mask_boundary<DIM, T><<<grid_for(total, 256), 256, 0, s>>>(x, M);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}
template <typename T>
int launch_coarse_gemv(const double* Ainv, const int* freeidx, int nf, const T* b, T* x, cudaStream_t s) {
  const int warps = nf < 152 * 16 ? nf : 152 * 16;
  k_coarse_gemv<T><<<(warps * 32 + 255) / 256, 256, 0, s>>>(Ainv, freeidx, nf, b, x);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}

template <typename T>
int launch_fma_chain(T* out, int grid, int block, int iters, cudaStream_t s) {
  k_fma_chain<T><<<grid, block, 0, s>>>(out, iters, T(0.9999999), T(1e-7));
  PMG_CHECK_LAUNCH();
  return ST_OK;
}

}  // namespace pmg

// Explicit instantiation of the patch kernels of one degree (their own
// translation unit each in 3D, so that they compile in parallel).
#define PMG_INSTANTIATE_PATCH(DIM, T, P)                                                   \
  namespace pmg {                                                                          \
  template int launch_patch_P<DIM, P, T>(int, int, const PatchArgs<T>&, cudaStream_t);     \
  template int launch_patch_persist_P<DIM, P, T>(const PersistArgs<T>&, int*, cudaStream_t); \
  }
// One launch-shape variant of a degree in a translation unit of its own (the
// heaviest degrees are split so that the build runs them in parallel), and
// the declaration that keeps the dispatcher's unit from instantiating it.
#define PMG_INSTANTIATE_PATCH_V(DIM, T, P, V)                                              \
  namespace pmg {                                                                          \
  template int launch_patch_PV<DIM, P, T, V>(int, const PatchArgs<T>&, cudaStream_t);      \
  }
#define PMG_EXTERN_PATCH_V(DIM, T, P, V)                                                   \
  namespace pmg {                                                                          \
  extern template int launch_patch_PV<DIM, P, T, V>(int, const PatchArgs<T>&, cudaStream_t); \
  }
// ... and the declarations that keep other translation units from
// instantiating them again.
#define PMG_EXTERN_PATCH(DIM, T, P)                                                        \
  namespace pmg {                                                                          \
  extern template int launch_patch_P<DIM, P, T>(int, int, const PatchArgs<T>&, cudaStream_t); \
  extern template int launch_patch_persist_P<DIM, P, T>(const PersistArgs<T>&, int*, cudaStream_t); \
  }

#define PMG_INSTANTIATE_DIM_T(DIM, T)                                                                       \
  namespace pmg {                                                                                           \
  template int launch_patch<DIM, T>(int, int, int, const PatchArgs<T>&, cudaStream_t);                      \
  template int launch_patch_persist<DIM, T>(int, const PersistArgs<T>&, int*, cudaStream_t);               \
  template void patch_config<DIM, T>(int, int, size_t*, int*, int*);                                        \
  template int launch_lanczos<DIM, T>(int, const LanczosArgs<T>&, cudaStream_t);                            \
  template int launch_cell_apply<DIM, T>(int, const T*, T*, const T*, int, cudaStream_t);                   \
  template int launch_geometry<DIM, T>(const double*, const double*, int, int, T*, int*, cudaStream_t);     \
  template int launch_additive_update<DIM, T>(T*, const T*, double, int, int, int, cudaStream_t);            \
  template int launch_mask_boundary<DIM, T>(T*, int, cudaStream_t);                                         \
  }
