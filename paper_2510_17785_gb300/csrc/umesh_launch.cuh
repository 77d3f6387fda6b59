// Definitions of the unstructured-mesh launchers declared in umesh_kern.cuh,
// included only by the explicit-instantiation units umesh_k*.cu.
#pragma once
#include "umesh_kern.cuh"

namespace pmg {

template <int DIM, int Q, typename T>
int ucell_apply_q(const T* u, const T* G, const int32_t* cd, const uint8_t* bnd, int64_t nc, T* Y,
                         cudaStream_t s) {
  constexpr int CPB = ucpb(Q);
  constexpr size_t sm = ucell_smem<DIM, Q, T>();
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (!attr[dev & 63]) {
    if (cudaFuncSetAttribute(k_ucell_apply<DIM, Q, T, CPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
        cudaSuccess)
      return ST_CUDA;
    attr[dev & 63] = true;
  }
  const int64_t grid = (nc + CPB - 1) / CPB;
  k_ucell_apply<DIM, Q, T, CPB><<<(unsigned)grid, 128, sm, s>>>(u, G, cd, bnd, nc, Y);
  return cudaPeekAtLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

template <int DIM, int P, typename T>
int upatch_launch_P(int mode, const UPatchArgs<T>& a, int grid, cudaStream_t s) {
  constexpr size_t sm0 = upatch_smem<DIM, P, T>();
  if constexpr (sm0 > 227 * 1024) {
    return ST_UNSUPPORTED;
  } else {
    // the workspace slice joins the shared memory when the caller says it fits
    const size_t sm = a.ws_shared ? upatch_smem_aligned<DIM, P, T>() + a.ws_stride * sizeof(T) : sm0;
    if (sm > 227 * 1024) return ST_ARG;
    int dev = 0;
    cudaGetDevice(&dev);
    static size_t attr[2][64] = {};                  // largest dynamic size set so far, per device
    if (mode == MODE_SWEEP) {
      if (attr[0][dev & 63] < sm) {
        if (cudaFuncSetAttribute(k_upatch<DIM, P, T, MODE_SWEEP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm) != cudaSuccess)
          return ST_CUDA;
        attr[0][dev & 63] = sm;
      }
      k_upatch<DIM, P, T, MODE_SWEEP><<<grid, unt(P), sm, s>>>(a);
    } else {
      if (attr[1][dev & 63] < sm) {
        if (cudaFuncSetAttribute(k_upatch<DIM, P, T, MODE_LOCAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm) != cudaSuccess)
          return ST_CUDA;
        attr[1][dev & 63] = sm;
      }
      k_upatch<DIM, P, T, MODE_LOCAL><<<grid, unt(P), sm, s>>>(a);
    }
    return cudaPeekAtLastError() == cudaSuccess ? ST_OK : ST_CUDA;
  }
}

// bytes of dynamic shared memory of the patch kernel without its workspace
template <int DIM, int P, typename T>
size_t upatch_smem_base() {
  return upatch_smem_aligned<DIM, P, T>();
}

template <int DIM, int P>
int ulanczos_launch(const UPatchArgs<double>& a, const ULanczos& z, int grid, cudaStream_t s) {
  constexpr size_t sm = upatch_smem<DIM, P, double>();
  if constexpr (sm > 200 * 1024) {
    return ST_UNSUPPORTED;
  } else {
    static bool attr[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (!attr[dev & 63]) {
      if (cudaFuncSetAttribute(k_ulanczos<DIM, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return ST_CUDA;
      attr[dev & 63] = true;
    }
    k_ulanczos<DIM, P><<<grid, unt(P), sm, s>>>(a, z);
    return cudaPeekAtLastError() == cudaSuccess ? ST_OK : ST_CUDA;
  }
}

#define PMG_UMESH_INSTANTIATE(DIM, P, T)                                                                     \
  template int upatch_launch_P<DIM, P, T>(int, const UPatchArgs<T>&, int, cudaStream_t);                   \
  template int ucell_apply_q<DIM, P, T>(const T*, const T*, const int32_t*, const uint8_t*, int64_t, T*, \
                                        cudaStream_t);
#define PMG_UMESH_INSTANTIATE_LANCZOS(DIM, P) \
  template int ulanczos_launch<DIM, P>(const UPatchArgs<double>&, const ULanczos&, int, cudaStream_t);

}  // namespace pmg
