// Kernels for d = 3 in FP32, and the precision-generic FP32 helpers.
#include <cuda_bf16.h>

#include "kernels_impl.cuh"
PMG_EXTERN_PATCH(3, float, 1)
PMG_EXTERN_PATCH(3, float, 2)
PMG_EXTERN_PATCH(3, float, 3)
PMG_EXTERN_PATCH(3, float, 4)
PMG_EXTERN_PATCH(3, float, 5)
PMG_EXTERN_PATCH(3, float, 6)
PMG_EXTERN_PATCH(3, float, 7)
PMG_EXTERN_PATCH(3, float, 8)
PMG_INSTANTIATE_DIM_T(3, float)
namespace pmg {
template int launch_fma_chain<float>(float*, int, int, int, cudaStream_t);
template int launch_band_sweep<float>(const float*, float*, const double*, const int*, int, int, int, size_t, size_t,
                                      int, cudaStream_t);
template int launch_fill<float>(float*, size_t, float, cudaStream_t);
template int launch_sub_from<float>(const float*, float*, size_t, cudaStream_t);
template int launch_add_to<float>(const float*, float*, size_t, cudaStream_t);
template int launch_coarse_gemv<float>(const double*, const int*, int, const float*, float*, cudaStream_t);

__global__ void k_round_bf16(const float* __restrict__ x, float* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = __bfloat162float(__float2bfloat16_rn(x[i]));
}
int launch_round_bf16(const float* x, float* y, size_t n, cudaStream_t s) {
  k_round_bf16<<<grid_for(n, 256), 256, 0, s>>>(x, y, n);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}

// [cell][ncomp][npt] FP32 values that are BF16 numbers -> [cell][(ncomp + 1) / 2][npt] words holding
// components 2j (low half) and 2j + 1 (high half, zero past the last component); exact
__global__ void k_pack_bf16(const float* __restrict__ x, unsigned* __restrict__ y, size_t ncell, int ncomp,
                            int npt) {
  const int npair = (ncomp + 1) / 2;
  const size_t n = ncell * npair * (size_t)npt;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int pt = (int)(i % npt);
    const size_t r = i / npt;
    const int j = (int)(r % npair);
    const size_t c = r / npair;
    const float* xc = x + c * ncomp * (size_t)npt + pt;
    const unsigned lo = __float_as_uint(xc[(2 * j) * (size_t)npt]) >> 16;
    const unsigned hi = 2 * j + 1 < ncomp ? __float_as_uint(xc[(2 * j + 1) * (size_t)npt]) & 0xffff0000u : 0u;
    y[i] = hi | lo;
  }
}
int launch_pack_bf16(const float* x, unsigned* y, size_t ncell, int ncomp, int npt, cudaStream_t s) {
  k_pack_bf16<<<grid_for(ncell * ((ncomp + 1) / 2) * (size_t)npt, 256), 256, 0, s>>>(x, y, ncell, ncomp, npt);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}
}  // namespace pmg
