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
}  // namespace pmg
