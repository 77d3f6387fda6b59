// Kernels for d = 2 in FP64 (see kernels_impl.cuh).
#include "kernels_impl.cuh"
PMG_INSTANTIATE_DIM_T(2, double)
namespace pmg {
template int launch_dense_patch<2>(int, const double*, int, int, int, double*, cudaStream_t);
template int launch_diag<2>(const double*, int, int, double*, double*, float*, cudaStream_t);
template int launch_rhs_manufactured<2>(const double*, int, int, double*, cudaStream_t);
}  // namespace pmg
