// Kernels for d = 2 in FP32 (see kernels_impl.cuh).
#include "kernels_impl.cuh"
PMG_INSTANTIATE_DIM_T(2, float)
