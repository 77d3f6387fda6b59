// Patch kernels for d = 3 in FP32, degree(s) 3 (see kernels_impl.cuh).
#include "kernels_impl.cuh"
PMG_INSTANTIATE_PATCH(3, float, 3)
