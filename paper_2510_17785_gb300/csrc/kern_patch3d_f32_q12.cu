// Patch kernels for d = 3 in FP32, degree(s) 1, 2 (see kernels_impl.cuh).
#include "kernels_impl.cuh"
PMG_INSTANTIATE_PATCH(3, float, 1)
PMG_INSTANTIATE_PATCH(3, float, 2)
