// Patch kernels for d = 3 in FP64, degree(s) 5 (see kernels_impl.cuh).
#include "kernels_impl.cuh"
PMG_INSTANTIATE_PATCH(3, double, 5)
