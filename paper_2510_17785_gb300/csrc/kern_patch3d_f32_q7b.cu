// Patch kernels for d = 3 in FP32, degree 7: launch-shape variants 4-7
// (see kern_patch3d_f32_q7.cu).
#include "kernels_impl.cuh"
PMG_INSTANTIATE_PATCH_V(3, float, 7, 4)
PMG_INSTANTIATE_PATCH_V(3, float, 7, 5)
PMG_INSTANTIATE_PATCH_V(3, float, 7, 6)
PMG_INSTANTIATE_PATCH_V(3, float, 7, 7)
