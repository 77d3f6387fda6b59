// Patch kernels for d = 3 in FP32, degree 7 (see kernels_impl.cuh): the
// dispatcher and variants 0-3; variants 4-7 are compiled in
// kern_patch3d_f32_q7b.cu.
#include "kernels_impl.cuh"
PMG_EXTERN_PATCH_V(3, float, 7, 4)
PMG_EXTERN_PATCH_V(3, float, 7, 5)
PMG_EXTERN_PATCH_V(3, float, 7, 6)
PMG_EXTERN_PATCH_V(3, float, 7, 7)
PMG_INSTANTIATE_PATCH(3, float, 7)
