// Unstructured-mesh kernels for d = 3, degree 8 (patch sweeps and local solves, cell
// applies, Lanczos intervals).
#include "umesh_launch.cuh"

namespace pmg {
PMG_UMESH_INSTANTIATE(3, 8, double)
PMG_UMESH_INSTANTIATE(3, 8, float)
PMG_UMESH_INSTANTIATE_LANCZOS(3, 8)
}  // namespace pmg
