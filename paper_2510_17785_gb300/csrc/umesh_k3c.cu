// Unstructured-mesh kernels for d = 3, degree 7 (patch sweeps and local solves, cell
// applies, Lanczos intervals).
#include "umesh_launch.cuh"

namespace pmg {
PMG_UMESH_INSTANTIATE(3, 7, double)
PMG_UMESH_INSTANTIATE(3, 7, float)
PMG_UMESH_INSTANTIATE_LANCZOS(3, 7)
}  // namespace pmg
