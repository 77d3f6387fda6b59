// Unstructured-mesh kernels for d = 3, degrees 5 and 6 (patch sweeps and local solves, cell
// applies, Lanczos intervals).
#include "umesh_launch.cuh"

namespace pmg {
PMG_UMESH_INSTANTIATE(3, 5, double)
PMG_UMESH_INSTANTIATE(3, 5, float)
PMG_UMESH_INSTANTIATE(3, 6, double)
PMG_UMESH_INSTANTIATE(3, 6, float)
PMG_UMESH_INSTANTIATE_LANCZOS(3, 5)
PMG_UMESH_INSTANTIATE_LANCZOS(3, 6)
}  // namespace pmg
