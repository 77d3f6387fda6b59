// Unstructured-mesh kernels for d = 3, degrees 1-4 (patch sweeps and local solves, cell
// applies, Lanczos intervals).
#include "umesh_launch.cuh"

namespace pmg {
PMG_UMESH_INSTANTIATE(3, 1, double)
PMG_UMESH_INSTANTIATE(3, 1, float)
PMG_UMESH_INSTANTIATE(3, 2, double)
PMG_UMESH_INSTANTIATE(3, 2, float)
PMG_UMESH_INSTANTIATE(3, 3, double)
PMG_UMESH_INSTANTIATE(3, 3, float)
PMG_UMESH_INSTANTIATE(3, 4, double)
PMG_UMESH_INSTANTIATE(3, 4, float)
PMG_UMESH_INSTANTIATE_LANCZOS(3, 2)
PMG_UMESH_INSTANTIATE_LANCZOS(3, 3)
PMG_UMESH_INSTANTIATE_LANCZOS(3, 4)
}  // namespace pmg
