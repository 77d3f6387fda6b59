// Kernels for d = 3 in FP64, the precision-generic FP64 helpers, and the
// FP64 CG vector operations.
#include "kernels_impl.cuh"
PMG_EXTERN_PATCH(3, double, 1)
PMG_EXTERN_PATCH(3, double, 2)
PMG_EXTERN_PATCH(3, double, 3)
PMG_EXTERN_PATCH(3, double, 4)
PMG_EXTERN_PATCH(3, double, 5)
PMG_EXTERN_PATCH(3, double, 6)
PMG_EXTERN_PATCH(3, double, 7)
PMG_EXTERN_PATCH(3, double, 8)
PMG_INSTANTIATE_DIM_T(3, double)
namespace pmg {
template int launch_dense_patch<3>(int, const double*, int, int, int, double*, cudaStream_t);
template int launch_fma_chain<double>(double*, int, int, int, cudaStream_t);
template int launch_diag<3>(const double*, int, int, double*, double*, float*, cudaStream_t);
template int launch_rhs_manufactured<3>(const double*, int, int, double*, cudaStream_t);
template int launch_band_sweep<double>(const double*, double*, const double*, const int*, int, int, int, size_t,
                                       size_t, int, cudaStream_t);
template int launch_fill<double>(double*, size_t, double, cudaStream_t);
template int launch_sub_from<double>(const double*, double*, size_t, cudaStream_t);
template int launch_add_to<double>(const double*, double*, size_t, cudaStream_t);
template int launch_coarse_gemv<double>(const double*, const int*, int, const double*, double*, cudaStream_t);

int launch_cast_d2f(const double* x, float* y, size_t n, cudaStream_t s) {
  k_cast<double, float><<<grid_for(n, 256), 256, 0, s>>>(x, y, n);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}
int launch_cast_f2d(const float* x, double* y, size_t n, cudaStream_t s) {
  k_cast<float, double><<<grid_for(n, 256), 256, 0, s>>>(x, y, n);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}
int launch_dot(const double* x, const double* y, size_t n, double* partial, double* scal, int slot, int op,
               cudaStream_t s) {
  k_dot_partial<<<DOT_BLOCKS, DOT_THREADS, 0, s>>>(x, y, n, partial);
  k_dot_final<<<1, 1024, 0, s>>>(partial, DOT_BLOCKS, scal, slot, op);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}
int launch_axpy(double a, const double* x, double* y, size_t n, cudaStream_t s) {
  k_axpy<<<grid_for(n, 256), 256, 0, s>>>(a, x, y, n);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}
int launch_scale(double a, const double* x, double* y, size_t n, cudaStream_t s) {
  k_scale<<<grid_for(n, 256), 256, 0, s>>>(a, x, y, n);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}
int launch_cg_update_p(const double* z, double* p, const double* scal, size_t n, cudaStream_t s) {
  k_cg_update_p<<<grid_for(n, 256), 256, 0, s>>>(z, p, scal, n);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}
int launch_cg_update_xr(double* x, double* r, const double* p, const double* Ap, const double* scal, size_t n,
                        cudaStream_t s) {
  k_cg_update_xr<<<grid_for(n, 256), 256, 0, s>>>(x, r, p, Ap, scal, n);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}
}  // namespace pmg
