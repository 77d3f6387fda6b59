// Host-side launchers of the device kernels, explicitly instantiated per
// (dimension, precision) in kern_<d>d_<prec>.cu.
#pragma once
#include <string>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cg_slots.h"
#include "patch.cuh"

namespace pmg {

// status codes (mirrors pmg.h)
enum { ST_OK = 0, ST_ARG = 1, ST_CUDA = 2, ST_DEGENERATE = 3, ST_NOT_SPD = 5, ST_UNSUPPORTED = 7 };


// one launch of the patch kernel over a.n_items patches (MODE_SWEEP or
// MODE_LOCAL) with launch-shape variant `variant` (0 = default; ST_UNSUPPORTED
// if the variant does not exist for this degree)
template <int DIM, typename T>
int launch_patch(int P, int mode, int variant, const PatchArgs<T>& a, cudaStream_t s);
// y = x rounded to BF16 (round to nearest even) and widened back to FP32
int launch_round_bf16(const float* x, float* y, size_t n, cudaStream_t s);
// geometry tensors already rounded to BF16, [cell][ncomp][npt] FP32 -> the
// packed pairs the FP32 patch kernels read, [cell][(ncomp + 1) / 2][npt]
// words (component 2j in the low half, 2j + 1 in the high half)
int launch_pack_bf16(const float* x, unsigned* y, size_t ncell, int ncomp, int npt, cudaStream_t s);
// one persistent cooperative launch sweeping every colour of a level
// (pa.n_colours lists, grid barrier between colours); *grid_out = CTAs used
template <int DIM, typename T>
int launch_patch_persist(int P, const PersistArgs<T>& pa, int* grid_out, cudaStream_t s);
// shared memory bytes per CTA, patches per CTA and threads per CTA of a
// variant of the patch kernel (all 0 if it does not exist)
template <int DIM, typename T>
void patch_config(int P, int variant, size_t* smem, int* ppb, int* nthreads);

template <int DIM, typename T>
int launch_lanczos(int q, const LanczosArgs<T>& a, cudaStream_t s);

// out = A u on the degree-q grid (zero fill + 2^DIM parity classes)
template <int DIM, typename T>
int launch_cell_apply(int q, const T* u, T* out, const T* G, int N, cudaStream_t s);

// dense patch matrices [n][Ni][Ni] of patches first .. first+n-1 at degree q (FP64)
template <int DIM>
int launch_dense_patch(int q, const double* G64, int N, int first, int n, double* A, cudaStream_t s);

template <int DIM, typename T>
int launch_geometry(const double* coords, const double* kappa, int N, int q, T* G, int* err, cudaStream_t s);
// additive sweep: u += theta (W) corr on free DoFs (W = 1 / patch multiplicity)
template <int DIM, typename T>
int launch_additive_update(T* u, const T* corr, double theta, int weighted, int q, int N, cudaStream_t s);

// FP64 only
template <int DIM>
int launch_diag(const double* G64, int N, int q, double* diag, double* dinv64, float* dinv32, cudaStream_t s);
template <int DIM>
int launch_rhs_manufactured(const double* coords, int N, int q, double* b, cudaStream_t s);

// precision-generic helpers (instantiated in the 3D translation units)
template <typename T>
int launch_band_sweep(const T* in, T* out, const double* W, const int* start, int width, int Lin, int Lout, size_t O,
                      size_t I, int mask, cudaStream_t s);
template <typename T>
int launch_fill(T* x, size_t n, T v, cudaStream_t s);
template <typename T>
int launch_sub_from(const T* x, T* y, size_t n, cudaStream_t s);
template <typename T>
int launch_add_to(const T* x, T* y, size_t n, cudaStream_t s);
template <int DIM, typename T>
int launch_mask_boundary(T* x, int M, cudaStream_t s);
template <typename T>
int launch_coarse_gemv(const double* Ainv, const int* freeidx, int nf, const T* b, T* x, cudaStream_t s);

// casts and CG vector ops (FP64 translation unit of 3D)
int launch_cast_d2f(const double* x, float* y, size_t n, cudaStream_t s);
int launch_cast_f2d(const float* x, double* y, size_t n, cudaStream_t s);
int launch_dot(const double* x, const double* y, size_t n, double* partial, double* scal, int slot, int op,
               cudaStream_t s);
int launch_axpy(double a, const double* x, double* y, size_t n, cudaStream_t s);
// dense coarse solver set-up (coarse.cu)
int launch_unit(double* x, size_t idx, cudaStream_t s);
int launch_gather_coarse(const double* cols, const int* fidx, int nf, size_t nd, double* A, cudaStream_t s);
int coarse_inverse(double* A, int n, cudaStream_t s, std::string* msg);
int launch_scale(double a, const double* x, double* y, size_t n, cudaStream_t s);
int launch_cg_update_p(const double* z, double* p, const double* scal, size_t n, cudaStream_t s);
int launch_cg_update_xr(double* x, double* r, const double* p, const double* Ap, const double* scal, size_t n,
                        cudaStream_t s);

// FMA microbenchmark: grid x block threads, each 32 * iters FMAs
template <typename T>
int launch_fma_chain(T* out, int grid, int block, int iters, cudaStream_t s);

}  // namespace pmg
