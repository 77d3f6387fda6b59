// Dense FP64 coarse solver set-up on the device: the coarsest-level matrix is
// assembled column by column (the operator applied to unit vectors, no host
// round trip per column), then factorised (Cholesky) and inverted with
// cuSOLVER.  Set-up only: the V-cycle applies the inverse with k_coarse_gemv.
#include <cusolverDn.h>

#include <string>

#include "kernels_impl.cuh"

namespace pmg {

static __global__ void k_unit(double* x, size_t idx) { x[idx] = 1.0; }

// A[i][j] = (C_j[f_i] + C_i[f_j]) / 2: column j of the operator (C_j, length
// nd) restricted to the free DoFs f, with the rounding symmetrised
static __global__ void k_gather_coarse(const double* __restrict__ cols, const int* __restrict__ fidx, int nf,
                                       size_t nd, double* __restrict__ A) {
  const size_t tot = (size_t)nf * nf;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / nf), j = (int)(e - (size_t)i * nf);
    A[e] = 0.5 * (cols[(size_t)j * nd + fidx[i]] + cols[(size_t)i * nd + fidx[j]]);
  }
}

// copy the lower triangle (column-major) onto the upper one
static __global__ void k_mirror_lower(double* A, int n) {
  const size_t tot = (size_t)n * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / n), r = (int)(e - (size_t)c * n);
    if (r < c) A[e] = A[(size_t)r * n + c];
  }
}

int launch_unit(double* x, size_t idx, cudaStream_t s) {
  k_unit<<<1, 1, 0, s>>>(x, idx);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}

int launch_gather_coarse(const double* cols, const int* fidx, int nf, size_t nd, double* A, cudaStream_t s) {
  k_gather_coarse<<<grid_for((size_t)nf * nf, 256), 256, 0, s>>>(cols, fidx, nf, nd, A);
  PMG_CHECK_LAUNCH();
  return ST_OK;
}

// A (n x n, symmetric positive definite, device) -> A^-1 in place.
// Returns ST_OK, ST_CUDA (msg set) or ST_NOT_SPD.
int coarse_inverse(double* A, int n, cudaStream_t s, std::string* msg) {
  cusolverDnHandle_t h = nullptr;
  if (cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS) {
    *msg = "cusolverDnCreate failed";
    return ST_CUDA;
  }
  int rc = ST_OK;
  double* work = nullptr;
  int* info = nullptr;
  int lw1 = 0, lw2 = 0, hinfo = 0;
  const cublasFillMode_t lo = CUBLAS_FILL_MODE_LOWER;
  do {
    if (cusolverDnSetStream(h, s) != CUSOLVER_STATUS_SUCCESS ||
        cusolverDnDpotrf_bufferSize(h, lo, n, A, n, &lw1) != CUSOLVER_STATUS_SUCCESS ||
        cusolverDnDpotri_bufferSize(h, lo, n, A, n, &lw2) != CUSOLVER_STATUS_SUCCESS) {
      *msg = "cuSOLVER workspace query failed";
      rc = ST_CUDA;
      break;
    }
    const int lw = lw1 > lw2 ? lw1 : lw2;
    if (cudaMalloc(&work, sizeof(double) * (size_t)(lw > 0 ? lw : 1)) != cudaSuccess ||
        cudaMalloc(&info, sizeof(int)) != cudaSuccess) {
      *msg = "cudaMalloc of the cuSOLVER workspace failed";
      rc = ST_CUDA;
      break;
    }
    if (cusolverDnDpotrf(h, lo, n, A, n, work, lw, info) != CUSOLVER_STATUS_SUCCESS) {
      *msg = "cusolverDnDpotrf failed";
      rc = ST_CUDA;
      break;
    }
    if (cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      *msg = "cudaMemcpy of the factorisation status failed";
      rc = ST_CUDA;
      break;
    }
    if (hinfo != 0) {
      *msg = "coarse matrix is not positive definite";
      rc = ST_NOT_SPD;
      break;
    }
    if (cusolverDnDpotri(h, lo, n, A, n, work, lw, info) != CUSOLVER_STATUS_SUCCESS) {
      *msg = "cusolverDnDpotri failed";
      rc = ST_CUDA;
      break;
    }
    k_mirror_lower<<<grid_for((size_t)n * n, 256), 256, 0, s>>>(A, n);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
      *msg = "coarse inverse kernels failed";
      rc = ST_CUDA;
      break;
    }
  } while (false);
  if (work) cudaFree(work);
  if (info) cudaFree(info);
  cusolverDnDestroy(h);
  return rc;
}

}  // namespace pmg
