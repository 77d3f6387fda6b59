// Internal launchers of the learned-interval kernels (mlp.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pmg {

// features of every patch of a level at degree q (npatch x 16 floats)
int features_launch(int dim, const double* coords, const double* kappa, int N, int q, int n_below, int npatch,
                    float* X, cudaStream_t s);
// Y (n x 2) = (log theta_max, log theta_min) predicted from raw features X
int mlp_infer_launch(const float* params, const float* norm, const float* X, int64_t n, int bf16, float* Y,
                     cudaStream_t s);
// [lo, hi] = [max(theta_min, hi / ratio), safety theta_max] from predicted logs
int bounds_from_logs_launch(const float* Y, int64_t n, double safety, double ratio, float* b32, double* b64,
                            cudaStream_t s);

// T (n x 2) = (log theta_max, log theta_min) from Ritz pairs (theta_min, theta_max)
int targets_launch(const double* ritz, int64_t n, float* T, cudaStream_t s);

}  // namespace pmg
