// Learned Chebyshev intervals: per-patch features, a 16 -> 64 -> 64 -> 2 MLP
// with BF16 inference and FP32 training, all on the GPU.
//
// The paper has no learned component; its smoother is damped Jacobi.  The
// Chebyshev variant needs, for every patch j and p-level q, an interval for the
// spectrum of D^-1 A_{j,q}.  A 16-step Lanczos run per (patch, level) gives it
// (k_lanczos); the MLP predicts (log theta_max, log theta_min) of that run from
// geometric and coefficient features at a tiny fraction of the cost, and
// Lanczos remains the reference the predictions are checked against (tests)
// and the fallback.
//
// Features of patch j at degree q, from its 2^d cells, with J_c the Jacobian
// of cell c at its centre, s_c its singular values, d_c = det J_c,
// r_c = min over the cell's vertices of det J / d_c, k_c = log kappa_c,
// t_c = k_c + log d_c - 2 log(mean s_c):
//    0 q/8   1 2^d/8   2 max k - min k   3 mean |k - mean k|
//    4/5/6 max/mean/min of log(s_max/s_min)   7 log(max d / min d)
//    8/9 min/mean r   10 max t - min t   11 mean |t - mean t|
//   12 log(max s_max / min s_min)   13 (q/8)^2   14 max |log d - mean log d|
//   15 (number of p-levels below q)/4
//
// Network (standardised inputs and targets): relu(W1 x + b1) -> relu(W2 h + b2)
// -> W3 h + b3.  Parameters: W1 (64x16, row-major), b1, W2 (64x64), b2,
// W3 (2x64), b3 = 5378 floats.  Normalisation: 36 floats, mean/std of the 16
// inputs then mean/std of the 2 targets.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <type_traits>
#include <random>
#include <vector>

#include "../../include/pmg.h"
#include "device_guard.h"
#include "mlp.h"

namespace pmg {
namespace {

constexpr int NF = 16, NH = 64, NO = 2;
constexpr int OW1 = 0, OB1 = OW1 + NH * NF, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH, OB3 = OW3 + NO * NH;
constexpr int NP = OB3 + NO;
static_assert(NP == PMG_MLP_NPARAM, "parameter count");

int grid_for(size_t work, int threads) {
  size_t g = (work + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return (int)std::max<size_t>(g, 1);
}

// ---------------------------------------------------------------- features
// singular values of a dim x dim matrix from the eigenvalues of J^T J
// (2x2: closed form; 3x3 symmetric: trigonometric solution of the cubic)
template <int DIM>
__device__ void singular_values(const double J[3][3], double* s) {
  double M[3][3];
  for (int i = 0; i < DIM; ++i)
    for (int j = 0; j < DIM; ++j) {
      double v = 0.0;
      for (int k = 0; k < DIM; ++k) v += J[k][i] * J[k][j];
      M[i][j] = v;
    }
  if (DIM == 2) {
    const double tr = M[0][0] + M[1][1], det = M[0][0] * M[1][1] - M[0][1] * M[1][0];
    const double disc = sqrt(fmax(0.25 * tr * tr - det, 0.0));
    s[0] = sqrt(fmax(0.5 * tr + disc, 0.0));
    s[1] = sqrt(fmax(0.5 * tr - disc, 0.0));
  } else {
    const double p1 = M[0][1] * M[0][1] + M[0][2] * M[0][2] + M[1][2] * M[1][2];
    const double q = (M[0][0] + M[1][1] + M[2][2]) / 3.0;
    double e0, e1, e2;
    if (p1 == 0.0) {
      e0 = M[0][0];
      e1 = M[1][1];
      e2 = M[2][2];
      const double mx = fmax(e0, fmax(e1, e2)), mn = fmin(e0, fmin(e1, e2));
      e1 = e0 + e1 + e2 - mx - mn;
      e0 = mx;
      e2 = mn;
    } else {
      const double p2 = (M[0][0] - q) * (M[0][0] - q) + (M[1][1] - q) * (M[1][1] - q) +
                        (M[2][2] - q) * (M[2][2] - q) + 2.0 * p1;
      const double p = sqrt(p2 / 6.0);
      double B[3][3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) B[i][j] = (M[i][j] - (i == j ? q : 0.0)) / p;
      const double detB = B[0][0] * (B[1][1] * B[2][2] - B[1][2] * B[2][1]) -
                          B[0][1] * (B[1][0] * B[2][2] - B[1][2] * B[2][0]) +
                          B[0][2] * (B[1][0] * B[2][1] - B[1][1] * B[2][0]);
      const double r = fmin(fmax(detB / 2.0, -1.0), 1.0);
      const double phi = acos(r) / 3.0;
      const double pi = 3.14159265358979323846;
      e0 = q + 2.0 * p * cos(phi);
      e2 = q + 2.0 * p * cos(phi + 2.0 * pi / 3.0);
      e1 = 3.0 * q - e0 - e2;
    }
    s[0] = sqrt(fmax(e0, 0.0));
    s[1] = sqrt(fmax(e1, 0.0));
    s[2] = sqrt(fmax(e2, 0.0));
  }
}

template <int DIM>
__device__ void jac(const double* X, const double* xi, double J[3][3]) {
  for (int i = 0; i < DIM; ++i)
    for (int j = 0; j < DIM; ++j) J[i][j] = 0.0;
  for (int v = 0; v < (1 << DIM); ++v)
    for (int j = 0; j < DIM; ++j) {
      double f = 1.0;
      for (int k = 0; k < DIM; ++k) {
        const int bit = (v >> k) & 1;
        f *= (k == j) ? (bit ? 1.0 : -1.0) : (bit ? xi[k] : 1.0 - xi[k]);
      }
      for (int i = 0; i < DIM; ++i) J[i][j] += X[v * DIM + i] * f;
    }
}

template <int DIM>
__device__ double det3(const double J[3][3]) {
  return DIM == 3 ? J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                        J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                        J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0])
                  : J[0][0] * J[1][1] - J[0][1] * J[1][0];
}

template <int DIM>
__global__ void k_features(const double* __restrict__ coords, const double* __restrict__ kappa, int N, int q,
                           int n_below, int npatch, float* __restrict__ Xout) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= npatch) return;
  constexpr int NC = 1 << DIM;
  const int Nv = N - 1;
  int v[3] = {1, 1, 1};
  {
    int rem = j;
    for (int ax = 0; ax < DIM; ++ax) { v[ax] = 1 + rem % Nv; rem /= Nv; }
  }
  double an[NC], dd[NC], rr[NC], kk[NC], tt[NC], smax[NC], smin[NC];
  for (int c = 0; c < NC; ++c) {
    int cc[3] = {0, 0, 0};
    for (int ax = 0; ax < DIM; ++ax) cc[ax] = v[ax] - 1 + ((c >> ax) & 1);
    double X[8 * 3];
    int cell = 0, cm = 1;
    for (int ax = 0; ax < DIM; ++ax) { cell += cc[ax] * cm; cm *= N; }
    for (int w = 0; w < (1 << DIM); ++w) {
      size_t id = 0, mul = 1;
      for (int ax = 0; ax < DIM; ++ax) { id += (size_t)(cc[ax] + ((w >> ax) & 1)) * mul; mul *= (N + 1); }
      for (int i = 0; i < DIM; ++i) X[w * DIM + i] = coords[id * DIM + i];
    }
    double J[3][3], xi[3] = {0.5, 0.5, 0.5};
    jac<DIM>(X, xi, J);
    double s[3];
    singular_values<DIM>(J, s);
    const double d = det3<DIM>(J);
    double rmin = 1e300;
    for (int w = 0; w < (1 << DIM); ++w) {
      double xw[3];
      for (int k = 0; k < DIM; ++k) xw[k] = (w >> k) & 1;
      double Jw[3][3];
      jac<DIM>(X, xw, Jw);
      rmin = fmin(rmin, det3<DIM>(Jw) / d);
    }
    double smean = 0.0;
    for (int k = 0; k < DIM; ++k) smean += s[k];
    smean /= DIM;
    smax[c] = s[0];
    smin[c] = s[DIM - 1];
    an[c] = log(s[0] / s[DIM - 1]);
    dd[c] = d;
    rr[c] = rmin;
    kk[c] = log(kappa[cell]);
    tt[c] = kk[c] + log(d) - 2.0 * log(smean);
  }
  auto mx = [&](const double* a) { double r = a[0]; for (int c = 1; c < NC; ++c) r = fmax(r, a[c]); return r; };
  auto mn = [&](const double* a) { double r = a[0]; for (int c = 1; c < NC; ++c) r = fmin(r, a[c]); return r; };
  auto mean = [&](const double* a) { double r = 0.0; for (int c = 0; c < NC; ++c) r += a[c]; return r / NC; };
  auto mad = [&](const double* a) {
    const double m = mean(a);
    double r = 0.0;
    for (int c = 0; c < NC; ++c) r += fabs(a[c] - m);
    return r / NC;
  };
  double ld[NC];
  for (int c = 0; c < NC; ++c) ld[c] = log(dd[c]);
  double ldm = mean(ld), ldmax = 0.0;
  for (int c = 0; c < NC; ++c) ldmax = fmax(ldmax, fabs(ld[c] - ldm));
  float* o = Xout + (size_t)j * NF;
  o[0] = (float)(q / 8.0);
  o[1] = (float)(NC / 8.0);
  o[2] = (float)(mx(kk) - mn(kk));
  o[3] = (float)mad(kk);
  o[4] = (float)mx(an);
  o[5] = (float)mean(an);
  o[6] = (float)mn(an);
  o[7] = (float)log(mx(dd) / mn(dd));
  o[8] = (float)mn(rr);
  o[9] = (float)mean(rr);
  o[10] = (float)(mx(tt) - mn(tt));
  o[11] = (float)mad(tt);
  o[12] = (float)log(mx(smax) / mn(smin));
  o[13] = (float)((q / 8.0) * (q / 8.0));
  o[14] = (float)ldmax;
  o[15] = (float)(n_below / 4.0);
}

// ------------------------------------------------------------ inference
// FP32 inference: one thread per sample, parameters in shared memory
__global__ void k_mlp_infer(const float* __restrict__ params, const float* __restrict__ norm,
                            const float* __restrict__ X, int64_t n, float* __restrict__ Y) {
  using W = float;
  __shared__ W w[NP];
  __shared__ float nm[36];
  for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = (W)params[i];
  for (int i = threadIdx.x; i < 36; i += blockDim.x) nm[i] = norm[i];
  __syncthreads();
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    float x[NF];
    for (int i = 0; i < NF; ++i) {
      x[i] = (X[s * NF + i] - nm[i]) / nm[NF + i];
    }
    float h1[NH];
    for (int r = 0; r < NH; ++r) {
      float a = (float)w[OB1 + r];
      for (int i = 0; i < NF; ++i) a += (float)w[OW1 + r * NF + i] * x[i];
      h1[r] = fmaxf(a, 0.f);
    }
    float y0 = (float)w[OB3], y1 = (float)w[OB3 + 1];
    for (int r = 0; r < NH; ++r) {
      float a = (float)w[OB2 + r];
      for (int i = 0; i < NH; ++i) a += (float)w[OW2 + r * NH + i] * h1[i];
      a = fmaxf(a, 0.f);
      y0 += (float)w[OW3 + r] * a;
      y1 += (float)w[OW3 + NH + r] * a;
    }
    // back to (log theta_max, log theta_min)
    Y[s * NO] = y0 * nm[2 * NF + 2] + nm[2 * NF];
    Y[s * NO + 1] = y1 * nm[2 * NF + 3] + nm[2 * NF + 1];
  }
}

// BF16 inference on the tensor cores: one warp per tile of 16 samples, the
// three layers as mma.sync m16n8k16 products with BF16 operands and FP32
// accumulation (16x16 inputs x 16x64 W1^T, 16x64 x 64x64 W2^T, 16x64 x 64x8
// W3^T with W3 padded to 8 rows).  Weights, biases, inputs and the two hidden
// activations are BF16 values; sums are FP32.  Fragment layouts (PTX ISA,
// m16n8k16 with .bf16): lane = 4 g + t; A holds rows g and g + 8, columns
// 2t, 2t+1, 2t+8, 2t+9 of the 16x16 tile; B holds rows (k) 2t, 2t+1, 2t+8,
// 2t+9 of column (n) g; C/D holds rows g, g + 8 and columns 2t, 2t+1.  The
// C tiles 2k and 2k+1 of one layer are exactly the A tile k of the next, so
// activations never leave the registers.
constexpr int MW1 = NF / 2 + 4;     // words per W1 row in shared memory (padded: conflict-free B loads)
constexpr int MW2 = NH / 2 + 4;     // words per W2 / W3 row
constexpr int MMA_THREADS = 128;

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);    // lo in the low half
  unsigned u;
  memcpy(&u, &v, 4);
  return u;
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// C tiles (n-tiles 0..7 of a 16x64 layer output) + bias, ReLU, rounded to BF16
// -> the four A tiles of the next layer
__device__ __forceinline__ void act_to_a(float (&c)[8][4], const float* bias, int t, unsigned (&a)[4][4]) {
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float b0 = bias[nt * 8 + 2 * t], b1 = bias[nt * 8 + 2 * t + 1];
    c[nt][0] = fmaxf(c[nt][0] + b0, 0.f);
    c[nt][1] = fmaxf(c[nt][1] + b1, 0.f);
    c[nt][2] = fmaxf(c[nt][2] + b0, 0.f);
    c[nt][3] = fmaxf(c[nt][3] + b1, 0.f);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    a[k][0] = pack_bf16(c[2 * k][0], c[2 * k][1]);
    a[k][1] = pack_bf16(c[2 * k][2], c[2 * k][3]);
    a[k][2] = pack_bf16(c[2 * k + 1][0], c[2 * k + 1][1]);
    a[k][3] = pack_bf16(c[2 * k + 1][2], c[2 * k + 1][3]);
  }
}

__global__ void __launch_bounds__(MMA_THREADS) k_mlp_infer_mma(const float* __restrict__ params,
                                                               const float* __restrict__ norm,
                                                               const float* __restrict__ X, int64_t n,
                                                               float* __restrict__ Y) {
  __shared__ unsigned w1[NH * MW1], w2[NH * MW2], w3[8 * MW2];
  __shared__ float bs[2 * NH + NO], nm[36];
  for (int i = threadIdx.x; i < NH * NF / 2; i += blockDim.x) {
    const int r = i / (NF / 2), c = i - r * (NF / 2);
    w1[r * MW1 + c] = pack_bf16(params[OW1 + 2 * i], params[OW1 + 2 * i + 1]);
  }
  for (int i = threadIdx.x; i < NH * NH / 2; i += blockDim.x) {
    const int r = i / (NH / 2), c = i - r * (NH / 2);
    w2[r * MW2 + c] = pack_bf16(params[OW2 + 2 * i], params[OW2 + 2 * i + 1]);
  }
  for (int i = threadIdx.x; i < 8 * NH / 2; i += blockDim.x) {
    const int r = i / (NH / 2), c = i - r * (NH / 2);
    w3[r * MW2 + c] = r < NO ? pack_bf16(params[OW3 + 2 * i], params[OW3 + 2 * i + 1]) : 0u;
  }
  // biases as BF16 values (the weights' precision), kept in FP32 registers
  for (int i = threadIdx.x; i < NH; i += blockDim.x) {
    bs[i] = __bfloat162float(__float2bfloat16_rn(params[OB1 + i]));
    bs[NH + i] = __bfloat162float(__float2bfloat16_rn(params[OB2 + i]));
  }
  if (threadIdx.x < NO) bs[2 * NH + threadIdx.x] = __bfloat162float(__float2bfloat16_rn(params[OB3 + threadIdx.x]));
  for (int i = threadIdx.x; i < 36; i += blockDim.x) nm[i] = norm[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int64_t ntile = (n + 15) / 16;
  const int64_t warps = (int64_t)gridDim.x * (MMA_THREADS / 32);
  for (int64_t tile = blockIdx.x * (int64_t)(MMA_THREADS / 32) + (threadIdx.x >> 5); tile < ntile; tile += warps) {
    const int64_t s0 = tile * 16 + g, s1 = s0 + 8;      // the two samples (rows) of this thread
    // layer-1 A tile: standardised inputs, rounded to BF16
    auto xin = [&](int64_t s, int c) { return s < n ? (X[s * NF + c] - nm[c]) / nm[NF + c] : 0.f; };
    unsigned a[4];
    a[0] = pack_bf16(xin(s0, 2 * t), xin(s0, 2 * t + 1));
    a[1] = pack_bf16(xin(s1, 2 * t), xin(s1, 2 * t + 1));
    a[2] = pack_bf16(xin(s0, 2 * t + 8), xin(s0, 2 * t + 9));
    a[3] = pack_bf16(xin(s1, 2 * t + 8), xin(s1, 2 * t + 9));
    float c[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.f;
      const unsigned* wr = w1 + (nt * 8 + g) * MW1;
      mma_bf16(c[nt], a, wr[t], wr[t + 4]);
    }
    unsigned h[4][4];
    act_to_a(c, bs, t, h);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      c[nt][0] = c[nt][1] = c[nt][2] = c[nt][3] = 0.f;
      const unsigned* wr = w2 + (nt * 8 + g) * MW2;
#pragma unroll
      for (int k = 0; k < 4; ++k) mma_bf16(c[nt], h[k], wr[k * 8 + t], wr[k * 8 + t + 4]);
    }
    act_to_a(c, bs + NH, t, h);
    float y[4] = {0.f, 0.f, 0.f, 0.f};
    const unsigned* wr = w3 + g * MW2;
#pragma unroll
    for (int k = 0; k < 4; ++k) mma_bf16(y, h[k], wr[k * 8 + t], wr[k * 8 + t + 4]);
    // columns 0 and 1 of the output tile sit in lanes with t = 0
    if (t == 0) {
      const float b0 = bs[2 * NH], b1 = bs[2 * NH + 1];
      if (s0 < n) {
        Y[s0 * NO] = (y[0] + b0) * nm[2 * NF + 2] + nm[2 * NF];
        Y[s0 * NO + 1] = (y[1] + b1) * nm[2 * NF + 3] + nm[2 * NF + 1];
      }
      if (s1 < n) {
        Y[s1 * NO] = (y[2] + b0) * nm[2 * NF + 2] + nm[2 * NF];
        Y[s1 * NO + 1] = (y[3] + b1) * nm[2 * NF + 3] + nm[2 * NF + 1];
      }
    }
  }
}

// predicted logs -> Chebyshev interval [lo, hi]
template <typename T>
__global__ void k_bounds_from_logs(const float* __restrict__ Y, int64_t n, double safety, double ratio,
                                   T* __restrict__ bounds, double* __restrict__ bounds64) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
    const double tmax = exp((double)Y[s * 2]), tmin = exp((double)Y[s * 2 + 1]);
    const double hi = safety * tmax;
    const double lo = fmax(tmin, hi / ratio);
    bounds[2 * s] = T(lo);
    bounds[2 * s + 1] = T(hi);
    bounds64[2 * s] = lo;
    bounds64[2 * s + 1] = hi;
  }
}

// ------------------------------------------------------------- training
// C (M x N) = sum_k A(m,k) B(k,n) [+ C if accumulate], A(m,k) = TA ? A[k*lda+m] : A[m*lda+k],
// B(k,n) = TB ? B[n*ldb+k] : B[k*ldb+n]; one thread per output, fixed order.
__global__ void k_gemm(int M, int N, int K, const float* A, int lda, int TA, const float* B, int ldb, int TB,
                       float* C, int ldc, int accumulate) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * N) return;
  const int m = idx / N, nn = idx - m * N;
  float s = 0.f;
  for (int k = 0; k < K; ++k) {
    const float a = TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
    const float b = TB ? B[(size_t)nn * ldb + k] : B[(size_t)k * ldb + nn];
    s += a * b;
  }
  C[(size_t)m * ldc + nn] = accumulate ? C[(size_t)m * ldc + nn] + s : s;
}

// gather a standardised batch: Xb[i] = (X[perm[i]] - mu) / sd, Tb likewise
__global__ void k_gather_batch(const float* X, const float* T, const int* perm, int b, const float* norm, float* Xb,
                               float* Tb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b) return;
  const int s = perm[i];
  for (int f = 0; f < NF; ++f) Xb[i * NF + f] = (X[(size_t)s * NF + f] - norm[f]) / norm[NF + f];
  for (int o = 0; o < NO; ++o) Tb[i * NO + o] = (T[(size_t)s * NO + o] - norm[2 * NF + o]) / norm[2 * NF + 2 + o];
}

// Z += bias (row broadcast), H = relu(Z)
__global__ void k_bias_relu(float* Z, const float* b, int rows, int cols, float* H) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const float z = Z[i] + b[i % cols];
  Z[i] = z;
  if (H) H[i] = fmaxf(z, 0.f);
}

// output layer: Y += b3; GY = w (Y - T) / rows; per-sample loss
__global__ void k_out_grad(float* Y, const float* b3, const float* T, int rows, float asym, float* GY, float* lossv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  float l = 0.f;
  for (int o = 0; o < NO; ++o) {
    const float y = Y[i * NO + o] + b3[o];
    Y[i * NO + o] = y;
    const float d = y - T[i * NO + o];
    const float w = (o == 0 && y < T[i * NO + o]) ? asym : 1.f;
    GY[i * NO + o] = w * d / rows;
    l += 0.5f * w * d * d;
  }
  lossv[i] = l / rows;
}

// G *= (Z > 0)
__global__ void k_relu_back(float* G, const float* Z, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !(Z[i] > 0.f)) G[i] = 0.f;
}

// column sums (bias gradients), fixed order
__global__ void k_colsum(const float* G, int rows, int cols, float* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += G[(size_t)r * cols + c];
  out[c] = s;
}

__global__ void k_sum(const float* v, int n, float* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += v[i];
    *out = s;
  }
}

__global__ void k_adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

struct Work {
  float *Xb, *Tb, *Z1, *H1, *Z2, *H2, *Y, *GY, *G2, *G1, *lossv, *loss;
};

void gemm(int M, int N, int K, const float* A, int lda, int TA, const float* B, int ldb, int TB, float* C, int ldc,
          int acc, cudaStream_t s) {
  k_gemm<<<(M * N + 255) / 256, 256, 0, s>>>(M, N, K, A, lda, TA, B, ldb, TB, C, ldc, acc);
}

// loss and gradient of a standardised batch (Xb, Tb in w) into grad
void fwd_bwd(const float* P, const Work& w, int b, float asym, float* grad, cudaStream_t s) {
  // forward
  gemm(b, NH, NF, w.Xb, NF, 0, P + OW1, NF, 1, w.Z1, NH, 0, s);          // Z1 = X W1^T
  k_bias_relu<<<(b * NH + 255) / 256, 256, 0, s>>>(w.Z1, P + OB1, b, NH, w.H1);
  gemm(b, NH, NH, w.H1, NH, 0, P + OW2, NH, 1, w.Z2, NH, 0, s);          // Z2 = H1 W2^T
  k_bias_relu<<<(b * NH + 255) / 256, 256, 0, s>>>(w.Z2, P + OB2, b, NH, w.H2);
  gemm(b, NO, NH, w.H2, NH, 0, P + OW3, NH, 1, w.Y, NO, 0, s);           // Y = H2 W3^T
  k_out_grad<<<(b + 255) / 256, 256, 0, s>>>(w.Y, P + OB3, w.Tb, b, asym, w.GY, w.lossv);
  k_sum<<<1, 32, 0, s>>>(w.lossv, b, w.loss);
  // backward
  gemm(NO, NH, b, w.GY, NO, 1, w.H2, NH, 0, grad + OW3, NH, 0, s);       // gW3 = GY^T H2
  k_colsum<<<1, 64, 0, s>>>(w.GY, b, NO, grad + OB3);
  gemm(b, NH, NO, w.GY, NO, 0, P + OW3, NH, 0, w.G2, NH, 0, s);          // GH2 = GY W3
  k_relu_back<<<(b * NH + 255) / 256, 256, 0, s>>>(w.G2, w.Z2, b * NH);
  gemm(NH, NH, b, w.G2, NH, 1, w.H1, NH, 0, grad + OW2, NH, 0, s);       // gW2 = GZ2^T H1
  k_colsum<<<1, 64, 0, s>>>(w.G2, b, NH, grad + OB2);
  gemm(b, NH, NH, w.G2, NH, 0, P + OW2, NH, 0, w.G1, NH, 0, s);          // GH1 = GZ2 W2
  k_relu_back<<<(b * NH + 255) / 256, 256, 0, s>>>(w.G1, w.Z1, b * NH);
  gemm(NH, NF, b, w.G1, NH, 1, w.Xb, NF, 0, grad + OW1, NF, 0, s);       // gW1 = GZ1^T X
  k_colsum<<<1, 64, 0, s>>>(w.G1, b, NH, grad + OB1);
}

int alloc_work(Work& w, int b) {
  float* base = nullptr;
  const size_t n = (size_t)b * (NF + NO + 4 * NH + 2 * NO + 2 * NH + 1) + 1;
  if (cudaMalloc(&base, n * sizeof(float)) != cudaSuccess) return PMG_ERR_CUDA;
  float* p = base;
  w.Xb = p; p += (size_t)b * NF;
  w.Tb = p; p += (size_t)b * NO;
  w.Z1 = p; p += (size_t)b * NH;
  w.H1 = p; p += (size_t)b * NH;
  w.Z2 = p; p += (size_t)b * NH;
  w.H2 = p; p += (size_t)b * NH;
  w.Y = p; p += (size_t)b * NO;
  w.GY = p; p += (size_t)b * NO;
  w.G2 = p; p += (size_t)b * NH;
  w.G1 = p; p += (size_t)b * NH;
  w.lossv = p; p += b;
  w.loss = p;
  return PMG_OK;
}

}  // namespace

// -------------------------------------------------------------- host API
int features_launch(int dim, const double* coords, const double* kappa, int N, int q, int n_below, int npatch,
                    float* X, cudaStream_t s) {
  if (npatch <= 0) return PMG_OK;
  if (dim == 2) k_features<2><<<grid_for(npatch, 128), 128, 0, s>>>(coords, kappa, N, q, n_below, npatch, X);
  else k_features<3><<<grid_for(npatch, 128), 128, 0, s>>>(coords, kappa, N, q, n_below, npatch, X);
  return cudaPeekAtLastError() == cudaSuccess ? PMG_OK : PMG_ERR_CUDA;
}

int mlp_infer_launch(const float* params, const float* norm, const float* X, int64_t n, int bf16, float* Y,
                     cudaStream_t s) {
  if (n <= 0) return PMG_OK;
  if (bf16) {
    const size_t tiles = ((size_t)n + 15) / 16;
    k_mlp_infer_mma<<<grid_for(tiles, MMA_THREADS / 32), MMA_THREADS, 0, s>>>(params, norm, X, n, Y);
  } else {
    k_mlp_infer<<<grid_for((size_t)n, 128), 128, 0, s>>>(params, norm, X, n, Y);
  }
  return cudaPeekAtLastError() == cudaSuccess ? PMG_OK : PMG_ERR_CUDA;
}

int bounds_from_logs_launch(const float* Y, int64_t n, double safety, double ratio, float* b32, double* b64,
                            cudaStream_t s) {
  if (n <= 0) return PMG_OK;
  k_bounds_from_logs<float><<<grid_for((size_t)n, 256), 256, 0, s>>>(Y, n, safety, ratio, b32, b64);
  return cudaPeekAtLastError() == cudaSuccess ? PMG_OK : PMG_ERR_CUDA;
}

// ---- training targets and normalisation ------------------------------------
// T[i] = (log theta_max, log theta_min) of patch i from its Ritz pair
// (theta_min, theta_max)
__global__ void k_log_targets(const double* __restrict__ ritz, int64_t n, float* __restrict__ T) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    T[2 * i] = (float)log(ritz[2 * i + 1]);
    T[2 * i + 1] = (float)log(ritz[2 * i]);
  }
}

// column c of an n x cols row-major matrix: out[c] = mean, out[cols + c] =
// population standard deviation + 1e-6 (two passes in FP64, one block per
// column, fixed reduction order: deterministic)
__global__ void __launch_bounds__(256) k_col_stats(const float* __restrict__ A, int64_t n, int cols,
                                                   float* __restrict__ out) {
  __shared__ double red[256];
  const int c = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 256) s += (double)A[i * cols + c];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double mean = red[0] / (double)n;
  __syncthreads();
  double v = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 256) {
    const double d = (double)A[i * cols + c] - mean;
    v += d * d;
  }
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[c] = (float)mean;
    out[cols + c] = (float)(sqrt(red[0] / (double)n) + 1e-6);
  }
}

int targets_launch(const double* ritz, int64_t n, float* T, cudaStream_t s) {
  if (n <= 0) return PMG_OK;
  k_log_targets<<<grid_for((size_t)n, 256), 256, 0, s>>>(ritz, n, T);
  return cudaPeekAtLastError() == cudaSuccess ? PMG_OK : PMG_ERR_CUDA;
}

}  // namespace pmg

using namespace pmg;

extern "C" {

void pmg_mlp_init(uint64_t seed, float* params) {
  if (!params) return;
  // SplitMix64 counter stream (Steele, Lea and Flood 2014): u_i in [0, 1)
  auto u01 = [seed](uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * 0x1.0p-53;
  };
  const int rows[3] = {NH, NH, NO}, cols[3] = {NF, NH, NH}, woff[3] = {OW1, OW2, OW3}, boff[3] = {OB1, OB2, OB3};
  uint64_t ctr = 0;
  for (int l = 0; l < 3; ++l) {
    const double lim = std::sqrt(6.0 / cols[l]);
    for (int i = 0; i < rows[l] * cols[l]; ++i) params[woff[l] + i] = (float)((2.0 * u01(ctr++) - 1.0) * lim);
    for (int i = 0; i < rows[l]; ++i) params[boff[l] + i] = 0.f;
  }
}

int pmg_mlp_norm(int device, const float* X, const float* T, int64_t n, float* norm_host) {
  if (!X || !T || !norm_host || n <= 0) return PMG_ERR_ARG;
  pmg::DeviceGuard guard(device);
  if (guard.err != cudaSuccess) return PMG_ERR_CUDA;
  float* out = nullptr;
  if (cudaMalloc(&out, PMG_MLP_NNORM * sizeof(float)) != cudaSuccess) return PMG_ERR_CUDA;
  k_col_stats<<<NF, 256>>>(X, n, NF, out);
  k_col_stats<<<NO, 256>>>(T, n, NO, out + 2 * NF);
  cudaError_t e = cudaMemcpy(norm_host, out, PMG_MLP_NNORM * sizeof(float), cudaMemcpyDeviceToHost);
  cudaFree(out);
  return e == cudaSuccess ? PMG_OK : PMG_ERR_CUDA;
}

void pmg_default_train_options(pmg_train_opts* o) {
  if (!o) return;
  o->epochs = 200;
  o->batch = 1024;
  o->lr = 2e-3f;
  o->beta1 = 0.9f;
  o->beta2 = 0.999f;
  o->eps = 1e-8f;
  o->asym = 4.0f;
  o->seed = 0;
}

int pmg_mlp_grad(int device, const float* params, const float* norm, const float* X, const float* T, int n,
                 float asym, float* loss, float* grad, void* stream) {
  if (!params || !norm || !X || !T || !grad || n <= 0) return PMG_ERR_ARG;
  pmg::DeviceGuard guard(device);
  if (guard.err != cudaSuccess) return PMG_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  Work w;
  if (alloc_work(w, n) != PMG_OK) return PMG_ERR_CUDA;
  int* perm = nullptr;
  if (cudaMalloc(&perm, n * sizeof(int)) != cudaSuccess) return PMG_ERR_CUDA;
  std::vector<int> id(n);
  std::iota(id.begin(), id.end(), 0);
  cudaMemcpyAsync(perm, id.data(), n * sizeof(int), cudaMemcpyHostToDevice, s);
  k_gather_batch<<<(n + 127) / 128, 128, 0, s>>>(X, T, perm, n, norm, w.Xb, w.Tb);
  fwd_bwd(params, w, n, asym, grad, s);
  if (loss) cudaMemcpyAsync(loss, w.loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
  const cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(perm);
  cudaFree(w.Xb);
  return e == cudaSuccess ? PMG_OK : PMG_ERR_CUDA;
}

int pmg_mlp_train(int device, float* params, const float* norm, const float* X, const float* T, int64_t n,
                  const pmg_train_opts* opt_in, float* loss_hist) {
  pmg_train_opts o;
  if (opt_in) o = *opt_in;
  else pmg_default_train_options(&o);
  if (!params || !norm || !X || !T || n <= 0 || o.batch <= 0 || o.epochs < 0) return PMG_ERR_ARG;
  pmg::DeviceGuard guard(device);
  if (guard.err != cudaSuccess) return PMG_ERR_CUDA;
  cudaStream_t s = nullptr;
  const int b = (int)std::min<int64_t>(o.batch, n);
  Work w;
  if (alloc_work(w, b) != PMG_OK) return PMG_ERR_CUDA;
  float *grad = nullptr, *m = nullptr, *v = nullptr;
  int* perm = nullptr;
  if (cudaMalloc(&grad, 3 * NP * sizeof(float)) != cudaSuccess) return PMG_ERR_CUDA;
  m = grad + NP;
  v = grad + 2 * NP;
  cudaMemset(m, 0, 2 * NP * sizeof(float));
  if (cudaMalloc(&perm, n * sizeof(int)) != cudaSuccess) return PMG_ERR_CUDA;
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::mt19937_64 rng(o.seed);
  int64_t step = 0;
  const int64_t nb = n / b;
  std::vector<float> eloss(std::max<int64_t>(nb, 1));
  for (int ep = 0; ep < o.epochs; ++ep) {
    std::shuffle(order.begin(), order.end(), rng);
    cudaMemcpyAsync(perm, order.data(), n * sizeof(int), cudaMemcpyHostToDevice, s);
    double tot = 0.0;
    for (int64_t bi = 0; bi < nb; ++bi) {
      k_gather_batch<<<(b + 127) / 128, 128, 0, s>>>(X, T, perm + bi * b, b, norm, w.Xb, w.Tb);
      fwd_bwd(params, w, b, o.asym, grad, s);
      ++step;
      const float c1 = 1.f - std::pow(o.beta1, (float)step), c2 = 1.f - std::pow(o.beta2, (float)step);
      k_adam<<<(NP + 255) / 256, 256, 0, s>>>(params, grad, m, v, NP, o.lr, o.beta1, o.beta2, o.eps, c1, c2);
      if (loss_hist) {
        float l = 0.f;
        cudaMemcpyAsync(&l, w.loss, sizeof(float), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        tot += l;
      }
    }
    if (loss_hist) loss_hist[ep] = (float)(tot / std::max<int64_t>(nb, 1));
  }
  const cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(perm);
  cudaFree(grad);
  cudaFree(w.Xb);
  return e == cudaSuccess ? PMG_OK : PMG_ERR_CUDA;
}

int pmg_mlp_predict(int device, const float* params, const float* norm, const float* X, int64_t n, int bf16,
                    float* Y, void* stream) {
  if (!params || !norm || !X || !Y || n < 0) return PMG_ERR_ARG;
  pmg::DeviceGuard guard(device);
  if (guard.err != cudaSuccess) return PMG_ERR_CUDA;
  return mlp_infer_launch(params, norm, X, n, bf16, Y, (cudaStream_t)stream);
}

}  // extern "C"
