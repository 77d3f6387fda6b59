// Mesh-level kernels: geometry tensors, level diagonals, the global operator,
// h-transfers, vector operations and the dense coarse solve.
#pragma once
#include "sf.cuh"
#include "cg_slots.h"

namespace pmg {

// ---------------------------------------------------------------------------
// Geometry (Section 2, eq. bilinear-form with Q1 cell maps): for every cell
// and every point of the (q+1)^d Gauss rule,
//   G = w kappa det(J) J^-1 J^-T   (components 00 01 02 11 12 22, or 00 01 11)
// Layout [cell][comp][(q+1)^d].  Computed in FP64; det J <= 0 at a Gauss point
// or at a vertex of the cell sets *err.
template <int DIM>
__device__ inline void q1_jacobian(const double* X, const double* xi, double J[3][3]) {
  for (int i = 0; i < DIM; ++i)
    for (int j = 0; j < DIM; ++j) J[i][j] = 0.0;
  for (int v = 0; v < (1 << DIM); ++v) {
    double dN[3];
    for (int j = 0; j < DIM; ++j) {
      double f = 1.0;
      for (int k = 0; k < DIM; ++k) {
        const int bit = (v >> k) & 1;
        if (k == j) f *= bit ? 1.0 : -1.0;
        else f *= bit ? xi[k] : 1.0 - xi[k];
      }
      dN[j] = f;
    }
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) J[i][j] += X[v * DIM + i] * dN[j];
  }
}

template <int DIM>
__device__ inline void cell_vertices(const double* coords, int N, int cell, double* X) {
  int c[3] = {0, 0, 0};
  int rem = cell;
  for (int ax = 0; ax < DIM; ++ax) { c[ax] = rem % N; rem /= N; }
  for (int v = 0; v < (1 << DIM); ++v) {
    size_t id = 0, mul = 1;
    for (int ax = 0; ax < DIM; ++ax) { id += (size_t)(c[ax] + ((v >> ax) & 1)) * mul; mul *= (N + 1); }
    for (int i = 0; i < DIM; ++i) X[v * DIM + i] = coords[id * DIM + i];
  }
}

// G = w kappa det(J) J^-1 J^-T at Gauss point g (index in the (q+1)^d rule)
// of the cell with vertices X (2^d x d, lexicographic corners), written to
// out[comp * ngc]; err gets bit 0 when det J <= 0 at the point or, for g = 0,
// at a vertex of the cell (an inverted or non-convex corner).
template <int DIM, typename T>
__device__ void geometry_point(const double* X, double kappa, int q, int g, T* out, int ngc, int* err) {
  const int n = q + 1;
  double xi[3];
  double w = 1.0;
  int rem = g;
  for (int ax = 0; ax < DIM; ++ax) {
    const int ga = rem % n;
    rem /= n;
    xi[ax] = c_rules.gx[q][ga];
    w *= c_rules.gw[q][ga];
  }
  double J[3][3];
  q1_jacobian<DIM>(X, xi, J);
  double det, Ji[3][3];
  if (DIM == 3) {
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    const double id = 1.0 / det;
    Ji[0][0] = c00 * id;
    Ji[1][0] = c01 * id;
    Ji[2][0] = c02 * id;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
  } else {
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    const double id = 1.0 / det;
    Ji[0][0] = J[1][1] * id;
    Ji[0][1] = -J[0][1] * id;
    Ji[1][0] = -J[1][0] * id;
    Ji[1][1] = J[0][0] * id;
  }
  if (!(det > 0.0)) atomicOr(err, 1);
  if (g == 0) {
    for (int v = 0; v < (1 << DIM); ++v) {
      double xv[3], Jv[3][3];
      for (int k = 0; k < DIM; ++k) xv[k] = (v >> k) & 1;
      q1_jacobian<DIM>(X, xv, Jv);
      const double dv = DIM == 3 ? Jv[0][0] * (Jv[1][1] * Jv[2][2] - Jv[1][2] * Jv[2][1]) -
                                       Jv[0][1] * (Jv[1][0] * Jv[2][2] - Jv[1][2] * Jv[2][0]) +
                                       Jv[0][2] * (Jv[1][0] * Jv[2][1] - Jv[1][1] * Jv[2][0])
                                 : Jv[0][0] * Jv[1][1] - Jv[0][1] * Jv[1][0];
      if (!(dv > 0.0)) atomicOr(err, 1);
    }
  }
  const double s = w * kappa * det;
  int comp = 0;
  for (int k = 0; k < DIM; ++k)
    for (int l = k; l < DIM; ++l) {
      double v = 0.0;
      for (int m = 0; m < DIM; ++m) v += Ji[k][m] * Ji[l][m];
      out[(size_t)comp * ngc] = T(s * v);
      ++comp;
    }
}

template <int DIM, typename T>
__global__ void k_geometry(const double* __restrict__ coords, const double* __restrict__ kappa, int N, int q,
                           T* __restrict__ G, int* err) {
  const int n = q + 1;
  const int ngc = DIM == 3 ? n * n * n : n * n;
  constexpr int NCOMP = DIM * (DIM + 1) / 2;
  const size_t ncells = DIM == 3 ? (size_t)N * N * N : (size_t)N * N;
  const size_t total = ncells * ngc;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int cell = (int)(t / ngc);
    const int g = (int)(t - (size_t)cell * ngc);
    double X[8 * 3];
    cell_vertices<DIM>(coords, N, cell, X);
    geometry_point<DIM, T>(X, kappa[cell], q, g, G + (size_t)cell * NCOMP * ngc + g, ngc, err);
  }
}

// diagonal entry of node a of a cell's degree-q operator:
// sum_g sum_kl G_kl(g) d_k phi_a(g) d_l phi_a(g), G of the cell at Gc
template <int DIM>
__device__ double cell_diag_entry(const double* __restrict__ Gc, int q, int a) {
  const int n = q + 1;
  const int ngc = DIM == 3 ? n * n * n : n * n;
  int aa[3] = {0, 0, 0}, rem = a;
  for (int ax = 0; ax < DIM; ++ax) { aa[ax] = rem % n; rem /= n; }
  double s = 0.0;
  for (int g = 0; g < ngc; ++g) {
    int gg[3] = {0, 0, 0}, r2 = g;
    for (int ax = 0; ax < DIM; ++ax) { gg[ax] = r2 % n; r2 /= n; }
    double grad[3];
    for (int k = 0; k < DIM; ++k) {
      double f = 1.0;
      for (int ax = 0; ax < DIM; ++ax)
        f *= (ax == k) ? c_rules.Bd[q][gg[ax]][aa[ax]] : c_tab_f64.B[q][gg[ax]][aa[ax]];
      grad[k] = f;
    }
    int comp = 0;
    for (int k = 0; k < DIM; ++k)
      for (int l = k; l < DIM; ++l) {
        const double gkl = Gc[(size_t)comp * ngc + g];
        s += (k == l ? 1.0 : 2.0) * gkl * grad[k] * grad[l];
        ++comp;
      }
  }
  return s;
}

// ---------------------------------------------------------------------------
// Level diagonal: diag_a += sum_g sum_kl G_kl(g) d_k phi_a(g) d_l phi_a(g) over
// the cells of one parity class (cells of one class share no node).
template <int DIM>
__global__ void k_diag(const double* __restrict__ G, int N, int q, int parity, double* __restrict__ diag) {
  const int n = q + 1;
  const int ngc = DIM == 3 ? n * n * n : n * n;
  constexpr int NCOMP = DIM * (DIM + 1) / 2;
  const int Nh = (N + 1) / 2;   // cells per direction with a given parity (upper bound)
  int nclass = 1;
  for (int ax = 0; ax < DIM; ++ax) nclass *= Nh;
  const size_t Mg = (size_t)q * N + 1;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)nclass * ngc;
       t += (size_t)gridDim.x * blockDim.x) {
    const int ci = (int)(t / ngc);
    const int a = (int)(t - (size_t)ci * ngc);
    int c[3] = {0, 0, 0}, rem = ci;
    bool ok = true;
    for (int ax = 0; ax < DIM; ++ax) {
      c[ax] = 2 * (rem % Nh) + ((parity >> ax) & 1);
      rem /= Nh;
      ok = ok && c[ax] < N;
    }
    if (!ok) continue;
    int cell = 0, mul = 1;
    for (int ax = 0; ax < DIM; ++ax) { cell += c[ax] * mul; mul *= N; }
    int aa[3] = {0, 0, 0};
    rem = a;
    for (int ax = 0; ax < DIM; ++ax) { aa[ax] = rem % n; rem /= n; }
    const double s = cell_diag_entry<DIM>(G + (size_t)cell * NCOMP * ngc, q, a);
    size_t idx = 0, m2 = 1;
    for (int ax = 0; ax < DIM; ++ax) { idx += (size_t)(q * c[ax] + aa[ax]) * m2; m2 *= Mg; }
    diag[idx] += s;
  }
}

// inverse diagonal on free nodes, 0 on Dirichlet nodes; optional cast
template <int DIM, typename T>
__global__ void k_invert_diag(const double* __restrict__ diag, int M, double* __restrict__ out64, T* __restrict__ outT) {
  size_t total = 1;
  for (int ax = 0; ax < DIM; ++ax) total *= M;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    size_t rem = t;
    bool bnd = false;
    for (int ax = 0; ax < DIM; ++ax) {
      const int k = (int)(rem % M);
      rem /= M;
      bnd = bnd || k == 0 || k == M - 1;
    }
    const double v = bnd ? 0.0 : 1.0 / diag[t];
    if (out64) out64[t] = v;
    if (outT) outT[t] = T(v);
  }
}

// ---------------------------------------------------------------------------
// Global operator on one parity class of cells: out += A_c u_c, u taken as 0
// on Dirichlet nodes, Dirichlet rows skipped.  CPB cells per CTA.
template <int DIM, int Q, typename T, int NT, int CPB>
struct CellApply {
  using Dm = Dims<DIM, 1, Q, (int)sizeof(T)>;
  static constexpr int NN = Dm::NN;
  static constexpr int PS = ((NN * 2 + Dm::SCRATCH) + 3) & ~3;
  static constexpr size_t smem = sizeof(T) * PS * CPB + sizeof(int) * CPB * 2;
};

template <int DIM, int Q, typename T, int NT, int CPB>
__global__ void __launch_bounds__(NT) k_cell_apply(const T* __restrict__ u, T* __restrict__ out, const T* __restrict__ G,
                                                   int N, int parity) {
  using CA = CellApply<DIM, Q, T, NT, CPB>;
  using Dm = typename CA::Dm;
  constexpr int NN = Dm::NN, M = Dm::M, PS = CA::PS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  int* cl = reinterpret_cast<int*>(smem_raw + sizeof(T) * PS * CPB);
  const int Nh = (N + 1) / 2;
  int nclass = 1;
  for (int ax = 0; ax < DIM; ++ax) nclass *= Nh;
  const size_t Mg = (size_t)Q * N + 1;
  if (threadIdx.x < CPB) {
    const int ci = blockIdx.x * CPB + threadIdx.x;
    int rem = ci, cell = 0, mul = 1, corner = 0;
    size_t cm = 1;
    bool ok = ci < nclass;
    for (int ax = 0; ax < DIM; ++ax) {
      const int c = 2 * (rem % Nh) + ((parity >> ax) & 1);
      rem /= Nh;
      ok = ok && c < N;
      cell += c * mul;
      mul *= N;
      corner += (int)((size_t)Q * c * cm);
      cm *= Mg;
    }
    cl[2 * threadIdx.x] = ok ? cell : -1;
    cl[2 * threadIdx.x + 1] = corner;
  }
  __syncthreads();
  auto node = [&](int cp, int i, bool& bnd) {
    size_t idx = 0, mul = 1;
    int rem = i, c = cl[2 * cp];
    bnd = false;
    for (int ax = 0; ax < DIM; ++ax) {
      const int k = rem % M;
      rem /= M;
      const int cc = c % N;
      c /= N;
      const int gk = Q * cc + k;
      bnd = bnd || gk == 0 || gk == (int)Mg - 1;
      idx += (size_t)gk * mul;
      mul *= Mg;
    }
    return idx;
  };
  coop<NT, CPB, NN>([&](int cp, int i) {
    T v = T(0);
    if (cl[2 * cp] >= 0) {
      bool bnd;
      const size_t idx = node(cp, i, bnd);
      v = bnd ? T(0) : u[idx];
    }
    sm[cp * PS + i] = v;
  });
  __syncthreads();
  auto gf = [G](int cp, int) {
    const int c = reinterpret_cast<const int*>(pmg_smem + sizeof(T) * PS * CPB)[2 * cp];
    return G + (size_t)(c < 0 ? 0 : c) * (Dm::NCOMP * Dm::NGC);
  };
  SF<DIM, 1, Q, T, NT, CPB>::template apply<false, false>(sm, PS, sm + NN, PS, sm + 2 * NN, PS, gf);
  coop<NT, CPB, NN>([&](int cp, int i) {
    if (cl[2 * cp] < 0) return;
    bool bnd;
    const size_t idx = node(cp, i, bnd);
    if (!bnd) out[idx] += sm[cp * PS + NN + i];
  });
}

// ---------------------------------------------------------------------------
// h-transfers (Section 2): prolongation = embedding through the reference
// cells, restriction = its transpose.  Both are Kronecker products of 1D
// banded matrices applied one direction at a time:
//   out[o][r][i] = sum_t W[r][t] in[o][s[r] + t][i].
template <typename T>
__global__ void k_band_sweep(const T* __restrict__ in, T* __restrict__ out, const double* __restrict__ W,
                             const int* __restrict__ start, int width, int Lin, int Lout, size_t O, size_t I,
                             int dirichlet_mask) {
  const size_t total = O * (size_t)Lout * I;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const size_t i = t % I;
    const size_t r = (t / I) % Lout;
    const size_t o = t / (I * Lout);
    T s = T(0);
    if (!(dirichlet_mask && (r == 0 || r == (size_t)Lout - 1))) {
      const int s0 = start[r];
      const T* src = in + (o * Lin) * I + i;
      for (int k = 0; k < width; ++k) {
        const int col = s0 + k;
        if (col >= 0 && col < Lin) s += T(W[r * width + k]) * src[(size_t)col * I];
      }
    }
    out[t] = s;
  }
}

// ---------------------------------------------------------------------------
// vector operations
template <typename T>
__global__ void k_fill(T* x, size_t n, T v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) x[i] = v;
}

template <typename A, typename B>
__global__ void k_cast(const A* __restrict__ x, B* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) y[i] = B(x[i]);
}

// y = x - y  (r = b - Au)
template <typename T>
__global__ void k_sub_from(const T* __restrict__ x, T* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) y[i] = x[i] - y[i];
}

template <typename T>
__global__ void k_add_to(const T* __restrict__ x, T* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) y[i] += x[i];
}

// zero the Dirichlet entries of a (M^DIM) grid vector
template <int DIM, typename T>
__global__ void k_mask_boundary(T* x, int M) {
  size_t total = 1;
  for (int ax = 0; ax < DIM; ++ax) total *= M;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    size_t rem = t;
    bool bnd = false;
    for (int ax = 0; ax < DIM; ++ax) {
      const int k = (int)(rem % M);
      rem /= M;
      bnd = bnd || k == 0 || k == M - 1;
    }
    if (bnd) x[t] = T(0);
  }
}

// Deterministic two-stage dot products: stage 1 writes one partial per block
// (fixed grid), stage 2 sums them in order and finishes the CG scalars.

__device__ inline double block_reduce_sum(double v) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  }
  __syncthreads();
  return s;
}

static __global__ void k_dot_partial(const double* __restrict__ x, const double* __restrict__ y, size_t n,
                              double* __restrict__ partial) {
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) s += x[i] * y[i];
  s = block_reduce_sum(s);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}


// sum partials into scal[slot]; op: 0 store, 1 rz (beta = rz/rz_old, rz_old = rz), 2 pAp (alpha = rz/pAp)
static __global__ void k_dot_final(const double* __restrict__ partial, int nparts, double* scal, int slot, int op) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += partial[i];
  s = block_reduce_sum(s);
  if (threadIdx.x == 0) {
    scal[slot] = s;
    if (op == 1) {
      scal[S_BETA] = s / scal[S_RZ_OLD];
      scal[S_RZ_OLD] = s;
    } else if (op == 2) {
      scal[S_ALPHA] = scal[S_RZ] / s;
    }
  }
}

// p = z + beta p
static __global__ void k_cg_update_p(const double* __restrict__ z, double* __restrict__ p, const double* scal, size_t n) {
  const double beta = scal[S_BETA];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = z[i] + beta * p[i];
}

// x += alpha p; r -= alpha Ap
static __global__ void k_cg_update_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                               const double* __restrict__ Ap, const double* scal, size_t n) {
  const double alpha = scal[S_ALPHA];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    r[i] -= alpha * Ap[i];
  }
}

// additive sweep: u += theta (W) corr on free DoFs, W = 1 / patch multiplicity
template <int DIM, typename T>
__global__ void k_additive_update(T* __restrict__ u, const T* __restrict__ corr, T theta, int weighted, int q,
                                  int N) {
  const int M = q * N + 1;
  size_t nd = 1;
  for (int ax = 0; ax < DIM; ++ax) nd *= M;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nd; i += (size_t)gridDim.x * blockDim.x) {
    size_t rem = i;
    int m = 1;
    bool bnd = false;
    for (int ax = 0; ax < DIM; ++ax) {
      const int g = (int)(rem % M);
      rem /= M;
      bnd = bnd || g == 0 || g == M - 1;
      m *= bnd ? 1 : patch_multiplicity_1d(g, q, N);
    }
    if (bnd) continue;
    u[i] += weighted ? theta * corr[i] / T(m) : theta * corr[i];
  }
}

// y += a x ; y = a x
static __global__ void k_axpy(double a, const double* __restrict__ x, double* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}
static __global__ void k_scale(double a, const double* __restrict__ x, double* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = a * x[i];
}

// ---------------------------------------------------------------------------
// Coarse solve: x_free = Ainv b_free (dense FP64 inverse of the coarsest
// matrix, computed once at set-up).  One warp per row.
template <typename T>
__global__ void k_coarse_gemv(const double* __restrict__ Ainv, const int* __restrict__ freeidx, int nf,
                              const T* __restrict__ b, T* __restrict__ x) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int row = warp; row < nf; row += nw) {
    double s = 0.0;
    const double* a = Ainv + (size_t)row * nf;
    for (int j = lane; j < nf; j += 32) s += a[j] * (double)b[freeidx[j]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[freeidx[row]] = T(s);
  }
}

// ---------------------------------------------------------------------------
// Load vector of f = d pi^2 prod_k sin(pi x_k) with the (q+2)-point Gauss
// rule, accumulated per parity class of cells.
template <int DIM>
__global__ void k_rhs_manufactured(const double* __restrict__ coords, int N, int q, int parity, double* __restrict__ b) {
  const int n = q + 1, nq = q + 2;
  const int nnode = DIM == 3 ? n * n * n : n * n;
  const int npt = DIM == 3 ? nq * nq * nq : nq * nq;
  const int Nh = (N + 1) / 2;
  int nclass = 1;
  for (int ax = 0; ax < DIM; ++ax) nclass *= Nh;
  const size_t Mg = (size_t)q * N + 1;
  const double pi = 3.14159265358979323846;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < (size_t)nclass * nnode;
       t += (size_t)gridDim.x * blockDim.x) {
    const int ci = (int)(t / nnode);
    const int a = (int)(t - (size_t)ci * nnode);
    int c[3] = {0, 0, 0}, rem = ci;
    bool ok = true;
    for (int ax = 0; ax < DIM; ++ax) {
      c[ax] = 2 * (rem % Nh) + ((parity >> ax) & 1);
      rem /= Nh;
      ok = ok && c[ax] < N;
    }
    if (!ok) continue;
    int cell = 0, mul = 1;
    for (int ax = 0; ax < DIM; ++ax) { cell += c[ax] * mul; mul *= N; }
    double X[8 * 3];
    cell_vertices<DIM>(coords, N, cell, X);
    int aa[3] = {0, 0, 0};
    rem = a;
    for (int ax = 0; ax < DIM; ++ax) { aa[ax] = rem % n; rem /= n; }
    double s = 0.0;
    for (int g = 0; g < npt; ++g) {
      int gg[3] = {0, 0, 0}, r2 = g;
      double xi[3], w = 1.0, phi = 1.0;
      for (int ax = 0; ax < DIM; ++ax) {
        gg[ax] = r2 % nq;
        r2 /= nq;
        xi[ax] = c_rules.gx2[q][gg[ax]];
        w *= c_rules.gw2[q][gg[ax]];
        phi *= c_rules.Bg[q][gg[ax]][aa[ax]];
      }
      double J[3][3];
      q1_jacobian<DIM>(X, xi, J);
      const double det = DIM == 3 ? J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                                        J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                                        J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0])
                                  : J[0][0] * J[1][1] - J[0][1] * J[1][0];
      double x[3] = {0, 0, 0};
      for (int v = 0; v < (1 << DIM); ++v) {
        double Nv = 1.0;
        for (int k = 0; k < DIM; ++k) Nv *= ((v >> k) & 1) ? xi[k] : 1.0 - xi[k];
        for (int i = 0; i < DIM; ++i) x[i] += Nv * X[v * DIM + i];
      }
      double f = DIM * pi * pi;
      for (int i = 0; i < DIM; ++i) f *= sin(pi * x[i]);
      s += w * det * f * phi;
    }
    size_t idx = 0, m2 = 1;
    bool bnd = false;
    for (int ax = 0; ax < DIM; ++ax) {
      const int gk = q * c[ax] + aa[ax];
      bnd = bnd || gk == 0 || gk == (int)Mg - 1;
      idx += (size_t)gk * m2;
      m2 *= Mg;
    }
    if (!bnd) b[idx] += s;
  }
}

// ---------------------------------------------------------------------------
// FMA-pipe peak: 8 independent FMA chains per thread (x <- x * a + b), the
// result summed and stored so that nothing is eliminated.
template <typename T>
__global__ void k_fma_chain(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * (size_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace pmg
