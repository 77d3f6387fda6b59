// Device side of the unstructured-mesh path (host side: umesh.cu).
//
// Unstructured quadrilateral / hexahedral meshes: the vertex-patch smoother
// with the local p-multigrid solver (Sections 2.1 and 3, Algorithms 1 and 2)
// on patches of any valence, the global operator, and a two-level
// preconditioner for CG.
//
// Patch kernel (k_upatch): one CTA per patch (grid-stride over the patches
// of a launch).  A patch is a list of cells (its valence); every level vector
// of its local V-cycle lives in a workspace slice of global memory owned by the
// CTA (L1/L2 resident), indexed by the patch's interior DoFs (sorted global
// ids).  The operator is applied cell by cell, CPB cells at a time, with the
// sum-factorised single-cell apply of sf.cuh in shared memory: the cell's
// nodal values are gathered through a per-cell map (interior index or -1 for
// the patch boundary's zero Dirichlet values), the cell outputs are stored,
// and every interior DoF sums the outputs of its cells in a fixed order (the
// assembly list: (cell slot, local node) pairs by slot), so results are
// deterministic.  p-transfers act per cell (Section 3.1): the prolongation is
// the tensor-product embedding, each fine DoF taking its value from the first
// of its cells; the restriction is its transpose, the fine residual weighted
// by 1 / (number of patch cells containing the DoF) before the per-cell
// transposed embedding and the coarse assembly, which reproduces P^T exactly
// (a coarse basis function is non-zero at a fine node only if every cell
// containing the node contains its support node).
//
// Global operator: per cell apply into a cell-output array, then per DoF the
// fixed-order sum over its cells (Dirichlet DoFs zero).  Two-level
// preconditioner: forward patch sweep, residual, restriction to the Q1 space
// of the same mesh (per-cell transposed vertex functions with the same 1/mult
// weights, per-vertex fixed-order sums), dense Q1 Cholesky inverse (operator
// re-evaluated with the 2-point Gauss rule, the reading of Section 3.1 "Level
// operators" at the global coarse level), prolongation, reverse sweep.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/pmg.h"
#include "kernels_impl.cuh"
#include "umesh.h"
#include "utopo.h"

namespace pmg {

constexpr int UMAXC = PMG_UMAXC;      // cells per patch the kernels accept
// threads per CTA of the patch kernel at degree p.  One CTA works on one
// patch at a time, so the threads are the patch's parallelism: measured on a
// batch of eight problems of degrees 2-8, 128 threads everywhere took 2.60 s,
// 256 everywhere 1.65 s, 512 from degree 6 on (256 below) 1.27 s, 384 there
// 1.36 s; giving the workspace slice to shared memory at one CTA per SM was
// slower (1.85 s) than keeping it in L1/L2 at several.
__host__ __device__ constexpr int unt(int p) { return p >= 6 ? 512 : 256; }
constexpr int UMAXL = 4;              // p-levels (p <= 8: p, p/2, p/4, 1)

__host__ __device__ constexpr int ucpb(int q) { return q <= 4 ? 4 : 2; }   // cells per pass (global operator)

// cells per pass of the patch kernel (nt threads) on a level of degree q:
// about one work item per thread in the line stages (n^(d-1) lines per cell
// and direction, n = q + 1), at most 16, and the cell buffers within 96 KB
template <int DIM, typename T>
__host__ __device__ constexpr int ucpb_patch(int q, int nt) {
  const int n = q + 1;
  const int lines = DIM == 3 ? n * n : n;
  const int per_cell = (int)sizeof(T) * (2 * lines * n + sf_scratch(DIM, 1, q, false, (int)sizeof(T)));
  const int by_threads = nt / lines < 1 ? 1 : (nt / lines > 16 ? 16 : nt / lines);
  const int by_smem = (96 * 1024) / per_cell < 1 ? 1 : (96 * 1024) / per_cell;
  return by_threads < by_smem ? by_threads : by_smem;
}

__device__ __forceinline__ double gl_node(int q, int i) { return c_rules.gll[q][i]; }

// ---------------------------------------------------------------- set-up kernels
template <int DIM, typename T>
__global__ void k_ugeometry(const double* __restrict__ coords, const int64_t* __restrict__ cells,
                            const double* __restrict__ kappa, int64_t nc, int q, T* __restrict__ G, int* err) {
  const int n = q + 1;
  const int ngc = DIM == 3 ? n * n * n : n * n;
  constexpr int NCOMP = DIM * (DIM + 1) / 2;
  const size_t total = (size_t)nc * ngc;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int64_t c = (int64_t)(t / ngc);
    const int g = (int)(t - (size_t)c * ngc);
    double X[8 * 3];
    for (int v = 0; v < (1 << DIM); ++v)
      for (int k = 0; k < DIM; ++k) X[v * DIM + k] = coords[cells[c * (1 << DIM) + v] * DIM + k];
    geometry_point<DIM, T>(X, kappa[c], q, g, G + (size_t)c * NCOMP * ngc + g, ngc, err);
  }
}

template <int DIM>
__global__ void k_ucell_diag(const double* __restrict__ G, int64_t nc, int q, double* __restrict__ Y) {
  const int n = q + 1;
  const int nloc = DIM == 3 ? n * n * n : n * n;
  constexpr int NCOMP = DIM * (DIM + 1) / 2;
  const size_t total = (size_t)nc * nloc;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int64_t c = (int64_t)(t / nloc);
    const int a = (int)(t - (size_t)c * nloc);
    Y[t] = cell_diag_entry<DIM>(G + (size_t)c * NCOMP * nloc, q, a);
  }
}

// out[g] = sum over the DoF's (cell, node) entries of Y, in their stored order;
// 0 on Dirichlet DoFs
template <typename T>
__global__ void k_uassemble(const T* __restrict__ Y, const int32_t* __restrict__ start, const int32_t* __restrict__ list,
                            const uint8_t* __restrict__ bnd, int64_t n, T* __restrict__ out) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    T s = T(0);
    if (!bnd[g])
      for (int e = start[g]; e < start[g + 1]; ++e) s += Y[list[e]];
    out[g] = s;
  }
}

template <typename T>
__global__ void k_uinvert(const double* __restrict__ diag, const uint8_t* __restrict__ bnd, int64_t n,
                          double* __restrict__ d64, T* __restrict__ dT) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const double v = bnd[g] ? 0.0 : 1.0 / diag[g];
    d64[g] = v;
    if (dT) dT[g] = T(v);
  }
}

template <typename T>
__global__ void k_umask(T* x, const uint8_t* __restrict__ bnd, int64_t n) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    if (bnd[g]) x[g] = T(0);
}

// ------------------------------------------------------------ global operator
// cell outputs Y[c][l] = (A_c u_c)_l, u gathered with its Dirichlet values zeroed
template <int DIM, int Q, typename T, int CPB>
__global__ void __launch_bounds__(128) k_ucell_apply(const T* __restrict__ u, const T* __restrict__ G,
                                                     const int32_t* __restrict__ cdofs,
                                                     const uint8_t* __restrict__ bnd, int64_t nc, T* __restrict__ Y) {
  constexpr int NT = 128;
  using S = SF<DIM, 1, Q, T, NT, CPB>;
  using Dm = typename S::D;
  constexpr int NL = Dm::NN, PS = 2 * NL + Dm::SCRATCH;
  T* sm = reinterpret_cast<T*>(pmg_smem);
  const int64_t c0 = (int64_t)blockIdx.x * CPB;
  for (int t = threadIdx.x; t < CPB * NL; t += NT) {
    const int cp = t / NL, l = t - cp * NL;
    const int64_t c = c0 + cp;
    T v = T(0);
    if (c < nc) {
      const int32_t g = cdofs[c * NL + l];
      v = bnd[g] ? T(0) : u[g];
    }
    sm[cp * PS + l] = v;
  }
  __syncthreads();
  struct GF {
    const T* G;
    int64_t c0, nc;
    __device__ const T* operator()(int cp, int) const {
      const int64_t c = c0 + cp < nc ? c0 + cp : 0;
      return G + (size_t)c * (Dm::NCOMP * Dm::NGC);
    }
  };
  S::template apply<false, false>(sm, PS, sm + NL, PS, sm + 2 * NL, PS, GF{G, c0, nc});
  for (int t = threadIdx.x; t < CPB * NL; t += NT) {
    const int cp = t / NL, l = t - cp * NL;
    if (c0 + cp < nc) Y[(c0 + cp) * NL + l] = sm[cp * PS + NL + l];
  }
}

template <int DIM, int Q, typename T>
constexpr size_t ucell_smem() {
  using Dm = Dims<DIM, 1, Q, (int)sizeof(T)>;
  return sizeof(T) * (size_t)(2 * Dm::NN + Dm::SCRATCH) * ucpb(Q);
}

// -------------------------------------------------------------- Q1 transfers
// fine DoF g (not Dirichlet): sum over the corners v of its first cell of
// phi_v(node) x1[v]
template <int DIM, typename T>
__global__ void k_uq1_prolong(const T* __restrict__ x1, const int64_t* __restrict__ cells,
                              const int32_t* __restrict__ start, const int32_t* __restrict__ list,
                              const uint8_t* __restrict__ bnd, const uint8_t* __restrict__ vbnd, int64_t n, int q,
                              T* __restrict__ xf) {
  const int nq = q + 1;
  const int nloc = DIM == 3 ? nq * nq * nq : nq * nq;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    T s = T(0);
    if (!bnd[g]) {
      const int e = list[start[g]];
      const int64_t c = e / nloc;
      int l = e - (int)(c * nloc);
      double xi[3];
      for (int k = 0; k < DIM; ++k) { xi[k] = gl_node(q, l % nq); l /= nq; }
      for (int v = 0; v < (1 << DIM); ++v) {
        const int64_t vid = cells[c * (1 << DIM) + v];
        if (vbnd[vid]) continue;
        double phi = 1.0;
        for (int k = 0; k < DIM; ++k) phi *= ((v >> k) & 1) ? xi[k] : 1.0 - xi[k];
        s += T(phi) * x1[vid];
      }
    }
    xf[g] = s;
  }
}

// per cell: Y1[c][v] = sum_l phi_v(node l) r[g_l] / mult(g_l)
template <int DIM, typename T>
__global__ void k_uq1_restrict_cells(const T* __restrict__ r, const int32_t* __restrict__ cdofs,
                                     const int32_t* __restrict__ start, const uint8_t* __restrict__ bnd, int64_t nc,
                                     int q, T* __restrict__ Y1) {
  const int nq = q + 1;
  const int nloc = DIM == 3 ? nq * nq * nq : nq * nq;
  const size_t total = (size_t)nc << DIM;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int64_t c = (int64_t)(t >> DIM);
    const int v = (int)(t & ((1 << DIM) - 1));
    T s = T(0);
    for (int l = 0; l < nloc; ++l) {
      const int32_t g = cdofs[c * nloc + l];
      if (bnd[g]) continue;
      int rem = l;
      double phi = 1.0;
      for (int k = 0; k < DIM; ++k) {
        const double x = gl_node(q, rem % nq);
        rem /= nq;
        phi *= ((v >> k) & 1) ? x : 1.0 - x;
      }
      s += T(phi) * (r[g] / T(start[g + 1] - start[g]));
    }
    Y1[t] = s;
  }
}

// ------------------------------------------------------------ patch kernel
template <typename T>
struct UPatchArgs {
  int n_items, n_patches;
  const int32_t* list;            // patch ids of a sweep launch, or NULL (ids64)
  const int64_t* ids64;
  const int32_t* p_cells;         // [np][UMAXC], -1 padded
  const int32_t* p_ncell;         // [np]
  const int32_t* p_vertex;        // [np]
  int nloc[UMAXL], nimax[UMAXL], lmax[UMAXL];
  const int32_t* p_nint[UMAXL];   // [np]
  const int32_t* p_int[UMAXL];    // [np][nimax]
  const int16_t* p_cmap[UMAXL];   // [np][UMAXC][nloc]
  const int32_t* p_astart[UMAXL]; // [np][nimax + 1]
  const int32_t* p_alist[UMAXL];  // [np][lmax]
  const int32_t* cdofs0;          // [nc][nloc0] (Evaluate: closure of the top level)
  const uint8_t* bnd0;
  const T* G[UMAXL];
  const T* dinv[UMAXL];           // global, on the level's DoF numbering
  const T* bounds[UMAXL];         // [np][2]
  T* u;
  const T* b;
  const T* r_in;                  // local mode: [n_items][nimax0]
  T* d_out;
  int smoother, cheb_degree, n_mg;
  T omega;
  T* ws;                          // workspace [gridDim.x][ws_stride]
  size_t ws_stride;
  int ws_shared;                  // 1: each CTA's workspace slice lives in its shared memory (it fits)
  int off[UMAXL][5];              // r, d, res, dir, dinv offsets in a slice
  int yoff;                       // cell-output buffer offset [UMAXC][nloc_max]
};

enum { UV_R = 0, UV_D, UV_RES, UV_DIR, UV_DINV };

struct ULanczos {
  double* V;                      // scratch [gridDim.x][stride]: k basis vectors, v, w, sqrt(dinv)
  size_t stride;
  int ksteps, level;              // Lanczos steps; p-level index K
  uint64_t seed;
  double safety, ratio;           // hi = safety * theta_max, lo = max(theta_min, hi / ratio)
  double* ritz;                   // [np][2] (theta_min, theta_max) of level K
  double* b64;                    // [np][2] (lo, hi)
  float* b32;                     // [np][2] (lo, hi) rounded to FP32, or NULL
};

template <int DIM, int P, typename T, int MODE>
struct UPatch {
  static constexpr int NL = nlevels(P);
  static constexpr int NT = unt(P);
  const UPatchArgs<T>* a;
  T* ws;               // this CTA's slice
  int pid, ncell, item;
  int* cells;          // smem [UMAXC]
  int* nint;           // smem [UMAXL]
  T* coef;             // smem [UMAXL][16]
  T* sm;               // smem work area

  template <int K>
  __host__ __device__ static constexpr int q() { return P >> K; }
  template <int K>
  __host__ __device__ static constexpr int nloc() { return ipow(q<K>() + 1, DIM); }

  __device__ T* vec(int K, int which) const { return ws + a->off[K][which]; }
  __device__ T* Yg() const { return ws + a->yoff; }

  // epilogue of an apply on level K: s = (A x)_i
  __device__ void epi(int K, int kind, int it, int i, T s) const {
    T* r = vec(K, UV_R);
    T* d = vec(K, UV_D);
    T* res = vec(K, UV_RES);
    T* dir = vec(K, UV_DIR);
    const T* dv = vec(K, UV_DINV);
    const T* cf = coef + K * 16;
    switch (kind) {
      case EPI_STORE: res[i] = s; break;
      case EPI_RESID: res[i] = r[i] - s; break;
      case EPI_EVAL: r[i] -= s; break;
      case EPI_CHEB0: {
        const T rs = dv[i] * (r[i] - s);
        const T dr = rs * cf[0];
        res[i] = rs;
        dir[i] = dr;
        d[i] += dr;
        break;
      }
      case EPI_CHEB: {
        const T rs = res[i] - dv[i] * s;
        const T dr = cf[it] * dir[i] + cf[7 + it] * rs;
        res[i] = rs;
        dir[i] = dr;
        d[i] += dr;
        break;
      }
      default: d[i] += a->omega * dv[i] * (r[i] - s);
    }
  }

  // A_q applied to the level-K vector `which` (or, with CLOSURE, to the
  // closure of u), every output through the epilogue
  template <int K, bool CLOSURE>
  __device__ void apply(int which, int kind, int it) {
    constexpr int Q = q<K>(), NLOC = nloc<K>(), CPB = ucpb_patch<DIM, T>(Q, NT);
    using S = SF<DIM, 1, Q, T, NT, CPB>;
    using Dm = typename S::D;
    constexpr int PS = 2 * NLOC + Dm::SCRATCH;
    const int16_t* cmap = a->p_cmap[K] + (size_t)pid * UMAXC * NLOC;
    const T* x = vec(K, which);
    T* Y = Yg();
    for (int c0 = 0; c0 < ncell; c0 += CPB) {
      for (int t = threadIdx.x; t < CPB * NLOC; t += NT) {
        const int cp = t / NLOC, l = t - cp * NLOC;
        const int c = c0 + cp;
        T v = T(0);
        if (c < ncell) {
          if (CLOSURE) {
            const int32_t g = a->cdofs0[(size_t)cells[c] * NLOC + l];
            v = a->bnd0[g] ? T(0) : a->u[g];
          } else {
            const int m = cmap[c * NLOC + l];
            v = m >= 0 ? x[m] : T(0);
          }
        }
        sm[cp * PS + l] = v;
      }
      __syncthreads();
      struct GF {
        const T* G;
        const int* cells;
        int c0, ncell;
        __device__ const T* operator()(int cp, int) const {
          const int c = c0 + cp < ncell ? cells[c0 + cp] : cells[0];
          return G + (size_t)c * (Dm::NCOMP * Dm::NGC);
        }
      };
      S::template apply<false, false>(sm, PS, sm + NLOC, PS, sm + 2 * NLOC, PS, GF{a->G[K], cells, c0, ncell});
      for (int t = threadIdx.x; t < CPB * NLOC; t += NT) {
        const int cp = t / NLOC, l = t - cp * NLOC;
        if (c0 + cp < ncell) Y[(c0 + cp) * NLOC + l] = sm[cp * PS + NLOC + l];
      }
      __syncthreads();
    }
    const int32_t* as = a->p_astart[K] + (size_t)pid * (a->nimax[K] + 1);
    const int32_t* al = a->p_alist[K] + (size_t)pid * a->lmax[K];
    for (int i = threadIdx.x; i < nint[K]; i += NT) {
      T s = T(0);
      for (int e = as[i]; e < as[i + 1]; ++e) {
        const int32_t v = al[e];
        s += Y[(v >> 16) * NLOC + (v & 0xffff)];
      }
      epi(K, kind, it, i, s);
    }
    __syncthreads();
  }

  // one-dimensional embedding of degree qc into degree qf applied to the
  // cell array in (TRANS: its transpose), along every axis (sum factorised)
  template <int QF, int QC, bool TRANS>
  __device__ void embed_cells(const T* in, T* out, T* t1, T* t2, int ncp) {
    constexpr int NF = QF + 1, NC = QC + 1;
    constexpr int NI = TRANS ? NF : NC, NO = TRANS ? NC : NF;
    constexpr int SI = ipow(NI, DIM), SO = ipow(NO, DIM);
    // pass along axis ax: [..] with axes < ax already of size NO, the rest NI
    auto pass = [&](const T* src, T* dst, int ax) {
      const int below = ipow_rt(NO, ax), above = ipow_rt(NI, DIM - 1 - ax);
      const int ssrc = below * NI * above, sdst = below * NO * above;
      for (int t = threadIdx.x; t < ncp * sdst; t += NT) {
        const int cp = t / sdst, r = t - cp * sdst;
        const int ib = r % below, rest = r / below, o = rest % NO, ia = rest / NO;
        T s = T(0);
        for (int j = 0; j < NI; ++j) {
          const T e = TRANS ? tabE<T>(QF, j, o) : tabE<T>(QF, o, j);
          s += e * src[cp * ssrc + ib + below * (j + NI * ia)];
        }
        dst[cp * sdst + ib + below * (o + NO * ia)] = s;
      }
      __syncthreads();
    };
    (void)SI;
    (void)SO;
    if (DIM == 2) {
      pass(in, t1, 0);
      pass(t1, out, 1);
    } else {
      pass(in, t1, 0);
      pass(t1, t2, 1);
      pass(t2, out, 2);
    }
  }
  __device__ static int ipow_rt(int b, int e) {
    int r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
  }

  // r_{K+1} = P^T res_K
  template <int K>
  __device__ void restrict_res() {
    constexpr int QF = q<K>(), QC = q<K + 1>(), NF = nloc<K>(), NCL = nloc<K + 1>(), CPB = ucpb_patch<DIM, T>(QF, NT);
    const int16_t* cmap = a->p_cmap[K] + (size_t)pid * UMAXC * NF;
    const int32_t* as = a->p_astart[K] + (size_t)pid * (a->nimax[K] + 1);
    const T* res = vec(K, UV_RES);
    T* w = vec(K, UV_DIR);                       // the direction is dead between the smoothers
    for (int i = threadIdx.x; i < nint[K]; i += NT) w[i] = res[i] / T(as[i + 1] - as[i]);
    __syncthreads();
    T* Y = Yg();
    T* X = sm;
    T* t1 = sm + CPB * NF;
    T* t2 = t1 + CPB * NF;
    T* O = t2 + CPB * NF;
    for (int c0 = 0; c0 < ncell; c0 += CPB) {
      const int ncp = min(CPB, ncell - c0);
      for (int t = threadIdx.x; t < ncp * NF; t += NT) {
        const int cp = t / NF, l = t - cp * NF;
        const int m = cmap[(c0 + cp) * NF + l];
        X[t] = m >= 0 ? w[m] : T(0);
      }
      __syncthreads();
      embed_cells<QF, QC, true>(X, O, t1, t2, ncp);
      for (int t = threadIdx.x; t < ncp * NCL; t += NT) Y[c0 * NCL + t] = O[t];
      __syncthreads();
    }
    const int32_t* asc = a->p_astart[K + 1] + (size_t)pid * (a->nimax[K + 1] + 1);
    const int32_t* alc = a->p_alist[K + 1] + (size_t)pid * a->lmax[K + 1];
    T* rc = vec(K + 1, UV_R);
    for (int i = threadIdx.x; i < nint[K + 1]; i += NT) {
      T s = T(0);
      for (int e = asc[i]; e < asc[i + 1]; ++e) {
        const int32_t v = alc[e];
        s += Y[(v >> 16) * NCL + (v & 0xffff)];
      }
      rc[i] = s;
    }
    __syncthreads();
  }

  // d_K += P d_{K+1}
  template <int K>
  __device__ void prolong_add() {
    constexpr int QF = q<K>(), QC = q<K + 1>(), NF = nloc<K>(), NCL = nloc<K + 1>(), CPB = ucpb_patch<DIM, T>(QF, NT);
    const int16_t* cmapc = a->p_cmap[K + 1] + (size_t)pid * UMAXC * NCL;
    const T* dc = vec(K + 1, UV_D);
    T* Y = Yg();
    T* X = sm;
    T* t1 = sm + CPB * NF;
    T* t2 = t1 + CPB * NF;
    T* O = t2 + CPB * NF;
    for (int c0 = 0; c0 < ncell; c0 += CPB) {
      const int ncp = min(CPB, ncell - c0);
      for (int t = threadIdx.x; t < ncp * NCL; t += NT) {
        const int cp = t / NCL, l = t - cp * NCL;
        const int m = cmapc[(c0 + cp) * NCL + l];
        X[t] = m >= 0 ? dc[m] : T(0);
      }
      __syncthreads();
      embed_cells<QF, QC, false>(X, O, t1, t2, ncp);
      for (int t = threadIdx.x; t < ncp * NF; t += NT) Y[c0 * NF + t] = O[t];
      __syncthreads();
    }
    const int32_t* as = a->p_astart[K] + (size_t)pid * (a->nimax[K] + 1);
    const int32_t* al = a->p_alist[K] + (size_t)pid * a->lmax[K];
    T* d = vec(K, UV_D);
    for (int i = threadIdx.x; i < nint[K]; i += NT) {
      const int32_t v = al[as[i]];
      d[i] += Y[(v >> 16) * NF + (v & 0xffff)];
    }
    __syncthreads();
  }

  template <int K>
  __device__ void smooth(bool zero_start) {
    const int n = nint[K];
    T* r = vec(K, UV_R);
    T* d = vec(K, UV_D);
    T* res = vec(K, UV_RES);
    T* dir = vec(K, UV_DIR);
    const T* dv = vec(K, UV_DINV);
    if (a->smoother == 1) {
      if (zero_start) {
        for (int i = threadIdx.x; i < n; i += NT) d[i] = a->omega * dv[i] * r[i];
        __syncthreads();
      } else {
        apply<K, false>(UV_D, EPI_JAC, 0);
      }
      return;
    }
    if (zero_start) {
      for (int i = threadIdx.x; i < n; i += NT) {
        const T rs = dv[i] * r[i];
        const T dr = rs * coef[K * 16];
        res[i] = rs;
        dir[i] = dr;
        d[i] = dr;
      }
      __syncthreads();
    } else {
      apply<K, false>(UV_D, EPI_CHEB0, 0);
    }
    for (int it = 1; it < a->cheb_degree; ++it) apply<K, false>(UV_DIR, EPI_CHEB, it);
  }

  template <int K>
  __device__ void vcycle(bool zero_start) {
    if constexpr (q<K>() == 1) {
      T* d = vec(K, UV_D);
      const T* r = vec(K, UV_R);
      const T* dv = vec(K, UV_DINV);
      for (int i = threadIdx.x; i < nint[K]; i += NT) d[i] = r[i] * dv[i];
      __syncthreads();
    } else {
      smooth<K>(zero_start);
      apply<K, false>(UV_D, EPI_RESID, 0);
      restrict_res<K>();
      vcycle<K + 1>(true);
      prolong_add<K>();
      smooth<K>(false);
    }
  }

  template <int K>
  __device__ void load_level() {
    const int n = a->p_nint[K][pid];
    if (threadIdx.x == 0) nint[K] = n;
    const int32_t* ids = a->p_int[K] + (size_t)pid * a->nimax[K];
    T* dv = vec(K, UV_DINV);
    for (int i = threadIdx.x; i < n; i += NT) dv[i] = a->dinv[K][ids[i]];
    if constexpr (q<K>() > 1) {
      if (a->smoother == 0 && threadIdx.x < 8) {
        // Chebyshev coefficients (closed form of the recurrence, one per thread)
        const int i = threadIdx.x;
        const T lo = a->bounds[K][2 * (size_t)pid], hi = a->bounds[K][2 * (size_t)pid + 1];
        const T theta = T(0.5) * (hi + lo), delta = T(0.5) * (hi - lo);
        T* cf = coef + K * 16;
        if (i == 0) {
          cf[0] = T(1) / theta;
        } else {
          const T sigma = theta / delta;
          T cm = T(1), c0 = sigma;
          for (int k = 1; k < i; ++k) {
            const T cn = T(2) * sigma * c0 - cm;
            cm = c0;
            c0 = cn;
          }
          const T cp = T(2) * sigma * c0 - cm;
          cf[i] = cm / cp;
          cf[7 + i] = (T(2) * c0) / (delta * cp);
        }
      }
    }
    if constexpr (K + 1 < NL) load_level<K + 1>();
  }

  // the patch's cells, level sizes, diagonals and Chebyshev coefficients (pid set)
  __device__ void begin() {
    const int nc = a->p_ncell[pid];
    for (int c = threadIdx.x; c < UMAXC; c += NT) cells[c] = c < nc ? a->p_cells[(size_t)pid * UMAXC + c] : -1;
    ncell = nc;
    __syncthreads();
    load_level<0>();
    __syncthreads();
  }

  // Lanczos estimate of the extreme eigenvalues of D^-1/2 A_{j,q} D^-1/2 at
  // p-level K: k steps with full reorthogonalisation (two classical
  // Gram-Schmidt passes), FP64 basis in global scratch, start vector
  // 1 + (u - 1/2) with u from counter-based SplitMix64, counter
  // (vertex << 20) | (q << 16) | i; extreme eigenvalues of the tridiagonal
  // matrix by Sturm-sequence bisection on its Gershgorin interval
  template <int K>
  __device__ void lanczos(const ULanczos& z, double* red, double* al, double* be, double* cf) {
    constexpr int QK = q<K>();
    const int n = nint[K];
    const size_t ni = (size_t)a->nimax[K];
    double* Vb = z.V + (size_t)blockIdx.x * z.stride;
    double* dv = Vb + (size_t)z.ksteps * ni;
    double* dw = dv + ni;
    double* ds = dw + ni;
    T* x = vec(K, UV_R);
    const T* Ax = vec(K, UV_RES);
    const T* dvT = vec(K, UV_DINV);
    const uint64_t vid = (uint64_t)a->p_vertex[pid];
    for (int i = threadIdx.x; i < n; i += NT) {
      ds[i] = sqrt((double)dvT[i]);
      const uint64_t ctr = (vid << 20) | ((uint64_t)QK << 16) | (uint64_t)i;
      const uint64_t zz = splitmix64_dev(z.seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull);
      dv[i] = 1.0 + ((double)(zz >> 11) * 0x1.0p-53 - 0.5);
    }
    __syncthreads();
    const int k = z.ksteps < n ? z.ksteps : n;
    {
      double t = 0.0;
      for (int i = threadIdx.x; i < n; i += NT) t += dv[i] * dv[i];
      const double nrm = sqrt(block_sum<NT>(t, red));
      for (int i = threadIdx.x; i < n; i += NT) dv[i] /= nrm;
      __syncthreads();
    }
    int nal = 0;
    for (int j = 0; j < k; ++j) {
      for (int i = threadIdx.x; i < n; i += NT) {
        Vb[(size_t)j * ni + i] = dv[i];
        x[i] = T(ds[i] * dv[i]);
      }
      __syncthreads();
      apply<K, false>(UV_R, EPI_STORE, 0);
      double t = 0.0;
      for (int i = threadIdx.x; i < n; i += NT) {
        dw[i] = ds[i] * (double)Ax[i];
        t += dv[i] * dw[i];
      }
      const double alpha = block_sum<NT>(t, red);
      if (threadIdx.x == 0) al[j] = alpha;
      nal = j + 1;
      for (int pass = 0; pass < 2; ++pass) {
        for (int m = 0; m <= j; ++m) {
          double c = 0.0;
          for (int i = threadIdx.x; i < n; i += NT) c += Vb[(size_t)m * ni + i] * dw[i];
          c = block_sum<NT>(c, red);
          if (threadIdx.x == 0) cf[m] = c;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += NT) {
          double w = dw[i];
          for (int m = 0; m <= j; ++m) w -= cf[m] * Vb[(size_t)m * ni + i];
          dw[i] = w;
        }
        __syncthreads();
      }
      if (j == k - 1) break;
      double b2 = 0.0;
      for (int i = threadIdx.x; i < n; i += NT) b2 += dw[i] * dw[i];
      const double b = sqrt(block_sum<NT>(b2, red));
      if (b <= 1e-300) break;
      if (threadIdx.x == 0) be[j] = b;
      for (int i = threadIdx.x; i < n; i += NT) dv[i] = dw[i] / b;
      __syncthreads();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double lo = 1e300, hi = -1e300;
      for (int i = 0; i < nal; ++i) {
        const double bl = i > 0 ? fabs(be[i - 1]) : 0.0, br = i < nal - 1 ? fabs(be[i]) : 0.0;
        lo = fmin(lo, al[i] - bl - br);
        hi = fmax(hi, al[i] + bl + br);
      }
      double ext[2];
      for (int e = 0; e < 2; ++e) {
        const int kidx = e == 0 ? 0 : nal - 1;
        double x0 = lo, x1 = hi;
        for (int it = 0; it < 100; ++it) {
          const double mid = 0.5 * (x0 + x1);
          if (sturm_count_dev(al, be, nal, mid) > kidx) x1 = mid;
          else x0 = mid;
        }
        ext[e] = 0.5 * (x0 + x1);
      }
      const double bhi = z.safety * ext[1];
      const double blo = fmax(ext[0], bhi / z.ratio);
      const size_t o = 2 * (size_t)pid;
      z.ritz[o] = ext[0];
      z.ritz[o + 1] = ext[1];
      z.b64[o] = blo;
      z.b64[o + 1] = bhi;
      if (z.b32) {
        z.b32[o] = (float)blo;
        z.b32[o + 1] = (float)bhi;
      }
    }
    __syncthreads();
  }

  template <int K>
  __device__ void lanczos_at(const ULanczos& z, double* red, double* al, double* be, double* cf) {
    if constexpr (K < NL) {
      if (z.level == K) {
        if constexpr (q<K>() > 1) lanczos<K>(z, red, al, be, cf);
      } else {
        lanczos_at<K + 1>(z, red, al, be, cf);
      }
    }
  }

  __device__ void run() {
    if (MODE == MODE_SWEEP) {
      pid = a->list[item];
    } else {
      const int64_t raw = a->ids64[item];
      if (raw < 0 || raw >= a->n_patches) {             // not a patch: a zero row
        for (int i = threadIdx.x; i < a->nimax[0]; i += NT) a->d_out[(size_t)item * a->nimax[0] + i] = T(0);
        return;
      }
      pid = (int)raw;
    }
    begin();
    constexpr int N0 = nloc<0>();
    const int32_t* ids = a->p_int[0] + (size_t)pid * a->nimax[0];
    T* r = vec(0, UV_R);
    if (MODE == MODE_SWEEP) {
      for (int i = threadIdx.x; i < nint[0]; i += NT) r[i] = a->b[ids[i]];
      __syncthreads();
      apply<0, true>(UV_R, EPI_EVAL, 0);                   // r = b - A u on the patch interior
    } else {
      for (int i = threadIdx.x; i < nint[0]; i += NT) r[i] = a->r_in[(size_t)item * a->nimax[0] + i];
      __syncthreads();
    }
    (void)N0;
    for (int cyc = 0; cyc < a->n_mg; ++cyc) vcycle<0>(cyc == 0);
    const T* d = vec(0, UV_D);
    if (MODE == MODE_SWEEP) {
      for (int i = threadIdx.x; i < nint[0]; i += NT) a->u[ids[i]] += d[i];
    } else {
      for (int i = threadIdx.x; i < a->nimax[0]; i += NT)
        a->d_out[(size_t)item * a->nimax[0] + i] = i < nint[0] ? d[i] : T(0);
    }
    __syncthreads();
  }
};

template <int DIM, int P, typename T>
constexpr size_t upatch_smem() {
  // max over levels of the apply buffers and the transfer buffers
  size_t m = 0;
  for (int k = 0, q = P; q >= 1; ++k, q >>= 1) {
    const int n = q + 1;
    const int nl = DIM == 3 ? n * n * n : n * n;
    const int cpb = ucpb_patch<DIM, T>(q, unt(P));
    const size_t ap = (size_t)cpb * (2 * nl + sf_scratch(DIM, 1, q, false, (int)sizeof(T)));
    const size_t tr = (size_t)cpb * 4 * nl;
    m = ap > m ? ap : m;
    m = tr > m ? tr : m;
  }
  return sizeof(T) * m + sizeof(int) * (UMAXC + UMAXL) + sizeof(T) * UMAXL * 16 + 64;
}

template <int DIM, int P, typename T>
__host__ __device__ constexpr size_t upatch_smem_aligned() {
  return (upatch_smem<DIM, P, T>() + 15) & ~size_t(15);
}

template <int DIM, int P, typename T, int MODE>
__global__ void __launch_bounds__(unt(P)) k_upatch(const __grid_constant__ UPatchArgs<T> args) {
  UPatch<DIM, P, T, MODE> k;
  k.a = &args;
  constexpr size_t WS_OFF = upatch_smem_aligned<DIM, P, T>();
  k.ws = args.ws_shared ? reinterpret_cast<T*>(pmg_smem + WS_OFF) : args.ws + (size_t)blockIdx.x * args.ws_stride;
  unsigned char* base = pmg_smem;
  k.cells = reinterpret_cast<int*>(base);
  k.nint = k.cells + UMAXC;
  k.coef = reinterpret_cast<T*>(base + ((sizeof(int) * (UMAXC + UMAXL) + 15) & ~size_t(15)));
  k.sm = k.coef + UMAXL * 16;
  for (int item = blockIdx.x; item < args.n_items; item += gridDim.x) {
    k.item = item;
    k.run();
  }
}

template <int DIM, int P>
__global__ void __launch_bounds__(unt(P)) k_ulanczos(const __grid_constant__ UPatchArgs<double> args,
                                                  const __grid_constant__ ULanczos z) {
  __shared__ double red[unt(P) / 32 + 2], al[64], be[64], cf[64];
  UPatch<DIM, P, double, MODE_LOCAL> k;
  k.a = &args;
  k.ws = args.ws + (size_t)blockIdx.x * args.ws_stride;
  unsigned char* base = pmg_smem;
  k.cells = reinterpret_cast<int*>(base);
  k.nint = k.cells + UMAXC;
  k.coef = reinterpret_cast<double*>(base + ((sizeof(int) * (UMAXC + UMAXL) + 15) & ~size_t(15)));
  k.sm = k.coef + UMAXL * 16;
  for (int item = blockIdx.x; item < args.n_patches; item += gridDim.x) {
    k.item = item;
    k.pid = item;
    k.begin();
    k.template lanczos_at<0>(z, red, al, be, cf);
  }
}

// Launchers of the heavy kernels; explicit instantiations per dimension and
// degree live in the umesh_k*.cu units (umesh_launch.cuh has the definitions).
template <int DIM, int Q, typename T>
int ucell_apply_q(const T* u, const T* G, const int32_t* cd, const uint8_t* bnd, int64_t nc, T* Y, cudaStream_t s);
template <int DIM, int P, typename T>
int upatch_launch_P(int mode, const UPatchArgs<T>& a, int grid, cudaStream_t s);
template <int DIM, int P>
int ulanczos_launch(const UPatchArgs<double>& a, const ULanczos& z, int grid, cudaStream_t s);

}  // namespace pmg
