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
constexpr int UNT = 128;              // threads per CTA of the patch kernel
constexpr int UMAXL = 4;              // p-levels (p <= 8: p, p/2, p/4, 1)

__host__ __device__ constexpr int ucpb(int q) { return q <= 4 ? 4 : 2; }   // cells per pass

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
  using Dm = Dims<DIM, 1, Q>;
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
  int n_items;
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
  int off[UMAXL][5];              // r, d, res, dir, dinv offsets in a slice
  int yoff;                       // cell-output buffer offset [UMAXC][nloc_max]
};

enum { UV_R = 0, UV_D, UV_RES, UV_DIR, UV_DINV };

template <int DIM, int P, typename T, int MODE>
struct UPatch {
  static constexpr int NL = nlevels(P);
  static constexpr int NT = UNT;
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
    constexpr int Q = q<K>(), NLOC = nloc<K>(), CPB = ucpb(Q);
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
    constexpr int QF = q<K>(), QC = q<K + 1>(), NF = nloc<K>(), NCL = nloc<K + 1>(), CPB = ucpb(QF);
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
    constexpr int QF = q<K>(), QC = q<K + 1>(), NF = nloc<K>(), NCL = nloc<K + 1>(), CPB = ucpb(QF);
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

  __device__ void run() {
    if (MODE == MODE_SWEEP) pid = a->list[item];
    else pid = (int)a->ids64[item];
    const int nc = a->p_ncell[pid];
    for (int c = threadIdx.x; c < UMAXC; c += NT) cells[c] = c < nc ? a->p_cells[(size_t)pid * UMAXC + c] : -1;
    ncell = nc;
    __syncthreads();
    load_level<0>();
    __syncthreads();
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
    const int NQ = DIM == 3 ? n * n * n : n * n;
    const int T1 = DIM == 3 ? n * n * n : n * n, T2 = DIM == 3 ? n * n * n : 0;
    const int R = (T1 + T2) > DIM * NQ ? (T1 + T2) : DIM * NQ;
    const size_t ap = (size_t)ucpb(q) * (2 * nl + NQ + R);
    const size_t tr = (size_t)ucpb(q) * 4 * nl;
    m = ap > m ? ap : m;
    m = tr > m ? tr : m;
  }
  return sizeof(T) * m + sizeof(int) * (UMAXC + UMAXL) + sizeof(T) * UMAXL * 16 + 64;
}

template <int DIM, int P, typename T, int MODE>
__global__ void __launch_bounds__(UNT) k_upatch(const __grid_constant__ UPatchArgs<T> args) {
  UPatch<DIM, P, T, MODE> k;
  k.a = &args;
  k.ws = args.ws + (size_t)blockIdx.x * args.ws_stride;
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

// ------------------------------------------------------------------ host side
struct ULevelD {
  int q = 0, nloc = 0, nimax = 0, lmax = 0;
  int64_t ndofs = 0;
  std::vector<int32_t> h_cdofs;
  std::vector<uint8_t> h_bnd;
  int32_t *cdofs = nullptr, *dstart = nullptr, *dlist = nullptr;
  uint8_t* bnd = nullptr;
  int32_t *p_nint = nullptr, *p_int = nullptr, *p_astart = nullptr, *p_alist = nullptr;
  int16_t* p_cmap = nullptr;
  double* G64 = nullptr;
  float* G32 = nullptr;
  double *dinv64 = nullptr, *bounds64 = nullptr;
  float *dinv32 = nullptr, *bounds32 = nullptr;
};

struct UMesh {
  int dim = 0;
  int64_t nv = 0, nc = 0;
  std::vector<double> h_coords, h_kappa;
  std::vector<int64_t> h_cells;
  std::vector<uint8_t> h_vob;
  UTopo topo;
  UOptions opt{};
  int p = 0, npl = 0;
  ULevelD L[UMAXL];
  std::vector<int64_t> pverts;
  std::vector<std::vector<int32_t>> pcells;
  std::vector<uint8_t> colour;
  int ncolours = 0;
  std::vector<std::vector<int32_t>> h_colour_list;
  std::vector<int32_t*> colour_list;
  int32_t *p_cells = nullptr, *p_ncell = nullptr, *p_vertex = nullptr;
  double *coords = nullptr, *kappa = nullptr;
  int64_t* cells = nullptr;
  uint8_t* vbnd = nullptr;
  int32_t *vstart = nullptr, *vlist = nullptr;
  // coarse Q1 space
  int nf1 = 0;
  int* freeidx1 = nullptr;
  double* Ainv = nullptr;
  // work vectors (FP64 and FP32)
  double *x64 = nullptr, *b64 = nullptr, *r64 = nullptr, *Y64 = nullptr, *r1_64 = nullptr, *x1_64 = nullptr;
  float *x32 = nullptr, *b32 = nullptr, *r32 = nullptr, *Y32 = nullptr, *r1_32 = nullptr, *x1_32 = nullptr;
  double* ws64 = nullptr;
  float* ws32 = nullptr;
  size_t ws_stride = 0;
  int ws_grid = 0;
  int off[UMAXL][5] = {};
  int yoff = 0;
  int* err = nullptr;
  int64_t launches = 0;
  std::vector<void*> allocs;
  ~UMesh() {
    for (void* q : allocs) cudaFree(q);
    for (int32_t* c : colour_list) cudaFree(c);
  }
  template <typename T>
  int alloc(T** ptr, size_t n) {
    if (cudaMalloc(ptr, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return ST_CUDA;
    allocs.push_back(*ptr);
    return ST_OK;
  }
  template <typename T>
  int upload(T** ptr, const std::vector<T>& h) {
    int st = alloc(ptr, h.size());
    if (st) return st;
    if (!h.empty() && cudaMemcpy(*ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
      return ST_CUDA;
    return ST_OK;
  }
};

#define UCK(x)                                  \
  do {                                          \
    const int st__ = (x);                       \
    if (st__) return st__;                      \
  } while (0)
#define UCU(x)                                          \
  do {                                                  \
    if ((x) != cudaSuccess) return ST_CUDA;             \
  } while (0)

UMesh* umesh_create(int dim, int64_t nv, const double* coords, int64_t nc, const int64_t* cells,
                    const uint8_t* vob, std::string* msg) {
  std::unique_ptr<UMesh> m(new UMesh());
  *msg = utopo_build(dim, nv, nc, cells, vob, &m->topo);
  if (!msg->empty()) return nullptr;
  m->dim = dim;
  m->nv = nv;
  m->nc = nc;
  m->h_coords.assign(coords, coords + nv * dim);
  m->h_cells.assign(cells, cells + nc * (1 << dim));
  m->h_kappa.assign(nc, 1.0);
  m->h_vob = m->topo.vertex_on_boundary;
  for (int64_t i = 0; i < nv * dim; ++i)
    if (!std::isfinite(coords[i])) {
      *msg = "coordinates must be finite";
      return nullptr;
    }
  return m.release();
}

void umesh_destroy(UMesh* m) { delete m; }

int umesh_set_kappa(UMesh* m, const double* kappa) {
  for (int64_t c = 0; c < m->nc; ++c)
    if (!std::isfinite(kappa[c]) || !(kappa[c] > 0)) return ST_ARG;
  m->h_kappa.assign(kappa, kappa + m->nc);
  return ST_OK;
}

template <int DIM, int Q, typename T>
static int ucell_apply_q(const T* u, const T* G, const int32_t* cd, const uint8_t* bnd, int64_t nc, T* Y,
                         cudaStream_t s) {
  constexpr int CPB = ucpb(Q);
  constexpr size_t sm = ucell_smem<DIM, Q, T>();
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (!attr[dev & 63]) {
    if (cudaFuncSetAttribute(k_ucell_apply<DIM, Q, T, CPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
        cudaSuccess)
      return ST_CUDA;
    attr[dev & 63] = true;
  }
  const int64_t grid = (nc + CPB - 1) / CPB;
  k_ucell_apply<DIM, Q, T, CPB><<<(unsigned)grid, 128, sm, s>>>(u, G, cd, bnd, nc, Y);
  return cudaPeekAtLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

template <int DIM, typename T>
static int ucell_apply(int q, const T* u, const T* G, const int32_t* cd, const uint8_t* bnd, int64_t nc, T* Y,
                       cudaStream_t s) {
  switch (q) {
    case 1: return ucell_apply_q<DIM, 1, T>(u, G, cd, bnd, nc, Y, s);
    case 2: return ucell_apply_q<DIM, 2, T>(u, G, cd, bnd, nc, Y, s);
    case 3: return ucell_apply_q<DIM, 3, T>(u, G, cd, bnd, nc, Y, s);
    case 4: return ucell_apply_q<DIM, 4, T>(u, G, cd, bnd, nc, Y, s);
    case 5: return ucell_apply_q<DIM, 5, T>(u, G, cd, bnd, nc, Y, s);
    case 6: return ucell_apply_q<DIM, 6, T>(u, G, cd, bnd, nc, Y, s);
    case 7: return ucell_apply_q<DIM, 7, T>(u, G, cd, bnd, nc, Y, s);
    case 8: return ucell_apply_q<DIM, 8, T>(u, G, cd, bnd, nc, Y, s);
    default: return ST_UNSUPPORTED;
  }
}

// global operator of level k (FP64 or FP32): out = A_k u, Dirichlet rows 0
template <typename T>
static int uglobal_apply(UMesh* m, int k, const T* u, T* out, T* Y, cudaStream_t s) {
  ULevelD& L = m->L[k];
  const T* G;
  if constexpr (sizeof(T) == 8) G = L.G64;
  else G = L.G32;
  const int st = m->dim == 2 ? ucell_apply<2, T>(L.q, u, G, L.cdofs, L.bnd, m->nc, Y, s)
                             : ucell_apply<3, T>(L.q, u, G, L.cdofs, L.bnd, m->nc, Y, s);
  if (st) return st;
  k_uassemble<T><<<grid_for((size_t)L.ndofs, 256), 256, 0, s>>>(Y, L.dstart, L.dlist, L.bnd, L.ndofs, out);
  m->launches += 2;
  return cudaPeekAtLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

// ---- patch structure of one p-level on the host
static std::string build_patch_level(UMesh* m, int k) {
  ULevelD& L = m->L[k];
  const int q = L.q;
  const int64_t np = (int64_t)m->pverts.size();
  const int nloc = L.nloc;
  // owner cells of every DoF (from the global assembly lists, increasing cell)
  std::vector<int32_t> dstart(L.ndofs + 1, 0);
  for (int64_t c = 0; c < m->nc; ++c)
    for (int l = 0; l < nloc; ++l) ++dstart[L.h_cdofs[c * nloc + l] + 1];
  for (int64_t g = 0; g < L.ndofs; ++g) dstart[g + 1] += dstart[g];
  std::vector<int32_t> dlist(dstart.back()), fill(dstart.begin(), dstart.end() - 1);
  for (int64_t c = 0; c < m->nc; ++c)
    for (int l = 0; l < nloc; ++l) dlist[fill[L.h_cdofs[c * nloc + l]]++] = (int32_t)(c * nloc + l);
  if (dlist.size() > (size_t)INT32_MAX) return "too many cell nodes";
  std::vector<std::vector<int32_t>> pint(np);
  std::vector<std::vector<int16_t>> cmap(np);
  std::vector<std::vector<int32_t>> astart(np), alist(np);
  int nimax = 1, lmax = 1;
  for (int64_t j = 0; j < np; ++j) {
    const auto& cs = m->pcells[j];
    std::vector<int32_t> closure;
    for (int32_t c : cs)
      for (int l = 0; l < nloc; ++l) closure.push_back(L.h_cdofs[(size_t)c * nloc + l]);
    std::sort(closure.begin(), closure.end());
    closure.erase(std::unique(closure.begin(), closure.end()), closure.end());
    for (int32_t g : closure) {
      if (L.h_bnd[g]) continue;
      bool inside = true;
      for (int e = dstart[g]; e < dstart[g + 1] && inside; ++e)
        inside = std::binary_search(cs.begin(), cs.end(), (int32_t)(dlist[e] / nloc));
      if (inside) pint[j].push_back(g);
    }
    if (pint[j].size() > 32767) return "a patch has more than 32767 interior DoFs";
    const int ni = (int)pint[j].size();
    cmap[j].assign((size_t)UMAXC * nloc, -1);
    std::vector<std::vector<int32_t>> entries(ni);
    for (size_t s = 0; s < cs.size(); ++s)
      for (int l = 0; l < nloc; ++l) {
        const int32_t g = L.h_cdofs[(size_t)cs[s] * nloc + l];
        auto it = std::lower_bound(pint[j].begin(), pint[j].end(), g);
        if (it != pint[j].end() && *it == g) {
          const int i = (int)(it - pint[j].begin());
          cmap[j][s * nloc + l] = (int16_t)i;
          entries[i].push_back((int32_t)((s << 16) | l));
        }
      }
    astart[j].assign(ni + 1, 0);
    for (int i = 0; i < ni; ++i) {
      astart[j][i + 1] = astart[j][i] + (int32_t)entries[i].size();
      for (int32_t e : entries[i]) alist[j].push_back(e);
    }
    nimax = std::max(nimax, ni);
    lmax = std::max(lmax, (int)alist[j].size());
  }
  if (nloc > 65535) return "cell too large";
  L.nimax = nimax;
  L.lmax = lmax;
  std::vector<int32_t> h_nint(np), h_int((size_t)np * nimax, 0), h_as((size_t)np * (nimax + 1), 0),
      h_al((size_t)np * lmax, 0);
  std::vector<int16_t> h_cmap((size_t)np * UMAXC * nloc, -1);
  for (int64_t j = 0; j < np; ++j) {
    h_nint[j] = (int32_t)pint[j].size();
    std::copy(pint[j].begin(), pint[j].end(), h_int.begin() + (size_t)j * nimax);
    std::copy(astart[j].begin(), astart[j].end(), h_as.begin() + (size_t)j * (nimax + 1));
    std::copy(alist[j].begin(), alist[j].end(), h_al.begin() + (size_t)j * lmax);
    std::copy(cmap[j].begin(), cmap[j].end(), h_cmap.begin() + (size_t)j * UMAXC * nloc);
  }
  if (m->upload(&L.dstart, dstart) || m->upload(&L.dlist, dlist) || m->upload(&L.p_nint, h_nint) ||
      m->upload(&L.p_int, h_int) || m->upload(&L.p_astart, h_as) || m->upload(&L.p_alist, h_al) ||
      m->upload(&L.p_cmap, h_cmap))
    return "device allocation failed";
  (void)q;
  return "";
}

template <typename T>
static void fill_args(UMesh* m, UPatchArgs<T>& a) {
  std::memset(&a, 0, sizeof(a));
  a.p_cells = m->p_cells;
  a.p_ncell = m->p_ncell;
  a.p_vertex = m->p_vertex;
  for (int k = 0; k < m->npl; ++k) {
    const ULevelD& L = m->L[k];
    a.nloc[k] = L.nloc;
    a.nimax[k] = L.nimax;
    a.lmax[k] = L.lmax;
    a.p_nint[k] = L.p_nint;
    a.p_int[k] = L.p_int;
    a.p_cmap[k] = L.p_cmap;
    a.p_astart[k] = L.p_astart;
    a.p_alist[k] = L.p_alist;
    if constexpr (sizeof(T) == 8) {
      a.G[k] = L.G64;
      a.dinv[k] = L.dinv64;
      a.bounds[k] = L.bounds64;
    } else {
      a.G[k] = L.G32;
      a.dinv[k] = L.dinv32;
      a.bounds[k] = L.bounds32;
    }
    for (int w = 0; w < 5; ++w) a.off[k][w] = m->off[k][w];
  }
  a.cdofs0 = m->L[0].cdofs;
  a.bnd0 = m->L[0].bnd;
  a.smoother = m->opt.smoother;
  a.cheb_degree = m->opt.cheb_degree;
  a.n_mg = m->opt.n_mg;
  a.omega = T(m->opt.omega);
  if constexpr (sizeof(T) == 8) a.ws = m->ws64;
  else a.ws = m->ws32;
  a.ws_stride = m->ws_stride;
  a.yoff = m->yoff;
}

template <int DIM, int P, typename T>
static int upatch_launch_P(int mode, const UPatchArgs<T>& a, int grid, cudaStream_t s) {
  constexpr size_t sm = upatch_smem<DIM, P, T>();
  if constexpr (sm > 227 * 1024) {
    return ST_UNSUPPORTED;
  } else {
    int dev = 0;
    cudaGetDevice(&dev);
    static bool attr[2][64] = {};
    if (mode == MODE_SWEEP) {
      if (!attr[0][dev & 63]) {
        if (cudaFuncSetAttribute(k_upatch<DIM, P, T, MODE_SWEEP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm) != cudaSuccess)
          return ST_CUDA;
        attr[0][dev & 63] = true;
      }
      k_upatch<DIM, P, T, MODE_SWEEP><<<grid, UNT, sm, s>>>(a);
    } else {
      if (!attr[1][dev & 63]) {
        if (cudaFuncSetAttribute(k_upatch<DIM, P, T, MODE_LOCAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sm) != cudaSuccess)
          return ST_CUDA;
        attr[1][dev & 63] = true;
      }
      k_upatch<DIM, P, T, MODE_LOCAL><<<grid, UNT, sm, s>>>(a);
    }
    return cudaPeekAtLastError() == cudaSuccess ? ST_OK : ST_CUDA;
  }
}

template <int DIM, typename T>
static int upatch_launch(int p, int mode, const UPatchArgs<T>& a, int grid, cudaStream_t s) {
  switch (p) {
    case 1: return upatch_launch_P<DIM, 1, T>(mode, a, grid, s);
    case 2: return upatch_launch_P<DIM, 2, T>(mode, a, grid, s);
    case 3: return upatch_launch_P<DIM, 3, T>(mode, a, grid, s);
    case 4: return upatch_launch_P<DIM, 4, T>(mode, a, grid, s);
    case 5: return upatch_launch_P<DIM, 5, T>(mode, a, grid, s);
    case 6: return upatch_launch_P<DIM, 6, T>(mode, a, grid, s);
    case 7: return upatch_launch_P<DIM, 7, T>(mode, a, grid, s);
    case 8: return upatch_launch_P<DIM, 8, T>(mode, a, grid, s);
    default: return ST_UNSUPPORTED;
  }
}

template <typename T>
static int usweep_colour_T(UMesh* m, int colour, const T* b, T* u, cudaStream_t s) {
  const int n = (int)m->h_colour_list[colour].size();
  if (n == 0) return ST_OK;
  UPatchArgs<T> a;
  fill_args(m, a);
  a.n_items = n;
  a.list = m->colour_list[colour];
  a.u = u;
  a.b = b;
  const int grid = std::min(n, m->ws_grid);
  ++m->launches;
  return m->dim == 2 ? upatch_launch<2, T>(m->p, MODE_SWEEP, a, grid, s)
                     : upatch_launch<3, T>(m->p, MODE_SWEEP, a, grid, s);
}

template <typename T>
static int usweep_T(UMesh* m, const T* b, T* u, bool reverse, cudaStream_t s) {
  for (int i = 0; i < m->ncolours; ++i) {
    const int c = reverse ? m->ncolours - 1 - i : i;
    UCK(usweep_colour_T<T>(m, c, b, u, s));
  }
  return ST_OK;
}

// ---- set-up
int umesh_setup(UMesh* m, int p, const UOptions& o, cudaStream_t s, int* err_dev, std::string* msg) {
  if (p < 1 || p > 8) {
    *msg = "degree must be in 1..8";
    return ST_UNSUPPORTED;
  }
  m->p = p;
  m->opt = o;
  m->err = err_dev;
  const int d = m->dim, ncorner = 1 << d;
  m->npl = 0;
  for (int q = p; q >= 1; q >>= 1) m->L[m->npl++].q = q;
  // patches and colours
  m->pverts = utopo_patch_vertices(m->topo);
  const int64_t np = (int64_t)m->pverts.size();
  m->pcells.assign(np, {});
  std::vector<int32_t> h_pcells((size_t)np * UMAXC, -1), h_ncell(np), h_pv(np);
  for (int64_t j = 0; j < np; ++j) {
    const auto& vc = m->topo.vertex_cells[m->pverts[j]];
    if ((int)vc.size() > UMAXC) {
      *msg = "a vertex has more cells than the unstructured patch kernel accepts (PMG_UMAXC)";
      return ST_UNSUPPORTED;
    }
    for (size_t i = 0; i < vc.size(); ++i) {
      m->pcells[j].push_back((int32_t)vc[i]);
      h_pcells[(size_t)j * UMAXC + i] = (int32_t)vc[i];
    }
    h_ncell[j] = (int32_t)vc.size();
    h_pv[j] = (int32_t)m->pverts[j];
  }
  m->colour = utopo_colours(m->topo, m->pverts, o.seed, &m->ncolours);
  m->h_colour_list.assign(m->ncolours, {});
  for (int64_t j = 0; j < np; ++j) m->h_colour_list[m->colour[j]].push_back((int32_t)j);
  for (auto& cl : m->h_colour_list) {
    int32_t* dptr = nullptr;
    if (cudaMalloc(&dptr, std::max<size_t>(cl.size(), 1) * sizeof(int32_t)) != cudaSuccess) return ST_CUDA;
    m->colour_list.push_back(dptr);
    if (!cl.empty()) UCU(cudaMemcpy(dptr, cl.data(), cl.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  }
  UCK(m->upload(&m->p_cells, h_pcells));
  UCK(m->upload(&m->p_ncell, h_ncell));
  UCK(m->upload(&m->p_vertex, h_pv));
  UCK(m->upload(&m->coords, m->h_coords));
  UCK(m->upload(&m->kappa, m->h_kappa));
  UCK(m->upload(&m->cells, m->h_cells));
  UCK(m->upload(&m->vbnd, m->h_vob));
  // vertex -> (cell, corner) lists for the Q1 restriction
  {
    std::vector<int32_t> vs(m->nv + 1, 0), vl;
    for (int64_t v = 0; v < m->nv; ++v) vs[v + 1] = vs[v] + (int32_t)m->topo.vertex_cells[v].size();
    vl.resize(vs.back());
    for (int64_t v = 0; v < m->nv; ++v) {
      int e = vs[v];
      for (int64_t c : m->topo.vertex_cells[v])
        for (int k = 0; k < ncorner; ++k)
          if (m->h_cells[c * ncorner + k] == v) vl[e++] = (int32_t)(c * ncorner + k);
    }
    UCK(m->upload(&m->vstart, vs));
    UCK(m->upload(&m->vlist, vl));
  }
  const bool mixed = o.precision == PMG_PREC_MIXED;
  size_t ymax = 0;
  for (int k = 0; k < m->npl; ++k) {
    ULevelD& L = m->L[k];
    const int q = L.q;
    L.nloc = 1;
    for (int i = 0; i < d; ++i) L.nloc *= q + 1;
    L.ndofs = utopo_ndofs(m->topo, q);
    if (L.ndofs > INT32_MAX) {
      *msg = "too many DoFs";
      return ST_UNSUPPORTED;
    }
    L.h_cdofs = utopo_cell_dofs(m->topo, q);
    L.h_bnd = utopo_boundary_dofs(m->topo, q);
    UCK(m->upload(&L.cdofs, L.h_cdofs));
    UCK(m->upload(&L.bnd, L.h_bnd));
    *msg = build_patch_level(m, k);
    if (!msg->empty()) return ST_CUDA;
    // geometry
    const size_t ng = (size_t)m->nc * (d * (d + 1) / 2) * L.nloc;
    UCK(m->alloc(&L.G64, ng));
    const int gb = grid_for(ng / (d * (d + 1) / 2), 256);
    if (d == 2) k_ugeometry<2, double><<<gb, 256, 0, s>>>(m->coords, m->cells, m->kappa, m->nc, q, L.G64, err_dev);
    else k_ugeometry<3, double><<<gb, 256, 0, s>>>(m->coords, m->cells, m->kappa, m->nc, q, L.G64, err_dev);
    UCU(cudaPeekAtLastError());
    if (mixed) {
      UCK(m->alloc(&L.G32, ng));
      if (d == 2) k_ugeometry<2, float><<<gb, 256, 0, s>>>(m->coords, m->cells, m->kappa, m->nc, q, L.G32, err_dev);
      else k_ugeometry<3, float><<<gb, 256, 0, s>>>(m->coords, m->cells, m->kappa, m->nc, q, L.G32, err_dev);
      UCU(cudaPeekAtLastError());
    }
    // level diagonal
    double *Yd = nullptr, *diag = nullptr;
    UCU(cudaMalloc(&Yd, (size_t)m->nc * L.nloc * sizeof(double)));
    UCU(cudaMalloc(&diag, (size_t)L.ndofs * sizeof(double)));
    if (d == 2) k_ucell_diag<2><<<grid_for((size_t)m->nc * L.nloc, 256), 256, 0, s>>>(L.G64, m->nc, q, Yd);
    else k_ucell_diag<3><<<grid_for((size_t)m->nc * L.nloc, 256), 256, 0, s>>>(L.G64, m->nc, q, Yd);
    k_uassemble<double><<<grid_for((size_t)L.ndofs, 256), 256, 0, s>>>(Yd, L.dstart, L.dlist, L.bnd, L.ndofs, diag);
    UCK(m->alloc(&L.dinv64, L.ndofs));
    if (mixed) UCK(m->alloc(&L.dinv32, L.ndofs));
    k_uinvert<float><<<grid_for((size_t)L.ndofs, 256), 256, 0, s>>>(diag, L.bnd, L.ndofs, L.dinv64, L.dinv32);
    UCU(cudaPeekAtLastError());
    UCU(cudaStreamSynchronize(s));
    cudaFree(Yd);
    cudaFree(diag);
    // Chebyshev intervals (fixed; replaced by pmg_set_bounds)
    std::vector<double> bd(2 * np);
    for (int64_t j = 0; j < np; ++j) { bd[2 * j] = o.fixed_lo; bd[2 * j + 1] = o.fixed_hi; }
    UCK(m->upload(&L.bounds64, bd));
    std::vector<float> bf(bd.begin(), bd.end());
    UCK(m->upload(&L.bounds32, bf));
    ymax = std::max(ymax, (size_t)UMAXC * L.nloc);
  }
  int h_err = 0;
  UCU(cudaMemcpy(&h_err, err_dev, sizeof(int), cudaMemcpyDeviceToHost));
  if (h_err) {
    *msg = "degenerate cell: det J <= 0 at a Gauss point or vertex";
    return ST_DEGENERATE;
  }
  // patch workspace: per CTA, per level r, d, res, dir, dinv, and the cell-output buffer
  size_t off = 0;
  for (int k = 0; k < m->npl; ++k)
    for (int w = 0; w < 5; ++w) {
      m->off[k][w] = (int)off;
      off += (size_t)m->L[k].nimax;
    }
  m->yoff = (int)off;
  off += ymax;
  m->ws_stride = (off + 31) & ~size_t(31);
  m->ws_grid = (int)std::min<int64_t>(std::max<int64_t>(np, 1), 152 * 8);
  UCK(m->alloc(&m->ws64, m->ws_stride * m->ws_grid));
  if (mixed) UCK(m->alloc(&m->ws32, m->ws_stride * m->ws_grid));
  // global work vectors
  const ULevelD& L0 = m->L[0];
  const size_t nd = (size_t)L0.ndofs, ny = (size_t)m->nc * L0.nloc;
  UCK(m->alloc(&m->x64, nd));
  UCK(m->alloc(&m->b64, nd));
  UCK(m->alloc(&m->r64, nd));
  UCK(m->alloc(&m->Y64, std::max(ny, (size_t)m->nc * ncorner)));
  UCK(m->alloc(&m->r1_64, m->nv));
  UCK(m->alloc(&m->x1_64, m->nv));
  if (mixed) {
    UCK(m->alloc(&m->x32, nd));
    UCK(m->alloc(&m->b32, nd));
    UCK(m->alloc(&m->r32, nd));
    UCK(m->alloc(&m->Y32, std::max(ny, (size_t)m->nc * ncorner)));
    UCK(m->alloc(&m->r1_32, m->nv));
    UCK(m->alloc(&m->x1_32, m->nv));
  }
  // coarse Q1 space: dense inverse of the Q1 operator on the free vertices
  {
    const int k1 = m->npl - 1;                      // the q = 1 level
    const ULevelD& L1 = m->L[k1];
    std::vector<int> fidx;
    for (int64_t v = 0; v < m->nv; ++v)
      if (!m->h_vob[v]) fidx.push_back((int)v);
    m->nf1 = (int)fidx.size();
    if (m->nf1 > 16384) {
      *msg = "the Q1 coarse space has more than 16384 free vertices";
      return ST_UNSUPPORTED;
    }
    if (m->nf1 > 0) {
      UCK(m->upload(&m->freeidx1, fidx));
      double *cols = nullptr, *e = nullptr, *A = nullptr, *Y1 = nullptr;
      UCU(cudaMalloc(&cols, (size_t)m->nf1 * m->nv * sizeof(double)));
      UCU(cudaMalloc(&e, (size_t)m->nv * sizeof(double)));
      UCU(cudaMalloc(&Y1, (size_t)m->nc * ncorner * sizeof(double)));
      for (int j = 0; j < m->nf1; ++j) {
        UCU(cudaMemsetAsync(e, 0, m->nv * sizeof(double), s));
        UCK(launch_unit(e, (size_t)fidx[j], s));
        UCK(uglobal_apply<double>(m, k1, e, cols + (size_t)j * m->nv, Y1, s));
      }
      UCK(m->alloc(&A, (size_t)m->nf1 * m->nf1));
      UCK(launch_gather_coarse(cols, m->freeidx1, m->nf1, (size_t)m->nv, A, s));
      UCU(cudaStreamSynchronize(s));
      cudaFree(cols);
      cudaFree(e);
      cudaFree(Y1);
      std::string cmsg;
      const int st = coarse_inverse(A, m->nf1, s, &cmsg);
      if (st) {
        *msg = "Q1 coarse factorisation: " + cmsg;
        return st;
      }
      m->Ainv = A;
      (void)L1;
    }
  }
  UCU(cudaStreamSynchronize(s));
  return ST_OK;
}

// ---- queries
int64_t umesh_ndofs(const UMesh* m) { return m->L[0].ndofs; }
int64_t umesh_nfree(const UMesh* m) {
  int64_t n = 0;
  for (uint8_t b : m->L[0].h_bnd) n += !b;
  return n;
}
int64_t umesh_npatch(const UMesh* m) { return (int64_t)m->pverts.size(); }
int umesh_ncolours(const UMesh* m) { return m->ncolours; }
int umesh_nplevels(const UMesh* m, int* q) {
  for (int k = 0; k < m->npl; ++k) q[k] = m->L[k].q;
  return m->npl;
}
int64_t umesh_kernel_launches(const UMesh* m) { return m->launches; }
int64_t umesh_interior_max(const UMesh* m) { return m->L[0].nimax; }
int umesh_max_valence(const UMesh* m) {
  int v = 0;
  for (const auto& c : m->pcells) v = std::max(v, (int)c.size());
  return v;
}
int umesh_cell_dofs(const UMesh* m, int k, int32_t* out) {
  if (k < 0 || k >= m->npl) return ST_ARG;
  std::copy(m->L[k].h_cdofs.begin(), m->L[k].h_cdofs.end(), out);
  return ST_OK;
}
int umesh_patches(const UMesh* m, int64_t* out, int width) {
  for (size_t j = 0; j < m->pverts.size(); ++j) {
    out[j * width] = m->pverts[j];
    for (int i = 1; i < width; ++i) out[j * width + i] = i - 1 < (int)m->pcells[j].size() ? m->pcells[j][i - 1] : -1;
  }
  return ST_OK;
}
int umesh_colours(const UMesh* m, uint8_t* out) {
  std::copy(m->colour.begin(), m->colour.end(), out);
  return ST_OK;
}
int umesh_get_bounds(const UMesh* m, int k, double* out) {
  if (k < 0 || k >= m->npl) return ST_ARG;
  return cudaMemcpy(out, m->L[k].bounds64, m->pverts.size() * 2 * sizeof(double), cudaMemcpyDeviceToHost) ==
                 cudaSuccess
             ? ST_OK
             : ST_CUDA;
}
int umesh_set_bounds(UMesh* m, int k, const double* lohi) {
  if (k < 0 || k >= m->npl) return ST_ARG;
  const size_t n = m->pverts.size() * 2;
  std::vector<float> f(lohi, lohi + n);
  if (cudaMemcpy(m->L[k].bounds64, lohi, n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) return ST_CUDA;
  if (cudaMemcpy(m->L[k].bounds32, f.data(), n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) return ST_CUDA;
  return ST_OK;
}

// ---- operations (FP64 interfaces; mixed precision casts to FP32 inside)
int umesh_mask(UMesh* m, double* x, cudaStream_t s) {
  k_umask<double><<<grid_for((size_t)m->L[0].ndofs, 256), 256, 0, s>>>(x, m->L[0].bnd, m->L[0].ndofs);
  ++m->launches;
  return cudaPeekAtLastError() == cudaSuccess ? ST_OK : ST_CUDA;
}

int umesh_apply(UMesh* m, const double* u, double* Au, cudaStream_t s) {
  return uglobal_apply<double>(m, 0, u, Au, m->Y64, s);
}

int umesh_sweep_colour(UMesh* m, int colour, const double* b, double* u, cudaStream_t s) {
  if (colour < 0 || colour >= m->ncolours) return ST_ARG;
  if (m->opt.precision == PMG_PREC_MIXED) {
    const size_t n = (size_t)m->L[0].ndofs;
    UCK(launch_cast_d2f(b, m->b32, n, s));
    UCK(launch_cast_d2f(u, m->x32, n, s));
    UCK(usweep_colour_T<float>(m, colour, m->b32, m->x32, s));
    UCK(launch_cast_f2d(m->x32, u, n, s));
    m->launches += 3;
    return ST_OK;
  }
  return usweep_colour_T<double>(m, colour, b, u, s);
}

int umesh_sweep(UMesh* m, const double* b, double* u, int n_sweeps, bool reverse, cudaStream_t s) {
  const size_t n = (size_t)m->L[0].ndofs;
  const bool mixed = m->opt.precision == PMG_PREC_MIXED;
  if (mixed) {
    UCK(launch_cast_d2f(b, m->b32, n, s));
    UCK(launch_cast_d2f(u, m->x32, n, s));
    m->launches += 2;
  }
  for (int i = 0; i < n_sweeps; ++i) {
    if (mixed) UCK(usweep_T<float>(m, m->b32, m->x32, reverse, s));
    else UCK(usweep_T<double>(m, b, u, reverse, s));
  }
  if (mixed) {
    UCK(launch_cast_f2d(m->x32, u, n, s));
    ++m->launches;
  }
  return ST_OK;
}

template <typename T>
static int ulocal_T(UMesh* m, int64_t n, const int64_t* ids, const T* r, T* d, cudaStream_t s) {
  UPatchArgs<T> a;
  fill_args(m, a);
  a.n_items = (int)n;
  a.ids64 = ids;
  a.r_in = r;
  a.d_out = d;
  const int grid = (int)std::min<int64_t>(n, m->ws_grid);
  ++m->launches;
  return m->dim == 2 ? upatch_launch<2, T>(m->p, MODE_LOCAL, a, grid, s)
                     : upatch_launch<3, T>(m->p, MODE_LOCAL, a, grid, s);
}

int umesh_local(UMesh* m, int64_t n, const int64_t* ids, const double* r, double* d, int n_cycles,
                cudaStream_t s) {
  if (n <= 0) return ST_OK;
  const int saved = m->opt.n_mg;
  m->opt.n_mg = n_cycles;
  int st;
  if (m->opt.precision == PMG_PREC_MIXED) {
    const size_t len = (size_t)n * m->L[0].nimax;
    float *r32 = nullptr, *d32 = nullptr;
    if (cudaMalloc(&r32, len * sizeof(float)) != cudaSuccess) return ST_CUDA;
    if (cudaMalloc(&d32, len * sizeof(float)) != cudaSuccess) {
      cudaFree(r32);
      return ST_CUDA;
    }
    st = launch_cast_d2f(r, r32, len, s);
    if (!st) st = ulocal_T<float>(m, n, ids, r32, d32, s);
    if (!st) st = launch_cast_f2d(d32, d, len, s);
    cudaStreamSynchronize(s);
    cudaFree(r32);
    cudaFree(d32);
  } else {
    st = ulocal_T<double>(m, n, ids, r, d, s);
  }
  m->opt.n_mg = saved;
  return st;
}

// two-level V-cycle in precision T: x = B b
template <typename T>
static int uvcycle_T(UMesh* m, const T* b, T* x, T* r, T* Y, T* r1, T* x1, cudaStream_t s) {
  const ULevelD& L0 = m->L[0];
  const size_t n = (size_t)L0.ndofs;
  UCK(launch_fill<T>(x, n, T(0), s));
  UCK(usweep_T<T>(m, b, x, false, s));                     // pre-smoothing
  UCK(uglobal_apply<T>(m, 0, x, r, Y, s));                  // r = b - A x
  UCK(launch_sub_from<T>(b, r, n, s));
  if (m->nf1 > 0) {
    const int d = m->dim;
    if (d == 2)
      k_uq1_restrict_cells<2, T><<<grid_for((size_t)m->nc * 4, 256), 256, 0, s>>>(r, L0.cdofs, L0.dstart, L0.bnd,
                                                                                  m->nc, L0.q, Y);
    else
      k_uq1_restrict_cells<3, T><<<grid_for((size_t)m->nc * 8, 256), 256, 0, s>>>(r, L0.cdofs, L0.dstart, L0.bnd,
                                                                                  m->nc, L0.q, Y);
    k_uassemble<T><<<grid_for((size_t)m->nv, 256), 256, 0, s>>>(Y, m->vstart, m->vlist, m->vbnd, m->nv, r1);
    UCK(launch_fill<T>(x1, (size_t)m->nv, T(0), s));
    UCK(launch_coarse_gemv<T>(m->Ainv, m->freeidx1, m->nf1, r1, x1, s));
    if (d == 2)
      k_uq1_prolong<2, T><<<grid_for(n, 256), 256, 0, s>>>(x1, m->cells, L0.dstart, L0.dlist, L0.bnd, m->vbnd,
                                                           L0.ndofs, L0.q, r);
    else
      k_uq1_prolong<3, T><<<grid_for(n, 256), 256, 0, s>>>(x1, m->cells, L0.dstart, L0.dlist, L0.bnd, m->vbnd,
                                                           L0.ndofs, L0.q, r);
    UCU(cudaPeekAtLastError());
    UCK(launch_add_to<T>(r, x, n, s));
    m->launches += 6;
  }
  return usweep_T<T>(m, b, x, true, s);                     // post-smoothing, colours reversed
}

int umesh_precondition(UMesh* m, const double* r, double* z, cudaStream_t s) {
  const size_t n = (size_t)m->L[0].ndofs;
  if (m->opt.precision == PMG_PREC_MIXED) {
    UCK(launch_cast_d2f(r, m->b32, n, s));
    UCK(uvcycle_T<float>(m, m->b32, m->x32, m->r32, m->Y32, m->r1_32, m->x1_32, s));
    UCK(launch_cast_f2d(m->x32, z, n, s));
    m->launches += 2;
    return ST_OK;
  }
  UCU(cudaMemcpyAsync(m->b64, r, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  UCK(uvcycle_T<double>(m, m->b64, m->x64, m->r64, m->Y64, m->r1_64, m->x1_64, s));
  UCU(cudaMemcpyAsync(z, m->x64, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return ST_OK;
}

}  // namespace pmg
