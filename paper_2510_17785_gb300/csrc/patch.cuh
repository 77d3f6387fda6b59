// Vertex-patch smoother with the nested p-multigrid local solver.
//
// Paper Section 2.1 and Algorithm 1: for each patch j (the 2^d cells around
// an interior vertex), Gather u and b (eq. gather), Evaluate the local
// residual r_j = b_j - Pi_j A_j-bar u_j (eq. main:4), Solve d_j ~ A_j^-1 r_j
// (eq. main:5) and Scatter u += Pi_j^T d_j (eq. scatter).  Section 3 and
// Algorithm 2: the local solve is a V-cycle over p-levels p, p/2, ..., 1 with a
// smoother on each level (damped Jacobi, or Chebyshev iteration on D^-1 A),
// p-restriction/prolongation by 1D interpolation matrices applied per
// direction, and the exact 1x1 solve on p = 1.
//
// GPU mapping: one CTA handles PPB patches of one colour (patches of one
// colour share no cell, so their interior DoF sets are disjoint and the
// in-place scatter is race-free).  Every vector of every p-level lives in
// shared memory; the operator is the sum-factorised block apply of sf.cuh on
// the 2^d-cell patch, with the per-point geometry tensors G read from global
// memory (L1/L2 resident across the applies of one patch).
#pragma once
#include "../../include/pmg.h"
#include "sf.cuh"

namespace pmg {

enum { MODE_SWEEP = 0, MODE_LOCAL = 1 };

__host__ __device__ constexpr int nlevels(int P) { return P <= 1 ? 1 : 1 + nlevels(P >> 1); }

template <typename T>
struct LevelArgs {
  const T* G;          // geometry tensors of degree q: [cells][ncomp][(q+1)^d]
  const unsigned* Gb;  // FP32 kernels: the same tensors as BF16 pairs, [cells][(ncomp+1)/2][(q+1)^d]
                       // (component 2j in the low half of a word, 2j + 1 in the high half), or NULL
  const T* dinv;       // 1 / diag(A_q) on the global degree-q grid, 0 on Dirichlet
  const T* bounds;     // [patches][2]: Chebyshev interval (lo, hi), q > 1
  const T* dense;      // small levels: [patches][Ni][Ni] row-major patch matrix A_{j,q}
  const T* fdm;        // Cartesian-reinforced smoother: reference-patch fast-diagonalisation table of
                       // degree q, [S: Mi x Mi][lambda: Mi][diag K: Mi][diag M: Mi], Mi = 2q - 1
};

// Levels whose patch operator is small enough to be applied as a dense
// matrix (Ni <= 64: q <= 2 in 3D, q <= 4 in 2D; never the p = 1 level).
__host__ __device__ constexpr bool dense_level(int dim, int q) {
  return q > 1 && (dim == 3 ? (2 * q - 1) * (2 * q - 1) * (2 * q - 1) : (2 * q - 1) * (2 * q - 1)) <= 64;
}

template <typename T>
struct PatchArgs {
  int N;                       // cells per direction
  int n_items;                 // patches handled by this launch
  const int32_t* list;         // patch ids (this colour), or NULL: item i = patch ids_dev[i]
  const int64_t* ids64;        // patch ids for MODE_LOCAL
  LevelArgs<T> lv[8];
  T* u;                        // MODE_SWEEP: degree-p global vector, updated in place
  const T* b;                  // MODE_SWEEP: right-hand side
  const T* r_in;               // MODE_LOCAL: [n_items][Ni]
  T* d_out;                    // MODE_LOCAL: [n_items][Ni]
  int smoother;                // 0 Chebyshev, 1 Jacobi, 2 Cartesian-reinforced
  int cheb_degree;
  double omega;
  int n_mg;
  int* err;                    // device error flag
  T* corr;                     // additive sweep: corrections are added here instead of to u, or NULL
  int weight_residual;         // additive sweep, transposed form: residual scaled by 1 / multiplicity
  const T* solveop;            // tabulated local solve: [patches][Ni][Ni], entry (m, k) = (B_j e_m)_k, or NULL
  int unit_rhs;                // MODE_LOCAL: item i solves patch i / Ni with right-hand side e_(i mod Ni)
};


// Epilogues of the patch operator applies: the smoother and residual updates
// applied to each output value as it is produced (no extra pass over Ad).
enum { EPI_STORE = 0, EPI_RESID, EPI_EVAL, EPI_CHEB0, EPI_CHEB, EPI_JAC };

template <typename T>
struct PatchEpi {
  T* sm;
  int PS;
  int kind;
  int r, d, res, dir, dinv, ad, coef, it;
  T omega;
  // the patch arrays start at the kernel's dynamic shared memory
  __device__ __forceinline__ PatchEpi rebase() const {
    PatchEpi e = *this;
    e.sm = reinterpret_cast<T*>(pmg_smem);
    return e;
  }
  __device__ __forceinline__ void operator()(int pp, int i, T s) const {
    T* b = sm + pp * PS;
    switch (kind) {
      case EPI_STORE: b[ad + i] = s; break;
      case EPI_RESID: b[res + i] = b[r + i] - s; break;          // res = r - A d
      case EPI_EVAL: b[r + i] -= s; break;                       // r = b - A u
      case EPI_CHEB0: {                                          // first step from d != 0
        const T rs = b[dinv + i] * (b[r + i] - s);
        const T dr = rs * b[coef];
        b[res + i] = rs;
        b[dir + i] = dr;
        b[d + i] += dr;
        break;
      }
      case EPI_CHEB: {                                           // step it of the recurrence
        const T rs = b[res + i] - b[dinv + i] * s;
        const T dr = b[coef + it] * b[dir + i] + b[coef + 7 + it] * rs;
        b[res + i] = rs;
        b[dir + i] = dr;
        b[d + i] += dr;
        break;
      }
      default: b[d + i] += omega * b[dinv + i] * (b[r + i] - s);  // damped Jacobi
    }
  }
};

// per-patch shared-memory layout (ES-byte elements)
template <int DIM, int P, int ES, bool LINE = false, bool GSMEM = false, int LR = 0>
struct Layout {
  static constexpr int NL = nlevels_rule(P, LR);
  __host__ __device__ static constexpr int q(int k) { return level_degree(P, LR, k); }
  __host__ __device__ static constexpr int ni(int k) { return q(k) == 1 ? 1 : ipow(2 * q(k) - 1, DIM); }
  // per-level vectors r, d, res, dir, [A x: dense levels only], 1/diag
  __host__ __device__ static constexpr bool dn(int k) { return dense_level(DIM, q(k)); }
  __host__ __device__ static constexpr int lb(int k) { return q(k) == 1 ? 4 : (dn(k) ? 6 : 5) * ni(k); }
  __host__ __device__ static constexpr int off(int k) { return k == 0 ? 0 : off(k - 1) + lb(k - 1); }
  __host__ __device__ static constexpr int R_(int k) { return off(k); }
  __host__ __device__ static constexpr int D_(int k) { return off(k) + ni(k); }
  __host__ __device__ static constexpr int RES(int k) { return off(k) + 2 * ni(k); }
  __host__ __device__ static constexpr int DIR(int k) { return off(k) + 3 * ni(k); }
  // A x of a dense level (the matrix-free levels hand every value to an epilogue instead)
  __host__ __device__ static constexpr int AD(int k) { return q(k) == 1 ? off(k) + 3 : off(k) + 4 * ni(k); }
  __host__ __device__ static constexpr int DINV(int k) {
    return q(k) == 1 ? off(k) + 2 : off(k) + (dn(k) ? 5 : 4) * ni(k);
  }
  // dense patch matrices of the small levels, staged per patch
  __host__ __device__ static constexpr int dsz(int k) { return dense_level(DIM, q(k)) ? ni(k) * ni(k) : 0; }
  __host__ __device__ static constexpr int doff(int k) { return k == 0 ? off(NL) : doff(k - 1) + dsz(k - 1); }
  __host__ __device__ static constexpr int DENSE(int k) { return doff(k); }
  // closure of u for Evaluate: it is read before d, res and dir of the top
  // level are first written, so it shares their storage when it fits there
  static constexpr int NN0 = ipow(2 * P + 1, DIM);
  static constexpr bool CLOS_SHARED = q(0) > 1 && !dn(0) && NN0 <= 3 * ni(0);
  static constexpr int CLOS = CLOS_SHARED ? D_(0) : doff(NL);
  static constexpr int SCR = CLOS_SHARED ? doff(NL) : doff(NL) + NN0;
  static constexpr int SCRATCH = LINE ? Dims<DIM, 2, P, ES>::SCRATCH_LINE : Dims<DIM, 2, P, ES>::SCRATCH;
  static constexpr int COEF = SCR + SCRATCH;      // per level: 1/theta, c1[1..7], c2[1..7]
  static constexpr int NCOEF = 16;
  // (the fast-diagonalisation tables of the Cartesian-reinforced smoother are
  // the same for every patch and are read from global memory)
  __host__ __device__ static constexpr int mi(int k) { return 2 * q(k) - 1; }
  static constexpr int END = COEF + NL * NCOEF;
  // geometry tensors of the patch's 2^d cells at the top degree, staged once
  // per patch (latency-oriented launch shapes): [cell slot][ncomp][(p+1)^d]
  static constexpr int GCELL = (DIM * (DIM + 1) / 2) * ipow(P + 1, DIM);
  static constexpr int GS = (END + 3) & ~3;
  static constexpr int PS_RAW = GSMEM ? GS + (1 << DIM) * GCELL : END;
  static constexpr int PS = (PS_RAW + 3) & ~3;    // per-patch stride in elements
};

// Launch shape of the patch kernel.  Variant 0 is the default; for 3D degrees
// 3..8 the set-up autotuner also times variants 1..9:
//   variant:          1     2     3     4     5     6     7     8     9    10    11    12    13    14    15
//   design:         stage stage stage line  line  line  line  line  stage line  line  line  line  line  line
//   threads / CTA:    256   128   512   256   128   512   128   256   256   224   320   416   192   256   128
//   patches / CTA:      2     1     1     2     1     1     2     2     2     2     3     4     3     4     4
//   geometry:                  staged            staged       staged staged
//   groups:                                               2                             3     4     4
// (patches per CTA are capped by shared memory).  "stage": every direction's
// flux in shared memory; "line": one thread per line along the last
// direction keeps that direction's gradient and flux in registers.  With
// groups, each patch of the CTA has its own threads and barrier.  "staged":
// the top level's geometry tensors are copied to shared memory once per
// patch instead of read from L2 by every apply; variants 3 and 6 are
// latency-oriented shapes for small launches (coarse mesh levels, one patch
// per 512 threads), 8 and 9 throughput shapes (two patches per 256 threads,
// a 128-register budget, two CTAs per SM).  Variants 10-12 size the CTA to
// about 100 threads per patch, the number of lines along the last direction
// at degree 4 (fewer idle threads at each barrier).  Variants 13-15 give each
// patch its own team of 64 or 32 threads (one or two warps) with its own
// barrier and several lines per thread (more independent work per thread,
// no waiting on the other patches of the CTA).
constexpr int NUM_VARIANTS = PMG_NUM_VARIANTS;
// the default launch shape with the paper's p-level rule (options.level_rule =
// 1); never chosen by the autotuner, which times launch shapes only
constexpr int VARIANT_PAPER_LEVELS = NUM_VARIANTS;

template <int DIM, int P, typename T, int V = 0>
struct Config {
  static constexpr int NT0 = (DIM == 3) ? 256 : 128;
  static constexpr int PPB0 = (DIM == 3) ? (P <= 2 ? 4 : 1) : (P <= 2 ? 8 : (P <= 4 ? 4 : 2));
  static constexpr int NTV[NUM_VARIANTS] = {NT0, 256, 128, 512, 256, 128, 512, 128, 256, 256, 224, 320, 416,
                                            192, 256, 128};
  static constexpr int PPBV[NUM_VARIANTS] = {PPB0, 2, 1, 1, 2, 1, 1, 2, 2, 2, 2, 3, 4, 3, 4, 4};
  static constexpr bool LINEV[NUM_VARIANTS] = {false, false, false, false, true, true, true, true, true, false,
                                               true, true, true, true, true, true};
  static constexpr bool GROUPV[NUM_VARIANTS] = {false, false, false, false, false, false, false, true, false, false,
                                                false, false, false, true, true, true};
  static constexpr bool GSMEMV[NUM_VARIANTS] = {false, false, false, true, false, false, true, false, true, true,
                                                false, false, false, false, false, false};
  // variant VARIANT_PAPER_LEVELS: the default shape with the paper's p-level rule
  static constexpr int VB = V == VARIANT_PAPER_LEVELS ? 0 : V;
  static constexpr int LR = V == VARIANT_PAPER_LEVELS ? 1 : 0;
  static constexpr int NT = NTV[VB];
  static constexpr int PPB_MAX = PPBV[VB];
  static constexpr bool LINE = LINEV[VB];
  static constexpr bool GSMEM = GSMEMV[VB];
  static constexpr size_t bytes_per_patch =
      sizeof(T) * Layout<DIM, P, (int)sizeof(T), LINE, GSMEM, LR>::PS + sizeof(int) * ((1 << DIM) + 6);
  static constexpr size_t SMEM_LIMIT = 227 * 1024;
  static constexpr int PPB_FIT = (int)(SMEM_LIMIT / bytes_per_patch);
  static constexpr int PPB = PPB_FIT < PPB_MAX ? (PPB_FIT < 1 ? 1 : PPB_FIT) : PPB_MAX;
  static constexpr size_t smem = bytes_per_patch * PPB;
  static constexpr bool fits = bytes_per_patch <= SMEM_LIMIT;
  // grouped only when the CTA really holds several patches
  static constexpr bool GROUPED = GROUPV[VB] && PPB > 1 && NT % PPB == 0 && (NT / PPB) % 32 == 0;
  // register budget per thread (launch bound): 64 for FP32 up to degree 5,
  // 128 otherwise (FP64, or the larger line registers at high degree)
  static constexpr int REG_TARGET = (sizeof(T) == 4 && P <= 5 && !GSMEMV[VB]) ? 64 : 128;
  // resident CTAs per SM: by the register target, and at most what shared
  // memory allows (small CTAs then get the registers shared memory leaves)
  static constexpr int MINB_REG_RAW = 65536 / (NT * REG_TARGET);
  static constexpr int MINB_REG = MINB_REG_RAW < 1 ? 1 : MINB_REG_RAW;
  static constexpr int MINB_SMEM = (int)((228 * 1024) / (smem + 1024));
  static constexpr int MINB_RAW = MINB_REG < MINB_SMEM ? MINB_REG : MINB_SMEM;
  static constexpr int MINB = MINB_RAW < 1 ? 1 : MINB_RAW;
  // a variant exists (is worth instantiating) if it fits and differs from
  // every lower-numbered variant
  template <int W>
  static constexpr bool same_as() {
    return Config<DIM, P, T, W>::NT == NT && Config<DIM, P, T, W>::PPB == PPB && Config<DIM, P, T, W>::LINE == LINE &&
           Config<DIM, P, T, W>::GROUPED == GROUPED && Config<DIM, P, T, W>::GSMEM == GSMEM;
  }
  template <int W>
  static constexpr bool distinct_from_lower() {
    if constexpr (W >= V) return true;
    else return !same_as<W>() && distinct_from_lower<W + 1>();
  }
  static constexpr bool distinct_impl() {
    if constexpr (V == VARIANT_PAPER_LEVELS) return rules_differ(P);   // exists where the rules differ
    else return distinct_from_lower<0>();
  }
  static constexpr bool distinct = distinct_impl();
  // worth compiling: a line variant keeps at most two lines' gradients and
  // fluxes per thread in registers (more spills and bloats the build); FP64,
  // bound by the FP64 FMA rate, keeps variants 0, 2, 4 and 6, and only 0 from
  // degree 7 on
  static constexpr int QPL = 2 * (P + 1);
  static constexpr int TPP_ = GROUPED ? NT / PPB : NT;
  static constexpr int SPAN_ = GROUPED ? 1 : PPB;
  static constexpr int LPT_ = (SPAN_ * ipow(QPL, DIM - 1) + TPP_ - 1) / TPP_;
  static constexpr bool worth = (!LINE || LPT_ <= (GROUPED ? 4 : 2)) &&
                                (sizeof(T) == 4 || VB == 0 || ((VB == 2 || VB == 4 || VB == 6) && P <= 6)) &&
                                (VB < 8 || (DIM == 3 && P >= 3)) &&
                                (VB < 10 || (sizeof(T) == 4 && (VB >= 13 || P <= 5)));
  static constexpr bool exists = fits && distinct && worth;
};

template <int DIM, int P, typename T, int MODE, int V = 0>
struct PatchKernel {
  using C = Config<DIM, P, T, V>;
  using L = Layout<DIM, P, (int)sizeof(T), C::LINE, C::GSMEM, C::LR>;
  using TM = Team<C::NT, C::PPB, C::GROUPED>;
  static constexpr int NT = C::NT, PPB = C::PPB, NL = L::NL, PS = L::PS;
  static constexpr int NCELL = 1 << DIM;

  T* sm;           // per-patch arrays, stride PS
  int* cells;      // [PPB][CST]: global cell ids, patch id, active flag, vertex indices (v_x, v_y, v_z)
  static constexpr int CST = NCELL + 6;
  const PatchArgs<T>* a;
  const int32_t* list;   // patch ids of the colour being swept (MODE_SWEEP)
  int n_items;           // patches of this launch (or of the colour, persistent launches)
  int blk;               // batch of PPB patches this CTA works on
  bool coherent = false; // u changes during the launch (persistent sweeps): read it through L2

  __device__ T* vec(int pp, int off) const { return sm + pp * PS + off; }

  // Shared-memory staging of global data: every thread issues the loads of
  // U items before it stores any of them, so U loads are in flight per thread
  // (one at a time, each staging pass is a chain of memory round trips).
  // ld(pp, item) loads, st(pp, item, value) stores.
  template <int ITEMS, typename LD, typename STF>
  __device__ __forceinline__ void stage(LD&& ld, STF&& st) const {
    constexpr int U = 8;
    constexpr int TOT = TM::SPAN * ITEMS;
#pragma unroll 1
    for (int base = TM::lane(); base < TOT; base += U * TM::TPP) {
      T v[U];
      int pp[U], e[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int it = base + u * TM::TPP;
        if constexpr (C::GROUPED) {
          pp[u] = TM::group();
          e[u] = it;
        } else {
          pp[u] = it / ITEMS;
          e[u] = it - pp[u] * ITEMS;
        }
        v[u] = it < TOT ? ld(pp[u], e[u]) : T(0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (base + u * TM::TPP < TOT) st(pp[u], e[u], v[u]);
    }
  }

  // geometry of cell `slot` of patch pp staged in shared memory (GSMEM variants)
  template <int stride>
  struct SharedGeom {
    static constexpr bool kShared = true;
    __device__ const T* operator()(int pp, int slot) const {
      return reinterpret_cast<const T*>(pmg_smem) + L::GS + pp * PS + slot * stride;
    }
  };

  // geometry of cell `slot` of patch pp in global memory: FP32/FP64 tensors,
  // or (FP32, when the level has them) the packed BF16 pairs, one word per
  // pair addressed like an FP32 value
  template <int stride, int pstride>
  struct GlobalGeom {
    static constexpr bool kPackable = sizeof(T) == 4;
    const T* G;
    bool packed;
    __device__ const T* operator()(int pp, int slot) const {
      // the cell list follows the PPB patch arrays in dynamic shared memory
      const int* cl = reinterpret_cast<const int*>(pmg_smem + sizeof(T) * (size_t)PS * PPB);
      return G + (size_t)cl[pp * CST + slot] * (packed ? pstride : stride);
    }
  };

  template <int K>
  __device__ auto gfun() const {
    constexpr int q = L::q(K);
    using Dq = Dims<DIM, 2, q, (int)sizeof(T)>;
    constexpr int stride = Dq::NCOMP * Dq::NGC;
    if constexpr (C::GSMEM && K == 0) {                 // staged in shared memory by load_level
      return SharedGeom<stride>{};
    } else {
      const bool packed = sizeof(T) == 4 && a->lv[K].Gb != nullptr;
      const T* G = packed ? reinterpret_cast<const T*>(a->lv[K].Gb) : a->lv[K].G;
      return GlobalGeom<stride, ((Dq::NCOMP + 1) / 2) * Dq::NGC>{G, packed};
    }
  }

  template <int K>
  __device__ PatchEpi<T> epi(int kind, int it = 0) const {
    PatchEpi<T> e;
    e.sm = sm;
    e.PS = PS;
    e.kind = kind;
    e.r = L::R_(K);
    e.d = L::D_(K);
    e.res = L::RES(K);
    e.dir = L::DIR(K);
    e.dinv = L::DINV(K);
    e.ad = L::AD(K);
    e.coef = L::COEF + K * L::NCOEF;
    e.it = it;
    e.omega = T(a->omega);
    return e;
  }

  // A_q x on the interior vector at in_off of level K, every output value
  // passed through the epilogue `e` (matrix-free, or the staged dense patch
  // matrix on small levels).  Ends with a barrier.
  template <int K>
  __device__ void apply_int(int in_off, const PatchEpi<T>& e) {
    constexpr int q = L::q(K);
    if constexpr (dense_level(DIM, q)) {
      // the epilogue may overwrite the input, which other rows still read:
      // products first, epilogue after a barrier
      constexpr int NI = L::ni(K);
      TM::template loop<NI>([&](int pp, int r) {
        const T* A = vec(pp, L::DENSE(K)) + r * NI;
        const T* x = vec(pp, in_off);
        T s = T(0);
#pragma unroll
        for (int c = 0; c < NI; ++c) s += A[c] * x[c];
        vec(pp, L::AD(K))[r] = s;
      });
      TM::sync();
      if (e.kind != EPI_STORE) {
        TM::template loop<NI>([&](int pp, int r) { e(pp, r, vec(pp, L::AD(K))[r]); });
        TM::sync();
      }
    } else {
      static_assert(sf_scratch(DIM, 2, q, C::LINE, (int)sizeof(T)) <= L::SCRATCH, "level scratch exceeds the top level's");
      SF<DIM, 2, q, T, NT, PPB, C::LINE, C::GROUPED>::template apply_epi<true>(vec(0, in_off), PS, vec(0, L::SCR), PS,
                                                                  gfun<K>(), e);
    }
  }

  // ---- p-transfers between level K (degree qf) and K+1 (degree qc = qf/2)
  // Prolongation along axis AX on interior nodes: [O][Mc][I] -> [O][Mf][I]
  template <int K, int AX, bool ACC>
  __device__ static void prol_item(const T* __restrict__ in, T* __restrict__ out, int item, int Mc, int Mf,
                                   int I, int O) {
    constexpr int qf = L::q(K), qc = L::q(K + 1);
    const int OI = O * I;
    const int c = item >= OI, pi = item - c * OI;
    const int i = pi % I, o = pi / I;
    const T* src = in + o * Mc * I + i;
    T* dst = out + o * Mf * I + i;
    T v[qc + 1];
#pragma unroll
    for (int b = 0; b <= qc; ++b) {
      const int kc = qc * c + b;
      v[b] = (kc >= 1 && kc <= 2 * qc - 1) ? src[(kc - 1) * I] : T(0);
    }
    const int amax = (c == 0) ? qf : qf - 1;
#pragma unroll
    for (int a = 1; a <= qf; ++a) {
      if (a > amax) break;
      T s = T(0);
#pragma unroll
      for (int b = 0; b <= qc; ++b) s += tabT<T, C::LR>(qf, a, b) * v[b];
      const int kf = qf * c + a;
      T* p = dst + (kf - 1) * I;
      *p = ACC ? *p + s : s;
    }
  }

  // Restriction (transpose) along axis AX: [O][Mf][I] -> [O][Mc][I]
  template <int K>
  __device__ static void rest_item(const T* __restrict__ in, T* __restrict__ out, int item, int Mc, int Mf,
                                   int I, int O) {
    constexpr int qf = L::q(K), qc = L::q(K + 1);
    const int OI = O * I;
    const int c = item >= OI, pi = item - c * OI;
    const int i = pi % I, o = pi / I;
    const T* src = in + o * Mf * I + i;
    T* dst = out + o * Mc * I + i;
    T f[qf];
    // fine nodes defined by cell c: c = 0 -> k_f = 1..qf, c = 1 -> k_f = qf+1..2qf-1
#pragma unroll
    for (int a = 1; a <= qf; ++a) {
      const int kf = qf * c + a;
      f[a - 1] = (kf <= 2 * qf - 1) ? src[(kf - 1) * I] : T(0);
    }
    if (c == 0) {
      T w[qf];
#pragma unroll
      for (int a = 1; a < qf; ++a) w[a - 1] = src[(qf + a - 1) * I];
#pragma unroll
      for (int b = 1; b <= qc; ++b) {
        T s = T(0);
#pragma unroll
        for (int a = 1; a <= qf; ++a) s += tabT<T, C::LR>(qf, a, b) * f[a - 1];
        if (b == qc) {
#pragma unroll
          for (int a = 1; a < qf; ++a) s += tabT<T, C::LR>(qf, a, 0) * w[a - 1];
        }
        dst[(b - 1) * I] = s;
      }
    } else {
#pragma unroll
      for (int b = 1; b < qc; ++b) {
        T s = T(0);
#pragma unroll
        for (int a = 1; a < qf; ++a) s += tabT<T, C::LR>(qf, a, b) * f[a - 1];
        dst[(qc + b - 1) * I] = s;
      }
    }
  }

  // r_{K+1} = E^T res_K
  template <int K>
  __device__ void restrict_res() {
    constexpr int qf = L::q(K), qc = L::q(K + 1);
    constexpr int Mf = 2 * qf - 1, Mc = (qc == 1) ? 1 : 2 * qc - 1;
    T* t = vec(0, L::SCR);
    if constexpr (DIM == 3) {
      TM::template loop<Mf * Mf * 2>([&](int pp, int it) {
        rest_item<K>(vec(pp, L::RES(K)), t + pp * PS, it, Mc, Mf, 1, Mf * Mf);
      });
      TM::sync();
      TM::template loop<Mf * Mc * 2>([&](int pp, int it) {
        rest_item<K>(t + pp * PS, t + pp * PS + Mf * Mf * Mc, it, Mc, Mf, Mc, Mf);
      });
      TM::sync();
      TM::template loop<Mc * Mc * 2>([&](int pp, int it) {
        rest_item<K>(t + pp * PS + Mf * Mf * Mc, vec(pp, L::R_(K + 1)), it, Mc, Mf, Mc * Mc, 1);
      });
      TM::sync();
    } else {
      TM::template loop<Mf * 2>([&](int pp, int it) { rest_item<K>(vec(pp, L::RES(K)), t + pp * PS, it, Mc, Mf, 1, Mf); });
      TM::sync();
      TM::template loop<Mc * 2>([&](int pp, int it) {
        rest_item<K>(t + pp * PS, vec(pp, L::R_(K + 1)), it, Mc, Mf, Mc, 1);
      });
      TM::sync();
    }
  }

  // d_K += E d_{K+1}
  template <int K>
  __device__ void prolong_add() {
    constexpr int qf = L::q(K), qc = L::q(K + 1);
    constexpr int Mf = 2 * qf - 1, Mc = (qc == 1) ? 1 : 2 * qc - 1;
    T* t = vec(0, L::SCR);
    if constexpr (DIM == 3) {
      TM::template loop<Mc * Mc * 2>([&](int pp, int it) {
        prol_item<K, 0, false>(vec(pp, L::D_(K + 1)), t + pp * PS, it, Mc, Mf, 1, Mc * Mc);
      });
      TM::sync();
      TM::template loop<Mc * Mf * 2>([&](int pp, int it) {
        prol_item<K, 1, false>(t + pp * PS, t + pp * PS + Mc * Mc * Mf, it, Mc, Mf, Mf, Mc);
      });
      TM::sync();
      TM::template loop<Mf * Mf * 2>([&](int pp, int it) {
        prol_item<K, 2, true>(t + pp * PS + Mc * Mc * Mf, vec(pp, L::D_(K)), it, Mc, Mf, Mf * Mf, 1);
      });
      TM::sync();
    } else {
      TM::template loop<Mc * 2>([&](int pp, int it) {
        prol_item<K, 0, false>(vec(pp, L::D_(K + 1)), t + pp * PS, it, Mc, Mf, 1, Mc);
      });
      TM::sync();
      TM::template loop<Mf * 2>([&](int pp, int it) {
        prol_item<K, 1, true>(t + pp * PS, vec(pp, L::D_(K)), it, Mc, Mf, Mf, 1);
      });
      TM::sync();
    }
  }

  // ---- Cartesian-reinforced step (Section 3.1):
  // d <- d + omega diag(A_j)^-1 diag(A_b) A_b^-1 (r - A_j d), with the reference
  // Cartesian patch operator A_b = sum over axes of K (x) M (x) M (permuted)
  // inverted by fast diagonalisation: with S^T M S = I and S^T K S = Lambda,
  // A_b^-1 = (S (x) S (x) S) (Lambda_x + Lambda_y + Lambda_z)^-1 (S (x) S (x) S)^T.
  // Stages: S^T along x, y; along z S^T, the eigenvalue scaling and S in one
  // thread per line; S along y; S along x with the update of d.
  template <int K, int AX, bool BACK>
  __device__ static void fdm_line(const T* __restrict__ Sm, const T* __restrict__ in, T* __restrict__ out, int line) {
    constexpr int Mi = L::mi(K);
    constexpr int I = ipow(Mi, AX);
    const int i0 = line % I, o = line / I;
    const T* src = in + o * Mi * I + i0;
    T* dst = out + o * Mi * I + i0;
    T v[Mi];
#pragma unroll
    for (int i = 0; i < Mi; ++i) v[i] = src[i * I];
#pragma unroll
    for (int k = 0; k < Mi; ++k) {
      T t = T(0);
#pragma unroll
      for (int i = 0; i < Mi; ++i) t += (BACK ? Sm[k * Mi + i] : Sm[i * Mi + k]) * v[i];
      dst[k * I] = t;
    }
  }

  template <int K>
  __device__ void fdm_step(bool zero_start) {
    constexpr int q = L::q(K), Mi = L::mi(K), NI = L::ni(K);
    constexpr int NLINE = NI / Mi;                     // lines along one axis
    static_assert(2 * NI <= L::SCRATCH, "the fast-diagonalisation buffers exceed the scratch region");
    int src = L::R_(K);
    if (!zero_start) {                                 // res = r - A d
      apply_int<K>(L::D_(K), epi<K>(EPI_RESID));
      src = L::RES(K);
    }
    auto X = [&](int pp) { return vec(pp, L::SCR); };
    auto Y = [&](int pp) { return vec(pp, L::SCR) + NI; };
    // reference-patch table of level K: [S: Mi x Mi][lambda: Mi][diag K: Mi][diag M: Mi]
    const T* const tab = a->lv[K].fdm;
    auto Sm = [&](int) { return tab; };
    auto lam = [&](int) { return tab + Mi * Mi; };
    TM::template loop<NLINE>([&](int pp, int l) { fdm_line<K, 0, false>(Sm(pp), vec(pp, src), X(pp), l); });
    TM::sync();
    if constexpr (DIM == 3) {
      TM::template loop<NLINE>([&](int pp, int l) { fdm_line<K, 1, false>(Sm(pp), X(pp), Y(pp), l); });
      TM::sync();
    }
    // last axis: forward, 1 / (lambda_x + lambda_y [+ lambda_z]), backward, in place
    TM::template loop<NLINE>([&](int pp, int l) {
      T* buf = (DIM == 3) ? Y(pp) : X(pp);
      const T* S = Sm(pp);
      const T* lm = lam(pp);
      const T lsum = (DIM == 3) ? lm[l % Mi] + lm[l / Mi] : lm[l];
      T v[Mi], w[Mi];
#pragma unroll
      for (int i = 0; i < Mi; ++i) v[i] = buf[i * NLINE + l];
#pragma unroll
      for (int k = 0; k < Mi; ++k) {
        T t = T(0);
#pragma unroll
        for (int i = 0; i < Mi; ++i) t += S[i * Mi + k] * v[i];
        w[k] = t / (lsum + lm[k]);
      }
#pragma unroll
      for (int i = 0; i < Mi; ++i) {
        T t = T(0);
#pragma unroll
        for (int k = 0; k < Mi; ++k) t += S[i * Mi + k] * w[k];
        buf[i * NLINE + l] = t;
      }
    });
    TM::sync();
    if constexpr (DIM == 3) {
      TM::template loop<NLINE>([&](int pp, int l) { fdm_line<K, 1, true>(Sm(pp), Y(pp), X(pp), l); });
      TM::sync();
    }
    // x: S, then d (+)= omega dinv diag(A_b) z, diag(A_b) from the 1D diagonals
    const T om = T(a->omega);
    TM::template loop<NLINE>([&](int pp, int l) {
      const T* S = Sm(pp);
      const T* Kd = tab + Mi * Mi + Mi;
      const T* Md = Kd + Mi;
      const T* in = X(pp) + l * Mi;
      T v[Mi];
#pragma unroll
      for (int k = 0; k < Mi; ++k) v[k] = in[k];
      int jy, jz;
      if constexpr (DIM == 3) {
        jy = l % Mi;
        jz = l / Mi;
      } else {
        jy = l;
        jz = 0;
      }
      T* d = vec(pp, L::D_(K)) + l * Mi;
      const T* dv = vec(pp, L::DINV(K)) + l * Mi;
#pragma unroll
      for (int i = 0; i < Mi; ++i) {
        T t = T(0);
#pragma unroll
        for (int k = 0; k < Mi; ++k) t += S[i * Mi + k] * v[k];
        T dg;
        if constexpr (DIM == 3)
          dg = Kd[i] * Md[jy] * Md[jz] + Md[i] * Kd[jy] * Md[jz] + Md[i] * Md[jy] * Kd[jz];
        else
          dg = Kd[i] * Md[jy] + Md[i] * Kd[jy];
        const T upd = om * dv[i] * dg * t;
        d[i] = zero_start ? upd : d[i] + upd;
      }
    });
    TM::sync();
    (void)q;
  }

  // ---- smoother on level K: d <- S(d; r), zero_start => d = 0 on entry
  template <int K>
  __device__ void smooth(bool zero_start) {
    constexpr int NI = L::ni(K);
    if (a->smoother == 2) {
      fdm_step<K>(zero_start);
      return;
    }
    if (a->smoother == 1) {   // damped Jacobi, d += omega D^-1 (r - A d)
      if (zero_start) {
        const T om = T(a->omega);
        TM::template loop<NI>([&](int pp, int i) { vec(pp, L::D_(K))[i] = om * vec(pp, L::DINV(K))[i] * vec(pp, L::R_(K))[i]; });
        TM::sync();
      } else {
        apply_int<K>(L::D_(K), epi<K>(EPI_JAC));
      }
      return;
    }
    // Chebyshev iteration (three-term recurrence on D^-1 A over [lo, hi])
    const int deg = a->cheb_degree;
    if (zero_start) {
      TM::template loop<NI>([&](int pp, int i) {
        const T* cf = vec(pp, L::COEF + K * L::NCOEF);
        const T res = vec(pp, L::DINV(K))[i] * vec(pp, L::R_(K))[i];
        const T dir = res * cf[0];
        vec(pp, L::RES(K))[i] = res;
        vec(pp, L::DIR(K))[i] = dir;
        vec(pp, L::D_(K))[i] = dir;
      });
      TM::sync();
    } else {
      apply_int<K>(L::D_(K), epi<K>(EPI_CHEB0));
    }
#pragma unroll 1
    for (int it = 1; it < deg; ++it) apply_int<K>(L::DIR(K), epi<K>(EPI_CHEB, it));
  }

  // ---- Algorithm 2
  template <int K>
  __device__ void vcycle(bool zero_start) {
    constexpr int q = L::q(K);
    if constexpr (q == 1) {
      TM::template loop<1>([&](int pp, int) { vec(pp, L::D_(K))[0] = vec(pp, L::R_(K))[0] * vec(pp, L::DINV(K))[0]; });
      TM::sync();
    } else {
      constexpr int NI = L::ni(K);
      smooth<K>(zero_start);                                      // pre-smoothing
      apply_int<K>(L::D_(K), epi<K>(EPI_RESID));                  // residual
      restrict_res<K>();                                          // restriction
      vcycle<K + 1>(true);                                        // coarse correction
      prolong_add<K>();                                           // prolongation
      smooth<K>(false);                                           // post-smoothing
    }
  }

  // ---- per-patch set-up: ids, cell list, level diagonals, Chebyshev coefficients
  __device__ void setup_patch(int pp, int item, bool active) {
    int pid = 0;
    const int N = a->N, Nv = N - 1;
    if (active) {
      if (MODE == MODE_SWEEP) {
        pid = list[item];
      } else {
        const int64_t raw = a->unit_rhs ? (int64_t)(item / L::ni(0)) : a->ids64[item];
        int64_t np = 1;
        for (int ax = 0; ax < DIM; ++ax) np *= Nv;
        if (raw >= 0 && raw < np) pid = (int)raw;
        else active = false;                            // not a patch: a zero row
      }
    }
    int v[3] = {1, 1, 1};
    int rem = pid;
    for (int ax = 0; ax < DIM; ++ax) { v[ax] = 1 + rem % Nv; rem /= Nv; }
    int* cl = cells + pp * CST;
    for (int s = 0; s < NCELL; ++s) {
      int id = 0, mul = 1;
      for (int ax = 0; ax < DIM; ++ax) { id += (v[ax] - 1 + ((s >> ax) & 1)) * mul; mul *= N; }
      cl[s] = active ? id : 0;
    }
    cl[NCELL] = pid;
    cl[NCELL + 1] = active ? 1 : 0;
    for (int ax = 0; ax < 3; ++ax) cl[NCELL + 2 + ax] = v[ax];
  }

  __device__ int patch_vertex(int pp, int ax) const { return cells[pp * CST + NCELL + 2 + ax]; }

  // global index on the degree-q grid of patch-local node (k_x, k_y[, k_z]) in [0, 2q]
  template <int q>
  __device__ size_t gindex(int pp, int i) const {
    constexpr int Mq = 2 * q + 1;
    const int N = a->N;
    const size_t Mg = (size_t)q * N + 1;
    size_t idx = 0, mul = 1;
    int rem = i;
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
      const int k = rem % Mq;
      rem /= Mq;
      idx += (size_t)(q * (patch_vertex(pp, ax) - 1) + k) * mul;
      mul *= Mg;
    }
    return idx;
  }
  // same for interior node i of the (2q-1)^d interior box
  template <int q>
  __device__ size_t gindex_int(int pp, int i) const {
    constexpr int Mi = 2 * q - 1;
    const int N = a->N;
    const size_t Mg = (size_t)q * N + 1;
    size_t idx = 0, mul = 1;
    int rem = i;
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
      const int k = rem % Mi;
      rem /= Mi;
      idx += (size_t)(q * (patch_vertex(pp, ax) - 1) + 1 + k) * mul;
      mul *= Mg;
    }
    return idx;
  }

  template <int K>
  __device__ void load_level() {
    constexpr int q = L::q(K);
    if constexpr (q == 1) {
      TM::template loop<1>([&](int pp, int) {
        const bool act = cells[pp * CST + NCELL + 1];
        const int N = a->N;
        size_t idx = 0, mul = 1;
        for (int ax = 0; ax < DIM; ++ax) { idx += (size_t)patch_vertex(pp, ax) * mul; mul *= (N + 1); }
        vec(pp, L::DINV(K))[0] = act ? a->lv[K].dinv[idx] : T(0);
      });
    } else {
      constexpr int NI = L::ni(K);
      const T* dinv = a->lv[K].dinv;
      stage<NI>([&](int pp, int i) {
        const bool act = cells[pp * CST + NCELL + 1];
        return act ? __ldg(dinv + gindex_int<q>(pp, i)) : T(0);
      }, [&](int pp, int i, T v) { vec(pp, L::DINV(K))[i] = v; });
      if constexpr (dense_level(DIM, q)) {
        const T* dense = a->lv[K].dense;
        stage<NI * NI>([&](int pp, int e) {
          const bool act = cells[pp * CST + NCELL + 1];
          const int pid = cells[pp * CST + NCELL];
          return act ? __ldg(dense + (size_t)pid * NI * NI + e) : T(0);
        }, [&](int pp, int e, T v) { vec(pp, L::DENSE(K))[e] = v; });
      }
      if constexpr (C::GSMEM && K == 0) {                // the cells' geometry tensors, once per patch
        constexpr int GC = L::GCELL;
        const T* G = a->lv[K].G;
        stage<NCELL * GC>([&](int pp, int e) {
          const bool act = cells[pp * CST + NCELL + 1];
          const int slot = e / GC;
          return act ? __ldg(G + (size_t)cells[pp * CST + slot] * GC + (e - slot * GC)) : T(0);
        }, [&](int pp, int e, T v) { vec(pp, L::GS)[e] = v; });
      }
      // Chebyshev coefficients of the three-term recurrence (Saad, Algorithm
      // 12.1): with sigma = theta / delta the recurrence rho_1 = 1 / sigma,
      // rho_{i+1} = 1 / (2 sigma - rho_i) has the closed form
      // rho_i = C_{i-1}(sigma) / C_i(sigma) (C_k: Chebyshev polynomials of the
      // first kind), so coefficient i is computed by thread i on its own, in
      // the kernel's precision: cf[i] = rho_{i+1} rho_i = C_{i-1} / C_{i+1},
      // cf[7 + i] = 2 rho_{i+1} / delta = 2 C_i / (delta C_{i+1}).
      if (a->smoother == 0) {
        TM::template loop<8>([&](int pp, int i) {
          const bool act = cells[pp * CST + NCELL + 1];
          const int pid = cells[pp * CST + NCELL];
          T lo = T(1), hi = T(2);
          if (act) { lo = a->lv[K].bounds[2 * (size_t)pid]; hi = a->lv[K].bounds[2 * (size_t)pid + 1]; }
          const T theta = T(0.5) * (hi + lo), delta = T(0.5) * (hi - lo);
          T* cf = vec(pp, L::COEF + K * L::NCOEF);
          if (i == 0) {
            cf[0] = T(1) / theta;
            return;
          }
          const T sigma = theta / delta;
          T cm = T(1), c0 = sigma;                       // C_{k-1}, C_k at k = 1
          for (int k = 1; k < i; ++k) {
            const T cn = T(2) * sigma * c0 - cm;
            cm = c0;
            c0 = cn;
          }
          const T cp = T(2) * sigma * c0 - cm;           // C_{i+1}
          cf[i] = cm / cp;
          cf[7 + i] = (T(2) * c0) / (delta * cp);
        });
      }
    }
    if constexpr (K + 1 < NL) load_level<K + 1>();
  }

  __device__ void run() {
    const int item0 = blk * PPB;
    TM::per_block([&](int pp) { setup_patch(pp, item0 + pp, item0 + pp < n_items); });
    TM::sync();
    load_level<0>();
    constexpr int NI0 = L::ni(0);
    if (MODE == MODE_SWEEP) {
      // Gather: closure of u, interior of b
      // (u is not written by any patch of this launch that another patch
      // reads: patches of one colour share no cell)
      constexpr int NN0 = L::NN0;
      const T* ug = a->u;
      const T* bg = a->b;
      stage<NN0>([&](int pp, int i) {
        const bool act = cells[pp * CST + NCELL + 1];
        if (!act) return T(0);
        const T* q = ug + gindex<P>(pp, i);
        return coherent ? __ldcg(q) : __ldg(q);
      }, [&](int pp, int i, T v) { vec(pp, L::CLOS)[i] = v; });
      stage<NI0>([&](int pp, int i) {
        const bool act = cells[pp * CST + NCELL + 1];
        return act ? __ldg(bg + gindex_int<P>(pp, i)) : T(0);
      }, [&](int pp, int i, T v) { vec(pp, L::R_(0))[i] = v; });
      TM::sync();
      // Evaluate: r = b - A u on the patch interior
      SF<DIM, 2, P, T, NT, PPB, C::LINE, C::GROUPED>::template apply_epi<false>(vec(0, L::CLOS), PS, vec(0, L::SCR), PS,
                                                                   gfun<0>(), epi<0>(EPI_EVAL));
      if (a->weight_residual) {               // transposed additive sweep: r <- W r
        TM::template loop<NI0>([&](int pp, int i) {
          constexpr int Mi = 2 * P - 1;
          int rem = i, m = 1;
#pragma unroll
          for (int ax = 0; ax < DIM; ++ax) {
            const int k = rem % Mi;
            rem /= Mi;
            m *= patch_multiplicity_1d(P * (patch_vertex(pp, ax) - 1) + 1 + k, P, a->N);
          }
          vec(pp, L::R_(0))[i] /= T(m);
        });
        TM::sync();
      }
    } else {
      TM::template loop<NI0>([&](int pp, int i) {
        const bool act = cells[pp * CST + NCELL + 1];
        const int it = item0 + pp;
        vec(pp, L::R_(0))[i] = !act ? T(0) : a->unit_rhs ? T(i == it % NI0 ? 1 : 0) : a->r_in[(size_t)it * NI0 + i];
      });
      TM::sync();
    }
    // Solve: N_MG V-cycles, the first from d = 0 (or their tabulated operator)
    if (MODE == MODE_SWEEP && a->solveop) {
      // tabulated local solve: d = B_j r, one owner per output, fixed order over m
      TM::template loop<NI0>([&](int pp, int k) {
        const bool act = cells[pp * CST + NCELL + 1];
        T s = T(0);
        if (act) {
          // 32 loads in flight per thread before their FMAs (the order over m is kept)
          const T* B = a->solveop + (size_t)cells[pp * CST + NCELL] * NI0 * NI0 + k;
          const T* r = vec(pp, L::R_(0));
          constexpr int W = 32;
          int m = 0;
#pragma unroll 1
          for (; m + W <= NI0; m += W) {
            T bv[W];
#pragma unroll
            for (int j = 0; j < W; ++j) bv[j] = __ldg(B + (size_t)(m + j) * NI0);
#pragma unroll
            for (int j = 0; j < W; ++j) s += bv[j] * r[m + j];
          }
#pragma unroll 1
          for (; m < NI0; ++m) s += __ldg(B + (size_t)m * NI0) * r[m];
        }
        vec(pp, L::D_(0))[k] = s;
      });
      TM::sync();
    } else {
#pragma unroll 1
      for (int cyc = 0; cyc < a->n_mg; ++cyc) vcycle<0>(cyc == 0);
    }
    // Scatter
    if (MODE == MODE_SWEEP) {
      T* dst = a->corr ? a->corr : a->u;      // additive: corrections collected apart from u
      TM::template loop<NI0>([&](int pp, int i) {
        const bool act = cells[pp * CST + NCELL + 1];
        if (act) {
          T* q = dst + gindex_int<P>(pp, i);
          *q = (coherent ? __ldcg(q) : *q) + vec(pp, L::D_(0))[i];
        }
      });
    } else {
      TM::template loop<NI0>([&](int pp, int i) {
        const bool act = cells[pp * CST + NCELL + 1];
        if (item0 + pp < n_items) a->d_out[(size_t)(item0 + pp) * NI0 + i] = act ? vec(pp, L::D_(0))[i] : T(0);
      });
    }
  }
};

template <int DIM, int P, typename T, int MODE, int V = 0>
__global__ void __launch_bounds__(Config<DIM, P, T, V>::NT, Config<DIM, P, T, V>::MINB)
    k_patch(const __grid_constant__ PatchArgs<T> args) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using PK = PatchKernel<DIM, P, T, MODE, V>;
  PK k;
  k.sm = reinterpret_cast<T*>(smem_raw);
  k.cells = reinterpret_cast<int*>(smem_raw + sizeof(T) * (size_t)PK::PS * PK::PPB);
  k.a = &args;
  k.list = args.list;
  k.n_items = args.n_items;
  k.blk = blockIdx.x;
  k.run();
}

// ------------------------------------------------------------------------
// Persistent sweep of one mesh level: one co-resident (cooperative) launch
// visits every colour in turn (Algorithm 1), the CTAs striding over the
// colour's patch batches, with a grid-wide barrier between colours.  The
// barrier is an arrival counter and a generation word in global memory; a
// CTA waits for the generation to move with a bounded spin (clock64 budget).
// When a wait runs out, the CTA sets the status word and returns, and every
// other CTA returns at its next barrier or wait: no CTA waits without limit,
// and the host reads the status (PMG_ERR_TIMEOUT).  The CTA that times out
// leaves the counter behind; the host zeroes counter and status before it
// reports the timeout.
struct GridSync {
  unsigned int* count;    // arrivals at the current barrier
  unsigned int* gen;      // barrier generation
  int* status;            // 0, or 1 after a wait ran out of budget
  long long budget;       // clock64 cycles one CTA waits at one barrier
};

__device__ inline bool grid_sync(const GridSync& g) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (*(volatile int*)g.status != 0) {
      ok = 0;
    } else {
      const unsigned int my = *(volatile unsigned int*)g.gen;   // before arriving
      __threadfence();                                          // this CTA's writes before its arrival
      if (atomicAdd(g.count, 1u) == gridDim.x - 1) {
        atomicExch(g.count, 0u);
        __threadfence();
        atomicAdd(g.gen, 1u);
      } else {
        const long long t0 = clock64();
        while (*(volatile unsigned int*)g.gen == my) {
          if (*(volatile int*)g.status != 0) {
            ok = 0;
            break;
          }
          if (clock64() - t0 > g.budget) {
            atomicExch(g.status, 1);
            ok = 0;
            break;
          }
          __nanosleep(64);
        }
      }
      __threadfence();                                          // the others' writes before ours reads
    }
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

template <typename T>
struct PersistArgs {
  PatchArgs<T> base;              // list and n_items unused
  const int32_t* lists[8];        // patch ids of every colour
  int counts[8];
  int n_colours;
  int reverse;                    // visit the colours in reverse order
  GridSync sync;
};

template <int DIM, int P, typename T, int V>
__global__ void __launch_bounds__(Config<DIM, P, T, V>::NT, Config<DIM, P, T, V>::MINB)
    k_patch_persist(const __grid_constant__ PersistArgs<T> pa) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using PK = PatchKernel<DIM, P, T, MODE_SWEEP, V>;
  PK k;
  k.sm = reinterpret_cast<T*>(smem_raw);
  k.cells = reinterpret_cast<int*>(smem_raw + sizeof(T) * (size_t)PK::PS * PK::PPB);
  k.a = &pa.base;
  k.coherent = true;                   // colours after the first read what earlier colours wrote
  for (int i = 0; i < pa.n_colours; ++i) {
    const int c = pa.reverse ? pa.n_colours - 1 - i : i;
    k.list = pa.lists[c];
    k.n_items = pa.counts[c];
    const int nblk = (k.n_items + PK::PPB - 1) / PK::PPB;
    for (int b = blockIdx.x; b < nblk; b += gridDim.x) {
      k.blk = b;
      k.run();
      __syncthreads();                 // shared memory is reused by the next batch
    }
    if (i + 1 < pa.n_colours && !grid_sync(pa.sync)) return;
  }
}

// ------------------------------------------------------------------------
// Dense patch matrices of a small level (set-up): column i of A_{j,q} is the
// matrix-free patch operator applied to the unit vector e_i.  One patch per
// CTA; FP64.
template <int DIM, int Q>
__global__ void __launch_bounds__(128) k_dense_patch(const double* __restrict__ G, int N, int first_patch,
                                                     int n_items, double* __restrict__ A) {
  constexpr int NT = 128;
  using Dm = Dims<DIM, 2, Q, 8>;
  constexpr int NI = Dm::NI;
  constexpr int NCELL = 1 << DIM;
  double* x = reinterpret_cast<double*>(pmg_smem);
  double* y = x + NI;
  double* scr = y + NI;
  int* cl = reinterpret_cast<int*>(scr + Dm::SCRATCH);
  const int item = blockIdx.x;
  if (item >= n_items) return;
  const int pid = first_patch + item;
  if (threadIdx.x < NCELL) {
    const int Nv = N - 1;
    int rem = pid, id = 0, mul = 1;
    for (int ax = 0; ax < DIM; ++ax) {
      const int v = 1 + rem % Nv;
      rem /= Nv;
      id += (v - 1 + ((threadIdx.x >> ax) & 1)) * mul;
      mul *= N;
    }
    cl[threadIdx.x] = id;
  }
  auto gf = [G](int, int slot) {
    const int* clp = reinterpret_cast<const int*>(pmg_smem + sizeof(double) * (2 * NI + Dm::SCRATCH));
    return G + (size_t)clp[slot] * (Dm::NCOMP * Dm::NGC);
  };
  for (int i = 0; i < NI; ++i) {
    for (int r = threadIdx.x; r < NI; r += NT) x[r] = r == i ? 1.0 : 0.0;
    __syncthreads();
    SF<DIM, 2, Q, double, NT, 1>::template apply<true, false>(x, 0, y, 0, scr, 0, gf);
    for (int r = threadIdx.x; r < NI; r += NT) A[((size_t)item * NI + r) * NI + i] = y[r];
    __syncthreads();
  }
}

template <int DIM, int Q>
constexpr size_t dense_patch_smem() {
  using Dm = Dims<DIM, 2, Q, 8>;
  return sizeof(double) * (2 * Dm::NI + Dm::SCRATCH) + sizeof(int) * (1 << DIM);
}

// ------------------------------------------------------------------------
// Lanczos estimate of the extreme eigenvalues of D^-1/2 A_{j,q} D^-1/2 for
// one p-level K of a batch of patches (one patch per CTA).  Full
// reorthogonalisation (two classical Gram-Schmidt passes); the basis lives in
// global scratch [n_items][ksteps][Ni].  Start vector 1 + (u - 1/2), u from
// counter-based SplitMix64 with counter (patch << 20) | (q << 16) | i.
// The extreme eigenvalues of the tridiagonal matrix come from Sturm-sequence
// bisection on its Gershgorin interval.
template <typename T>
struct LanczosArgs {
  int N;
  int n_items;
  int first_patch;        // patch id of item 0 (items are consecutive patches)
  const T* G;
  const T* dinv;
  double* V;              // scratch [n_items][ksteps][Ni] (FP64 basis)
  int ksteps;
  uint64_t seed;
  double safety, ratio;
  double* ritz;           // [patches][2] (theta_min, theta_max), FP64
  T* bounds;              // [patches][2] (lo, hi), or NULL
  double* bounds_f64;     // [patches][2] (lo, hi) rounded to T, then widened to FP64, or NULL
  int64_t out_offset;     // patch id written to entry 0 of ritz / bounds / bounds_f64
};

__device__ __forceinline__ uint64_t splitmix64_dev(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <int NT>
__device__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NT / 32; ++i) s += red[i];
    red[NT / 32] = s;
  }
  __syncthreads();
  return red[NT / 32];
}

__device__ inline int sturm_count_dev(const double* al, const double* be, int n, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < n; ++i) {
    d = al[i] - x - (i > 0 ? be[i - 1] * be[i - 1] / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

template <int DIM, int Q, typename T>
__global__ void __launch_bounds__(256) k_lanczos(const __grid_constant__ LanczosArgs<T> a) {
  constexpr int NT = 256;
  using Dm = Dims<DIM, 2, Q, (int)sizeof(T)>;
  constexpr int NI = Dm::NI;
  constexpr int NCELL = 1 << DIM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sv = reinterpret_cast<T*>(smem_raw);          // S v input (T)
  T* sAd = sv + NI;                                  // A output
  T* scr = sAd + NI;                                 // apply scratch
  double* dv = reinterpret_cast<double*>(scr + Dm::SCRATCH + 2);   // v (FP64)
  dv = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(dv) + 15) & ~uintptr_t(15));
  double* dw = dv + NI;
  double* ds = dw + NI;                              // sqrt(dinv)
  double* red = ds + NI;                             // reduction scratch (NT/32 + 1)
  double* al = red + NT / 32 + 2;                    // alpha[ksteps]
  double* be = al + 64;                              // beta[ksteps]
  double* cf = be + 64;                              // CGS coefficients[ksteps]
  int* cl = reinterpret_cast<int*>(cf + 64);
  const size_t cl_byte = reinterpret_cast<unsigned char*>(cl) - smem_raw;

  const int item = blockIdx.x;
  if (item >= a.n_items) return;
  const int pid = a.first_patch + item;
  const int N = a.N, Nv = N - 1;
  int v[3] = {1, 1, 1};
  {
    int rem = pid;
    for (int ax = 0; ax < DIM; ++ax) { v[ax] = 1 + rem % Nv; rem /= Nv; }
  }
  if (threadIdx.x < NCELL) {
    int id = 0, mul = 1;
    for (int ax = 0; ax < DIM; ++ax) { id += (v[ax] - 1 + ((threadIdx.x >> ax) & 1)) * mul; mul *= N; }
    cl[threadIdx.x] = id;
  }
  const size_t Mg = (size_t)Q * N + 1;
  for (int i = threadIdx.x; i < NI; i += NT) {
    size_t idx = 0, mul = 1;
    int rem = i;
    for (int ax = 0; ax < DIM; ++ax) {
      const int k = rem % (2 * Q - 1);
      rem /= (2 * Q - 1);
      idx += (size_t)(Q * (v[ax] - 1) + 1 + k) * mul;
      mul *= Mg;
    }
    ds[i] = sqrt((double)a.dinv[idx]);
    const uint64_t ctr = ((uint64_t)pid << 20) | ((uint64_t)Q << 16) | (uint64_t)i;
    const uint64_t z = splitmix64_dev(a.seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull);
    dv[i] = 1.0 + ((double)(z >> 11) * 0x1.0p-53 - 0.5);
  }
  __syncthreads();
  const int k = a.ksteps < NI ? a.ksteps : NI;
  double* Vb = a.V + (size_t)item * a.ksteps * NI;
  {
    double s = 0.0;
    for (int i = threadIdx.x; i < NI; i += NT) s += dv[i] * dv[i];
    const double nrm = sqrt(block_sum<NT>(s, red));
    for (int i = threadIdx.x; i < NI; i += NT) dv[i] /= nrm;
    __syncthreads();
  }
  const T* G = a.G;
  auto gf = [G, cl_byte](int, int slot) {
    return G + (size_t)reinterpret_cast<const int*>(pmg_smem + cl_byte)[slot] * (Dm::NCOMP * Dm::NGC);
  };
  int nal = 0;
  for (int j = 0; j < k; ++j) {
    for (int i = threadIdx.x; i < NI; i += NT) {
      Vb[(size_t)j * NI + i] = dv[i];
      sv[i] = T(ds[i] * dv[i]);
    }
    __syncthreads();
    SF<DIM, 2, Q, T, NT, 1>::template apply<true, false>(sv, 0, sAd, 0, scr, 0, gf);
    double s = 0.0;
    for (int i = threadIdx.x; i < NI; i += NT) {
      dw[i] = ds[i] * (double)sAd[i];
      s += dv[i] * dw[i];
    }
    const double alpha = block_sum<NT>(s, red);
    if (threadIdx.x == 0) al[j] = alpha;
    nal = j + 1;
    for (int pass = 0; pass < 2; ++pass) {
      for (int m = 0; m <= j; ++m) {
        double t = 0.0;
        for (int i = threadIdx.x; i < NI; i += NT) t += Vb[(size_t)m * NI + i] * dw[i];
        const double c = block_sum<NT>(t, red);
        if (threadIdx.x == 0) cf[m] = c;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < NI; i += NT) {
        double w = dw[i];
        for (int m = 0; m <= j; ++m) w -= cf[m] * Vb[(size_t)m * NI + i];
        dw[i] = w;
      }
      __syncthreads();
    }
    if (j == k - 1) break;
    double t = 0.0;
    for (int i = threadIdx.x; i < NI; i += NT) t += dw[i] * dw[i];
    const double b = sqrt(block_sum<NT>(t, red));
    if (b <= 1e-300) break;
    if (threadIdx.x == 0) be[j] = b;
    for (int i = threadIdx.x; i < NI; i += NT) dv[i] = dw[i] / b;
    __syncthreads();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int n = nal;
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < n; ++i) {
      const double bl = i > 0 ? fabs(be[i - 1]) : 0.0, br = i < n - 1 ? fabs(be[i]) : 0.0;
      lo = fmin(lo, al[i] - bl - br);
      hi = fmax(hi, al[i] + bl + br);
    }
    double ext[2];
    for (int e = 0; e < 2; ++e) {
      const int kidx = e == 0 ? 0 : n - 1;
      double x0 = lo, x1 = hi;
      for (int it = 0; it < 100; ++it) {
        const double mid = 0.5 * (x0 + x1);
        if (sturm_count_dev(al, be, n, mid) > kidx) x1 = mid;
        else x0 = mid;
      }
      ext[e] = 0.5 * (x0 + x1);
    }
    const double bhi = a.safety * ext[1];
    const double blo = fmax(ext[0], bhi / a.ratio);
    const size_t o = 2 * (size_t)((int64_t)pid - a.out_offset);
    a.ritz[o] = ext[0];
    a.ritz[o + 1] = ext[1];
    if (a.bounds) {
      a.bounds[o] = T(blo);
      a.bounds[o + 1] = T(bhi);
    }
    if (a.bounds_f64) {
      a.bounds_f64[o] = (double)T(blo);
      a.bounds_f64[o + 1] = (double)T(bhi);
    }
  }
}

template <int DIM, int Q, typename T>
constexpr size_t lanczos_smem() {
  using Dm = Dims<DIM, 2, Q, (int)sizeof(T)>;
  return sizeof(T) * (2 * Dm::NI + Dm::SCRATCH + 2) + 16 +
         sizeof(double) * (3 * Dm::NI + 256 / 32 + 2 + 3 * 64) + sizeof(int) * 16;
}

}  // namespace pmg
