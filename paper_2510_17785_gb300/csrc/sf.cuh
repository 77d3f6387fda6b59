// Sum-factorised evaluation of the Q_q operator a(u,v) = int kappa grad u . grad v
// on a tensor-product block of NC^DIM cells (NC = 2: a vertex patch; NC = 1: one
// cell).  Paper Section 3.1 ("Level operators"): the operator is applied
// matrix-free; per cell d one-dimensional contractions take the nodal values
// to gradients at the quadrature points and d more integrate the fluxes back,
// O(d q^{d+1}) work and O(q^d) memory.
//
// Along one direction the block has M = NC*q + 1 Gauss-Lobatto nodes and
// QP = NC*(q+1) Gauss points; cell c owns nodes c*q .. c*q+q and points
// c*n .. c*n+n-1 (n = q+1).  A node shared by two cells receives the
// contributions of both in the transposed sweep, so the block result is the
// assembled sum without atomics.  For a patch (NC = 2) the outer nodes carry
// homogeneous Dirichlet values: inputs may be given on the Mi = 2q-1 interior
// nodes only, and outputs are produced on interior nodes only.
//
// Data layout: [z][y][x] with x fastest.  Forward: interpolate to Gauss points
// along x, y, z (B), then differentiate along each direction at the Gauss
// points (collocation derivative D).  Each point multiplies the reference
// gradient by the symmetric tensor G = w kappa det(J) J^-1 J^-T (stored per
// cell as DIM*(DIM+1)/2 components).  Backward: D^T along each direction
// summed, then B^T along z, y, x.  Along the last direction one thread owns a
// whole line for the interpolation, the point products and the transposed
// sweeps, keeping that direction's gradient and flux in registers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "tables.cuh"

namespace pmg {

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// Dynamic shared memory of the launching kernel: every kernel that applies
// the operator keeps its vectors and scratch there.  A pointer into it that
// crosses a non-inlined call is only a generic address to the callee, whose
// loads and stores then go through the generic path; smem_ptr() re-derives
// the same address from this __shared__ array so that they stay shared-memory
// accesses.
extern __shared__ __align__(16) unsigned char pmg_smem[];

// d = a * b + c on both lanes (one packed FP32 FMA, fma.rn.f32x2)
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long ra, rb, rc, rd;
  memcpy(&ra, &a, 8);
  memcpy(&rb, &b, 8);
  memcpy(&rc, &c, 8);
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
  float2 d;
  memcpy(&d, &rd, 8);
  return d;
}

// Geometry functors (gcell) return the G base pointer of a cell; a functor
// type that declares `static constexpr bool kShared = true` serves G from
// shared memory, every other one from global memory, where it is read
// through the read-only data path (ld.global.nc), since G does not change
// during a launch.
template <typename GF, typename = void>
struct GeomInShared {
  static constexpr bool value = false;
};
template <typename GF>
struct GeomInShared<GF, decltype((void)GF::kShared)> {
  static constexpr bool value = GF::kShared;
};
template <typename GF, typename T>
__device__ __forceinline__ T gload(const T* p) {
  if constexpr (GeomInShared<GF>::value) return *p;
  else return __ldg(p);
}
// A functor that declares `static constexpr bool kPackable = true` and a
// member `bool packed` may serve FP32 geometry as BF16 pairs: when `packed`
// is set, its base pointers address words of two BF16 components (2j in the
// low half, 2j + 1 in the high half), pair j at offset j * (points per cell).
template <typename GF, typename = void>
struct GeomPackable {
  static constexpr bool value = false;
};
template <typename GF>
struct GeomPackable<GF, decltype((void)GF::kPackable)> {
  static constexpr bool value = GF::kPackable;
};
// the NCOMP components of G at point p of a cell (component stride NGC),
// from packed BF16 pairs (PACKED) or from values of type T
template <bool PACKED, int NCOMP, int NGC, typename GF, typename T>
__device__ __forceinline__ void gtensor(const T* p, T (&g)[NCOMP]) {
  if constexpr (PACKED) {
    static_assert(sizeof(T) == 4, "packed BF16 geometry feeds FP32 kernels");
    const unsigned* w = reinterpret_cast<const unsigned*>(p);
#pragma unroll
    for (int j = 0; j < (NCOMP + 1) / 2; ++j) {
      const unsigned x = __ldg(w + j * NGC);
      g[2 * j] = __uint_as_float(x << 16);                   // BF16 -> FP32 is exact
      if (2 * j + 1 < NCOMP) g[2 * j + 1] = __uint_as_float(x & 0xffff0000u);
    }
  } else {
#pragma unroll
    for (int k = 0; k < NCOMP; ++k) g[k] = gload<GF>(p + k * NGC);
  }
}
// f(std::true_type) when gcell serves packed BF16 pairs, else
// f(std::false_type): the geometry format is decided once per stage, so
// each stage body is compiled for one format (no per-point selection)
template <typename T, typename GF, typename F>
__device__ __forceinline__ void with_geom_format(const GF& gcell, F&& f) {
  if constexpr (sizeof(T) == 4 && GeomPackable<GF>::value) {
    if (gcell.packed) {
      f(std::true_type{});
      return;
    }
  }
  f(std::false_type{});
}

template <typename T>
__device__ __forceinline__ T* smem_ptr(T* p) {
  const unsigned off = (unsigned)(__cvta_generic_to_shared((const void*)p) - __cvta_generic_to_shared(pmg_smem));
  return reinterpret_cast<T*>(pmg_smem + off);
}
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }

// Shared-memory layout of the point arrays of the sum factorisation: rows of
// QP values along x.  A stage along x gives each thread one row, so a warp
// reads one element of 32 consecutive rows at a time; with rows packed at
// pitch QP those fall into 32 / gcd(QP, 32) banks (QP = 16: two banks, a
// 16-way conflict).  For QP a power of two the rows are therefore stored in
// groups of G rows (G * QP = one sweep of the 32 banks) with one element of
// slack after each group: row r starts at r * QP + r / G.  The 32 rows of a
// warp then start in 32 distinct banks, and the points of one group (what a
// stage along the last direction reads, one line per thread) stay
// contiguous.  A group holds at least two rows: where a single row would
// fill the banks (8-byte elements at QP = 16) the slack is halved at the
// price of a 2-way conflict (that keeps the FP64 degree-7 patch within
// shared memory).  sf_rows() is the size of an array of r rows of es-byte
// elements (128 / es of them per sweep of the banks).
__host__ __device__ constexpr bool sf_skew(int qp) { return (qp & (qp - 1)) == 0; }
__host__ __device__ constexpr int sf_group(int qp, int es) { return sf_skew(qp) ? cmax(128 / es / qp, 2) : 1; }
__host__ __device__ constexpr int sf_rows(int qp, int r, int es) {
  return r * qp + (sf_skew(qp) ? r / sf_group(qp, es) : 0);
}
// scratch elements of one block (V and R below; line: the line design)
__host__ __device__ constexpr int sf_scratch(int dim, int nc, int q, bool line, int es) {
  const int n = q + 1, M = nc * q + 1, QP = nc * n;
  const int Lo = nc == 2 ? 2 * q - 1 : M;
  const int NQS = sf_rows(QP, ipow(QP, dim - 1), es);
  // forward temporaries for the widest input (all nodes): [M]^(d-1) x QP and M x QP x QP
  const int T1 = sf_rows(QP, ipow(M, dim - 1), es), T2 = dim == 3 ? sf_rows(QP, M * QP, es) : 0;
  // backward temporaries: [Lo][QP][QP] and [Lo][Lo][QP] (3D), [Lo][QP] (2D)
  const int B = dim == 3 ? sf_rows(QP, Lo * Lo, es) + sf_rows(QP, Lo * QP, es) : sf_rows(QP, Lo, es);
  // stage design: all DIM flux arrays in R; line design: DIM - 1 of them
  const int R = line ? cmax(cmax(T1 + T2, (dim - 1) * NQS), B) : cmax(T1 + T2, dim * NQS);
  return NQS + R;
}

// sizes of the NC^DIM block of degree Q with ES-byte elements
template <int DIM, int NC, int Q, int ES>
struct Dims {
  static constexpr int n = Q + 1;
  static constexpr int M = NC * Q + 1;
  static constexpr int Mi = (NC == 2) ? 2 * Q - 1 : M;
  static constexpr int QP = NC * n;
  static constexpr int NQ = ipow(QP, DIM);        // quadrature points of the block
  static constexpr int NN = ipow(M, DIM);         // all nodes
  static constexpr int NI = ipow(Mi, DIM);        // interior nodes (patch) / all (cell)
  static constexpr int NCOMP = DIM * (DIM + 1) / 2;
  static constexpr int NGC = ipow(n, DIM);        // quadrature points per cell
  static constexpr int SCRATCH = sf_scratch(DIM, NC, Q, false, ES);      // V + R (stage design)
  static constexpr int SCRATCH_LINE = sf_scratch(DIM, NC, Q, true, ES);  // V + R (line design)
};

// Number of vertex patches whose interior holds the node with per-axis index
// g (degree q, N cells per direction, interior vertices 1..N-1): a node on a
// vertex line lies in that vertex's patches only, any other node in the
// patches of both end vertices of its cell that are interior.
__host__ __device__ inline int patch_multiplicity_1d(int g, int q, int N) {
  if (g % q == 0) return 1;
  const int c = g / q;
  return (c >= 1 && c <= N - 1) + (c + 1 >= 1 && c + 1 <= N - 1);
}

// A cooperative loop over PPB blocks x ITEMS work items.
template <int NT, int PPB, int ITEMS, typename F>
__device__ __forceinline__ void coop(F&& f) {
#pragma unroll 1
  for (int it = threadIdx.x; it < PPB * ITEMS; it += NT) {
    const int pp = it / ITEMS;
    f(pp, it - pp * ITEMS);
  }
}

// How the NT threads of a CTA share its PPB blocks.
//  GROUPED = false: every thread works on every block; a stage ends with a
//    CTA-wide barrier.
//  GROUPED = true: the CTA is PPB independent groups of TPP = NT / PPB threads
//    (a multiple of 32); group g works on block g only and synchronises with a
//    barrier of its own (named barrier g + 1, or a warp barrier for one-warp
//    groups), so no group waits for another group's block.
template <int NT, int PPB, bool GROUPED>
struct Team {
  static_assert(!GROUPED || (NT % PPB == 0 && (NT / PPB) % 32 == 0 && PPB <= 15), "bad grouped team");
  static constexpr int TPP = GROUPED ? NT / PPB : NT;      // threads sharing one item loop
  static constexpr int SPAN = GROUPED ? 1 : PPB;           // blocks covered by one item loop
  __device__ __forceinline__ static int group() { return GROUPED ? (int)threadIdx.x / TPP : 0; }
  __device__ __forceinline__ static int lane() { return GROUPED ? (int)threadIdx.x % TPP : (int)threadIdx.x; }
  __device__ __forceinline__ static void sync() {
    if constexpr (!GROUPED || PPB == 1) {
      __syncthreads();
    } else if constexpr (TPP == 32) {
      __syncwarp();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(group() + 1), "n"(TPP) : "memory");
    }
  }
  // f(pp, item) for item in [0, ITEMS) of every block this thread serves
  template <int ITEMS, typename F>
  __device__ __forceinline__ static void loop(F&& f) {
    if constexpr (GROUPED) {
      const int pp = group();
#pragma unroll 1
      for (int it = lane(); it < ITEMS; it += TPP) f(pp, it);
    } else {
      coop<NT, PPB, ITEMS>(f);
    }
  }
  // the l-th (block, item) slot of this thread in a loop over ITEMS items
  // per block: false when the thread has no l-th slot
  template <int ITEMS>
  __device__ __forceinline__ static bool slot(int l, int& pp, int& item) {
    const int it = lane() + l * TPP;
    if constexpr (GROUPED) {
      pp = group();
      item = it;
    } else {
      pp = it / ITEMS;
      item = it - pp * ITEMS;
    }
    return it < SPAN * ITEMS;
  }
  // f(pp) once for every block, by one thread
  template <typename F>
  __device__ __forceinline__ static void per_block(F&& f) {
    if constexpr (GROUPED) {
      if (lane() == 0) f(group());
    } else {
      for (int pp = threadIdx.x; pp < PPB; pp += NT) f(pp);
    }
  }
};

template <int DIM, int NC, int Q, typename T, int NT, int PPB, bool LINE = false, bool GROUPED = false>
struct SF {
  using D = Dims<DIM, NC, Q, (int)sizeof(T)>;
  using TM = Team<NT, PPB, GROUPED>;
  static constexpr int n = D::n, M = D::M, Mi = D::Mi, QP = D::QP, NQ = D::NQ;

  // ---- point-array addressing (see sf_rows): row r starts at rowa(r)
  static constexpr bool SKEW = sf_skew(QP);
  static constexpr int G = sf_group(QP, (int)sizeof(T));     // rows per group
  static constexpr int LG = ilog2(G);
  static_assert((1 << LG) == G, "");
  __host__ __device__ static constexpr int rowa(int r) { return r * QP + (SKEW ? (r >> LG) : 0); }
  static constexpr int NQS = rowa(ipow(QP, DIM - 1));         // one array of all points
  static_assert(NQS == sf_rows(QP, ipow(QP, DIM - 1), (int)sizeof(T)), "");
  // Along the last direction (z in 3D, y in 2D) point g of line i sits at
  // loff(g) + lbase(i): with QP rows per plane, rowa(z QP + y) = rowa(z QP) +
  // rowa(y) for y < QP (G divides QP, or QP divides G and the group index
  // does not change within a plane's first QP rows)
  __host__ __device__ static constexpr int loff(int g) { return DIM == 3 ? rowa(g * QP) : rowa(g); }
  __device__ __forceinline__ static int lbase(int i) {
    if constexpr (DIM == 3 && SKEW) return rowa(i / QP) + i % QP;
    else return i;
  }
  // lines along x (AX = 0: row `item`) and y (AX = 1, 3D: x = item % QP in
  // plane item / QP) of an array with QP rows per plane: first point, and
  // the offset of point h
  template <int AX>
  __device__ __forceinline__ static int lstart(int item) {
    static_assert(AX == 0 || (AX == 1 && DIM == 3), "lines along x, or along y in 3D");
    if constexpr (AX == 0) return rowa(item);
    else return rowa((item / QP) * QP) + item % QP;
  }
  template <int AX>
  __host__ __device__ static constexpr int lstep(int h) { return AX == 0 ? h : rowa(h); }

  // ---- line helpers: one item is a whole line of the block along an axis
  // (all NC cells).  The node values of a line with the patch's Dirichlet
  // ends (INTIN) are zero at both ends; those terms are skipped.
  template <bool INTIN>
  __device__ __forceinline__ static void load_line(const T* __restrict__ src, int stride, T (&v)[M]) {
#pragma unroll
    for (int k = 0; k < M; ++k) {
      if (INTIN && NC == 2) v[k] = (k == 0 || k == M - 1) ? T(0) : src[(k - 1) * stride];
      else v[k] = src[k * stride];
    }
  }
  // ---- y = M x for the n x n matrix KIND (EO_B, EO_BT, EO_D, EO_DT) of
  // degree Q, from the even and odd parts of x: with h = n / 2 and
  // M[n-1-i][n-1-j] = S M[i][j], the outputs i and n-1-i are E_i + O_i and
  // S (E_i - O_i), E_i = sum_j Ee[i][j] (x_j + x_{n-1-j}) (+ Em[i] x_h for odd n),
  // O_i = sum_j Eo[i][j] (x_j - x_{n-1-j}); about half the multiplications of
  // the plain product (12-13 instead of 25 at n = 5, 41 instead of 81 at n = 9).
  template <int KIND>
  __device__ __forceinline__ static void eo_apply(const T (&x)[n], T (&y)[n]) {
    constexpr int h = n / 2;
    constexpr bool odd = (n & 1) != 0;
    constexpr bool anti = (KIND == EO_D || KIND == EO_DT);
    T xe[h > 0 ? h : 1], xo[h > 0 ? h : 1];
#pragma unroll
    for (int j = 0; j < h; ++j) {
      xe[j] = x[j] + x[n - 1 - j];
      xo[j] = x[j] - x[n - 1 - j];
    }
#pragma unroll
    for (int i = 0; i < h; ++i) {
      T e, o;
      if constexpr (sizeof(T) == 4) {
        // the even and odd sums of output pair i as the two lanes of packed FMAs
        // (each lane the same FMAs in the same order as the scalar form)
        float2 acc = make_float2(odd ? tabEm<T>(KIND, Q, i) * x[h] : T(0), T(0));
#pragma unroll
        for (int j = 0; j < h; ++j) acc = ffma2(tabEO2(KIND, Q, i, j), make_float2(xe[j], xo[j]), acc);
        e = acc.x;
        o = acc.y;
      } else {
        e = odd ? tabEm<T>(KIND, Q, i) * x[h] : T(0);
#pragma unroll
        for (int j = 0; j < h; ++j) e += tabEe<T>(KIND, Q, i, j) * xe[j];
        o = T(0);
#pragma unroll
        for (int j = 0; j < h; ++j) o += tabEo<T>(KIND, Q, i, j) * xo[j];
      }
      y[i] = e + o;
      y[n - 1 - i] = anti ? o - e : e - o;
    }
    if constexpr (odd) {
      T m = T(0);
      if constexpr (anti) {
#pragma unroll
        for (int j = 0; j < h; ++j) m += tabEo<T>(KIND, Q, h, j) * xo[j];
      } else {
        m = tabEm<T>(KIND, Q, h) * x[h];
#pragma unroll
        for (int j = 0; j < h; ++j) m += tabEe<T>(KIND, Q, h, j) * xe[j];
      }
      y[h] = m;
    }
  }
  // the same on cell c of a line: x = in[c * step .. c * step + n), y to out[c * n ..)
  template <int KIND, int LIN, int LOUT>
  __device__ __forceinline__ static void eo_cell(const T (&in)[LIN], int base_in, T (&out)[LOUT], int base_out) {
    T x[n], y[n];
#pragma unroll
    for (int a = 0; a < n; ++a) x[a] = in[base_in + a];
    eo_apply<KIND>(x, y);
#pragma unroll
    for (int a = 0; a < n; ++a) out[base_out + a] = y[a];
  }

  // nodes -> Gauss points of every cell of the line (the patch's Dirichlet
  // end values are zero in v)
  template <bool INTIN>
  __device__ __forceinline__ static void interp_line(const T (&v)[M], T (&w)[QP]) {
#pragma unroll
    for (int c = 0; c < NC; ++c) eo_cell<EO_B>(v, c * Q, w, c * n);
  }
  // Gauss points of every cell -> nodes (transposed interpolation); NC = 2:
  // interior nodes 1..M-2 only, written to out[(k-1)*stride] (ACC: added);
  // NC = 1: all nodes.  The node shared by the two cells sums cell 0's terms,
  // then cell 1's.
  template <bool ACC, typename PUT>
  __device__ __forceinline__ static void integ_line(const T (&w)[QP], const PUT& put) {
    T y[QP];
#pragma unroll
    for (int c = 0; c < NC; ++c) eo_cell<EO_BT>(w, c * n, y, c * n);
    if constexpr (NC == 1) {
#pragma unroll
      for (int a = 0; a <= Q; ++a) put(a, ACC ? put.init(a) + y[a] : y[a]);
    } else {
#pragma unroll
      for (int k = 1; k <= M - 2; ++k) {
        const T t = (k < Q) ? y[k] : (k == Q ? y[Q] + y[n] : y[n + k - Q]);
        put(k - 1, ACC ? put.init(k - 1) + t : t);
      }
    }
  }
  // output sinks for integ_line: column x of rows row0, row0 + 1, ... of a
  // point array (ACC: add) / epilogue
  template <bool ACC>
  struct LineStore {
    T* dst;
    int row0, x;
    __device__ __forceinline__ T init(int k) const { return ACC ? dst[rowa(row0 + k) + x] : T(0); }
    __device__ __forceinline__ void operator()(int k, T s) const { dst[rowa(row0 + k) + x] = s; }
  };
  template <typename EPI>
  struct LineEpi {
    const EPI& epi;
    int pp, base;
    __device__ __forceinline__ T init(int) const { return T(0); }
    __device__ __forceinline__ void operator()(int k, T s) const { epi(pp, base + k, s); }
  };

  // ---- forward interpolation along axis AX, one line per item.  AX = 0: the
  // block's nodes [..][L] (packed) -> row `item` of T1; AX = 1 (3D): T1
  // [L][L][QP] -> T2 [L][QP][QP] (x = item % QP in plane item / QP)
  template <int AX, bool INTIN>
  __device__ __forceinline__ static void fwd_item(const T* __restrict__ in, T* __restrict__ out, int item) {
    constexpr int L = INTIN ? Mi : M;
    T v[M], w[QP];
    if constexpr (AX == 0) {
      load_line<INTIN>(in + item * L, 1, v);
      interp_line<INTIN>(v, w);
      T* dst = out + rowa(item);
#pragma unroll
      for (int g = 0; g < QP; ++g) dst[g] = w[g];
    } else {
      static_assert(AX == 1 && DIM == 3, "x, or y in 3D");
      const int i = item % QP, o = item / QP;
#pragma unroll
      for (int k = 0; k < M; ++k) {
        if (INTIN && NC == 2) v[k] = (k == 0 || k == M - 1) ? T(0) : in[rowa(o * L + k - 1) + i];
        else v[k] = in[rowa(o * L + k) + i];
      }
      interp_line<INTIN>(v, w);
      T* dst = out + rowa(o * QP) + i;
#pragma unroll
      for (int g = 0; g < QP; ++g) dst[rowa(g)] = w[g];
    }
  }

  // the M node values of line i along the last direction (INTIN: rows of the
  // interior nodes only, the patch's Dirichlet ends zero)
  template <bool INTIN>
  __device__ __forceinline__ static void load_last(const T* __restrict__ in, int b, T (&v)[M]) {
#pragma unroll
    for (int k = 0; k < M; ++k) {
      if (INTIN && NC == 2) v[k] = (k == 0 || k == M - 1) ? T(0) : in[loff(k - 1) + b];
      else v[k] = in[loff(k) + b];
    }
  }

  // ---- forward interpolation along the last axis fused with the collocation
  // derivative along it: writes the point values V and the derivative F.
  template <bool INTIN>
  __device__ __forceinline__ static void fwd_der_last_item(const T* __restrict__ in, T* __restrict__ V,
                                                           T* __restrict__ F, int i) {
    const int b = lbase(i);
    T v[M], w[QP], f[QP];
    load_last<INTIN>(in, b, v);
    interp_line<INTIN>(v, w);
#pragma unroll
    for (int g = 0; g < QP; ++g) V[loff(g) + b] = w[g];
#pragma unroll
    for (int c = 0; c < NC; ++c) eo_cell<EO_D>(w, c * n, f, c * n);
#pragma unroll
    for (int g = 0; g < QP; ++g) F[loff(g) + b] = f[g];
  }

  // ---- backward along the last axis for one line: w = (partial sums of the
  // other directions) + D^T f per cell, then B^T per cell; out[loff(k - 1)]
  // receives interior node k (NC = 2), out[loff(k)] node k (NC = 1).
  __device__ __forceinline__ static void last_bwd(const T (&part)[QP], const T (&f)[QP], T* __restrict__ out) {
    T t[QP], w[QP], y[QP];
#pragma unroll
    for (int c = 0; c < NC; ++c) eo_cell<EO_DT>(f, c * n, t, c * n);
#pragma unroll
    for (int g = 0; g < QP; ++g) w[g] = part[g] + t[g];
#pragma unroll
    for (int c = 0; c < NC; ++c) eo_cell<EO_BT>(w, c * n, y, c * n);
    if constexpr (NC == 1) {
#pragma unroll
      for (int a = 0; a <= Q; ++a) out[loff(a)] = y[a];
    } else {
#pragma unroll
      for (int k = 1; k <= M - 2; ++k)
        out[loff(k - 1)] = (k < Q) ? y[k] : (k == Q ? y[Q] + y[n] : y[n + k - Q]);
    }
  }

  // ---- transposed derivative along the last axis, added to the partial sums
  // in Vp (the other directions), fused with the backward integration along
  // that axis: one item per line (both cells), output [Lo][I].
  // (3D: the partial sums are the two arrays Vp + Vq)
  __device__ __forceinline__ static void dert_bwd_last_item(const T* __restrict__ F, const T* __restrict__ Vp,
                                                            const T* __restrict__ Vq, T* __restrict__ out, int i) {
    const int b = lbase(i);
    T f[QP], part[QP];
#pragma unroll
    for (int g = 0; g < QP; ++g) {
      f[g] = F[loff(g) + b];
      part[g] = Vp[loff(g) + b];
      if (DIM == 3) part[g] += Vq[loff(g) + b];
    }
    last_bwd(part, f, out + b);
  }

  // ---- line-owner stages along the last axis (z in 3D, y in 2D).
  // One thread owns one line (both cells, 2n points); the last-axis gradient
  // and flux of the line stay in its registers between stages.
  static constexpr int NLINE = ipow(QP, DIM - 1);          // lines per block
  static constexpr int LPT = (TM::SPAN * NLINE + TM::TPP - 1) / TM::TPP;  // lines per thread

  // forward interpolation along the last axis + collocation derivative:
  // writes V (point values), keeps the last-axis gradient in gz
  template <bool INTIN>
  __device__ __forceinline__ static void line_fwd(const T* __restrict__ in, T* __restrict__ V, int i, T (&gz)[QP]) {
    const int b = lbase(i);
    T v[M], w[QP];
    load_last<INTIN>(in, b, v);
    interp_line<INTIN>(v, w);
#pragma unroll
    for (int g = 0; g < QP; ++g) V[loff(g) + b] = w[g];
#pragma unroll
    for (int c = 0; c < NC; ++c) eo_cell<EO_D>(w, c * n, gz, c * n);
  }

  // quadrature-point product along one line: F_0 .. F_{d-2} (other-direction
  // gradients in shared memory) and gz (registers) -> fluxes in place / in fz
  template <typename GF>
  __device__ __forceinline__ static void line_quad(T* __restrict__ F, int i, const T (&gz)[QP], T (&fz)[QP],
                                                   const GF& gcell, int pp) {
    constexpr int NGC = D::NGC;
    const int b = lbase(i);
    // position of the line in the other directions
    int cslot0 = 0, lg0 = 0;
    {
      int rem = i, mul = 1, cmul = 1;
#pragma unroll
      for (int ax = 0; ax < DIM - 1; ++ax) {
        const int qa = rem % QP;
        rem /= QP;
        const int ca = (NC == 2) ? (qa >= n) : 0;
        cslot0 += ca * cmul;
        lg0 += (qa - ca * n) * mul;
        cmul *= NC;
        mul *= n;
      }
    }
    constexpr int CSTRIDE = ipow(NC, DIM - 1);   // cell-slot step along the last axis
    constexpr int GSTRIDE = ipow(n, DIM - 1);    // local point step along the last axis
    with_geom_format<T>(gcell, [&](auto packed) {
      constexpr bool PK = decltype(packed)::value;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T* Gc = gcell(pp, cslot0 + c * CSTRIDE) + lg0;
#pragma unroll
        for (int g = 0; g < n; ++g) {
          const int pt = loff(c * n + g) + b;
          T Gv[D::NCOMP];
          gtensor<PK, D::NCOMP, NGC, GF>(Gc + g * GSTRIDE, Gv);
          if (DIM == 3) {
            const T G00 = Gv[0], G01 = Gv[1], G02 = Gv[2], G11 = Gv[3], G12 = Gv[4], G22 = Gv[5];
            const T g0 = F[pt], g1 = F[NQS + pt], g2 = gz[c * n + g];
            F[pt] = G00 * g0 + G01 * g1 + G02 * g2;
            F[NQS + pt] = G01 * g0 + G11 * g1 + G12 * g2;
            fz[c * n + g] = G02 * g0 + G12 * g1 + G22 * g2;
          } else {
            const T G00 = Gv[0], G01 = Gv[1], G11 = Gv[2];
            const T g0 = F[pt], g1 = gz[c * n + g];
            F[pt] = G00 * g0 + G01 * g1;
            fz[c * n + g] = G01 * g0 + G11 * g1;
          }
        }
      }
    });
  }

  // transposed derivative along the last axis (fz in registers) added to the
  // other directions' sums (Vp, and Vq in 3D), then backward integration
  // along that axis: output [Lo][I]
  __device__ __forceinline__ static void line_bwd(const T (&fz)[QP], const T* __restrict__ Vp,
                                                  const T* __restrict__ Vq, T* __restrict__ out, int i) {
    const int b = lbase(i);
    T part[QP];
#pragma unroll
    for (int g = 0; g < QP; ++g) {
      part[g] = Vp[loff(g) + b];
      if (DIM == 3) part[g] += Vq[loff(g) + b];
    }
    last_bwd(part, fz, out + b);
  }

  // ---- collocation derivative along AX (x, or y in 3D) on an array of all
  // points, one line per item
  template <int AX>
  __device__ __forceinline__ static void der_item(const T* __restrict__ in, T* __restrict__ out, int item) {
    const int s = lstart<AX>(item);
    const T* src = in + s;
    T* dst = out + s;
    T v[QP], y[QP];
#pragma unroll
    for (int h = 0; h < QP; ++h) v[h] = src[lstep<AX>(h)];
#pragma unroll
    for (int c = 0; c < NC; ++c) eo_cell<EO_D>(v, c * n, y, c * n);
#pragma unroll
    for (int g = 0; g < QP; ++g) dst[lstep<AX>(g)] = y[g];
  }

  // ---- transposed derivative along AX, written (ACC = false) or added
  template <int AX, bool ACC>
  __device__ __forceinline__ static void dert_item(const T* __restrict__ in, T* __restrict__ out, int item) {
    const int s = lstart<AX>(item);
    const T* src = in + s;
    T* dst = out + s;
    T v[QP], y[QP];
#pragma unroll
    for (int g = 0; g < QP; ++g) v[g] = src[lstep<AX>(g)];
#pragma unroll
    for (int c = 0; c < NC; ++c) eo_cell<EO_DT>(v, c * n, y, c * n);
#pragma unroll
    for (int g = 0; g < QP; ++g) dst[lstep<AX>(g)] = ACC ? dst[lstep<AX>(g)] + y[g] : y[g];
  }

  // ---- transposed derivative along AX in place: the thread reads its whole
  // line before writing it back
  template <int AX>
  __device__ __forceinline__ static void dert_inplace_item(T* __restrict__ F, int item) {
    T* p = F + lstart<AX>(item);
    T v[QP], y[QP];
#pragma unroll
    for (int g = 0; g < QP; ++g) v[g] = p[lstep<AX>(g)];
#pragma unroll
    for (int c = 0; c < NC; ++c) eo_cell<EO_DT>(v, c * n, y, c * n);
#pragma unroll
    for (int g = 0; g < QP; ++g) p[lstep<AX>(g)] = y[g];
  }

  // ---- final backward integration along x: like bwd_item<0, false> but every
  // output value goes through put(pp, index, value) (the apply's epilogue)
  template <typename PUT>
  __device__ __forceinline__ static void bwd0_item(const T* __restrict__ in, int o, int pp, const PUT& put) {
    constexpr int Lout = (NC == 2) ? Mi : M;
    const T* src = in + rowa(o);
    T w[QP];
#pragma unroll
    for (int g = 0; g < QP; ++g) w[g] = src[g];
    integ_line<false>(w, LineEpi<PUT>{put, pp, o * Lout});
  }

  // ---- backward integration along y (3D): [O][QP][QP] -> [O][Lout][QP], one
  // line per item (x = item % QP in plane item / QP).  NC = 2: interior
  // nodes only (Lout = Mi); NC = 1: all nodes (Lout = M).  ACC: add into the
  // output instead of writing.
  template <int AX, bool ACC>
  __device__ __forceinline__ static void bwd_item(const T* __restrict__ in, T* __restrict__ out, int item) {
    static_assert(AX == 1 && DIM == 3, "backward integration along y in 3D");
    constexpr int Lout = (NC == 2) ? Mi : M;
    const int i = item % QP, o = item / QP;
    const T* src = in + lstart<1>(item);
    T w[QP];
#pragma unroll
    for (int g = 0; g < QP; ++g) w[g] = src[lstep<1>(g)];
    integ_line<ACC>(w, LineStore<ACC>{out, o * Lout, i});
  }

  template <bool INTIN, typename GF, typename EPI>
  __device__ __forceinline__ static void apply_line(const T* in, int sin, T* scr, int sscr, const GF& gcell,
                                                    const EPI& epi) {
    constexpr int L = INTIN ? Mi : M;
    constexpr int Lo = (NC == 2) ? Mi : M;
    // scratch: V = scr[0..NQS) (point values, later the transposed sums),
    // R = scr[NQS..): forward temporaries, then F_0 (and F_1 in 3D).
    auto Vp = [&](int pp) { return scr + pp * sscr; };
    auto Rp = [&](int pp) { return scr + pp * sscr + NQS; };
    T gz[LPT][QP], fz[LPT][QP];
    if constexpr (DIM == 3) {
      constexpr int T1 = rowa(L * L);
      TM::template loop<L * L>([&](int pp, int it) { fwd_item<0, INTIN>(in + pp * sin, Rp(pp), it); });
      TM::sync();
      TM::template loop<L * QP>([&](int pp, int it) { fwd_item<1, INTIN>(Rp(pp), Rp(pp) + T1, it); });
      TM::sync();
#pragma unroll
      for (int l = 0; l < LPT; ++l) {
        int pp, line;
        if (TM::template slot<NLINE>(l, pp, line)) {
          line_fwd<INTIN>(Rp(pp) + T1, Vp(pp), line, gz[l]);
        }
      }
      TM::sync();
      constexpr int ND = QP * QP;           // lines per direction
      TM::template loop<2 * ND>([&](int pp, int it) {
        const int ax = it / ND, r = it - ax * ND;
        if (ax == 0) der_item<0>(Vp(pp), Rp(pp), r);
        else der_item<1>(Vp(pp), Rp(pp) + NQS, r);
      });
      TM::sync();
#pragma unroll
      for (int l = 0; l < LPT; ++l) {
        int pp, line;
        if (TM::template slot<NLINE>(l, pp, line)) {
          line_quad(Rp(pp), line, gz[l], fz[l], gcell, pp);
        }
      }
      TM::sync();
      // transposed derivatives along x and y, each in place on its flux array
      TM::template loop<2 * ND>([&](int pp, int it) {
        const int ax = it / ND, r = it - ax * ND;
        if (ax == 0) dert_inplace_item<0>(Rp(pp), r);
        else dert_inplace_item<1>(Rp(pp) + NQS, r);
      });
      TM::sync();
      // z: their sum + D^T of the z flux, integrated along z into V [Lo][QP][QP]
      static_assert(rowa(Lo * QP) <= NQS, "z output exceeds V");
#pragma unroll
      for (int l = 0; l < LPT; ++l) {
        int pp, line;
        if (TM::template slot<NLINE>(l, pp, line)) {
          line_bwd(fz[l], Rp(pp), Rp(pp) + NQS, Vp(pp), line);
        }
      }
      TM::sync();
      TM::template loop<Lo * QP>([&](int pp, int it) { bwd_item<1, false>(Vp(pp), Rp(pp), it); });
      TM::sync();
      TM::template loop<Lo * Lo>([&](int pp, int it) { bwd0_item(Rp(pp), it, pp, epi); });
      TM::sync();
    } else {
      TM::template loop<L>([&](int pp, int it) { fwd_item<0, INTIN>(in + pp * sin, Rp(pp), it); });
      TM::sync();
#pragma unroll
      for (int l = 0; l < LPT; ++l) {
        int pp, line;
        if (TM::template slot<NLINE>(l, pp, line)) {
          line_fwd<INTIN>(Rp(pp), Vp(pp), line, gz[l]);
        }
      }
      TM::sync();
      constexpr int ND = QP;                // lines per direction
      TM::template loop<ND>([&](int pp, int it) { der_item<0>(Vp(pp), Rp(pp), it); });
      TM::sync();
#pragma unroll
      for (int l = 0; l < LPT; ++l) {
        int pp, line;
        if (TM::template slot<NLINE>(l, pp, line)) {
          line_quad(Rp(pp), line, gz[l], fz[l], gcell, pp);
        }
      }
      TM::sync();
      TM::template loop<ND>([&](int pp, int it) { dert_item<0, false>(Rp(pp), Vp(pp), it); });
      TM::sync();
      // R [Lo][QP] (F_0 is dead)
#pragma unroll
      for (int l = 0; l < LPT; ++l) {
        int pp, line;
        if (TM::template slot<NLINE>(l, pp, line)) {
          line_bwd(fz[l], Vp(pp), nullptr, Rp(pp), line);
        }
      }
      TM::sync();
      TM::template loop<Lo>([&](int pp, int it) { bwd0_item(Rp(pp), it, pp, epi); });
      TM::sync();
    }
  }
  // ---- batched stages: every thread takes U items per iteration and issues
  // all their loads before any arithmetic, so the latencies of independent
  // items overlap (one item per thread and iteration leaves them serial).
  static constexpr int U = 2;

  // quadrature-point products over all points of the served blocks (stage design)
  template <typename GF>
  __device__ __forceinline__ static void quad_stage(T* scr, int sscr, const GF& gcell) {
    with_geom_format<T>(gcell, [&](auto packed) { quad_stage_as<decltype(packed)::value>(scr, sscr, gcell); });
  }
  template <bool PK, typename GF>
  __device__ __forceinline__ static void quad_stage_as(T* scr, int sscr, const GF& gcell) {
    constexpr int NGC = D::NGC;
    constexpr int NCOMP = D::NCOMP;
    constexpr int TOT = TM::SPAN * NQ;
    constexpr int STEP = TM::TPP;
#pragma unroll 1
    for (int base = TM::lane(); base < TOT; base += U * STEP) {
      T g[U][DIM], G[U][NCOMP];
      int off[U];
      bool ok[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int it0 = base + u * STEP;
        ok[u] = it0 < TOT;
        const int it = ok[u] ? it0 : base;
        int pp, pt;
        if constexpr (GROUPED) {
          pp = TM::group();
          pt = it;
        } else {
          pp = it / NQ;
          pt = it - pp * NQ;
        }
        int cslot = 0, lg = 0, rem = pt, mul = 1, cmul = 1;
#pragma unroll
        for (int ax = 0; ax < DIM; ++ax) {
          const int qa = rem % QP;
          rem /= QP;
          const int ca = (NC == 2) ? (qa >= n) : 0;
          cslot += ca * cmul;
          lg += (qa - ca * n) * mul;
          cmul *= NC;
          mul *= n;
        }
        const T* Gp = gcell(pp, cslot) + lg;
        off[u] = pp * sscr + NQS + (SKEW ? rowa(pt / QP) + pt % QP : pt);
#pragma unroll
        for (int d = 0; d < DIM; ++d) g[u][d] = scr[off[u] + d * NQS];
        gtensor<PK, NCOMP, NGC, GF>(Gp, G[u]);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (!ok[u]) continue;
        T* F = scr + off[u];
        if (DIM == 3) {
          F[0] = G[u][0] * g[u][0] + G[u][1] * g[u][1] + G[u][2] * g[u][2];
          F[NQS] = G[u][1] * g[u][0] + G[u][3] * g[u][1] + G[u][4] * g[u][2];
          F[2 * NQS] = G[u][2] * g[u][0] + G[u][4] * g[u][1] + G[u][5] * g[u][2];
        } else {
          F[0] = G[u][0] * g[u][0] + G[u][1] * g[u][1];
          F[NQS] = G[u][1] * g[u][0] + G[u][2] * g[u][1];
        }
      }
    }
  }

  // collocation derivative (TRANS = false: out[g] = sum_h D[g][h] v[h]) or its
  // transpose (TRANS = true: out[h] (+)= sum_g D[g][h] v[g]) on every cell of
  // a line, ITEMS lines per block; map(pp, item, src, dst, ax) locates an
  // item's line (its first point in the input and the output, and its
  // direction: 0 = x, 1 = y).
  template <bool TRANS, bool ACC, int ITEMS, typename Map>
  __device__ __forceinline__ static void dseg_stage(const Map& map) {
    constexpr int TOT = TM::SPAN * ITEMS;
    constexpr int STEP = TM::TPP;
#pragma unroll 1
    for (int base = TM::lane(); base < TOT; base += U * STEP) {
      T v[U][QP], a[U][QP];
      T* dst[U];
      int axu[U];
      bool ok[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int it0 = base + u * STEP;
        ok[u] = it0 < TOT;
        const int it = ok[u] ? it0 : base;
        int pp, r;
        if constexpr (GROUPED) {
          pp = TM::group();
          r = it;
        } else {
          pp = it / ITEMS;
          r = it - pp * ITEMS;
        }
        const T* src;
        map(pp, r, src, dst[u], axu[u]);
#pragma unroll
        for (int h = 0; h < QP; ++h) v[u][h] = src[axu[u] ? lstep<1>(h) : h];
        if (ACC) {
#pragma unroll
          for (int h = 0; h < QP; ++h) a[u][h] = dst[u][axu[u] ? lstep<1>(h) : h];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (!ok[u]) continue;
        T y[QP];
#pragma unroll
        for (int c = 0; c < NC; ++c) eo_cell<TRANS ? EO_DT : EO_D>(v[u], c * n, y, c * n);
#pragma unroll
        for (int g = 0; g < QP; ++g) dst[u][axu[u] ? lstep<1>(g) : g] = ACC ? a[u][g] + y[g] : y[g];
      }
    }
  }

  // line r of direction AX (x, or y in 3D) of a block in point arrays
  // starting at in / out
  template <int AX>
  __device__ __forceinline__ static void seg(int r, const T* in, T* out, const T*& src, T*& dst, int& ax) {
    const int offs = lstart<AX>(r);
    src = in + offs;
    dst = out + offs;
    ax = AX;
  }

  template <bool INTIN, typename GF, typename EPI>
  __device__ __forceinline__ static void apply_stage(const T* in, int sin, T* scr, int sscr, const GF& gcell,
                                                     const EPI& epi) {
    constexpr int L = INTIN ? Mi : M;
    constexpr int Lo = (NC == 2) ? Mi : M;
    // scratch: V = scr[0..NQS), R = scr[NQS..); F_ax = R + ax*NQS
    auto Vp = [&](int pp) { return scr + pp * sscr; };
    auto Rp = [&](int pp) { return scr + pp * sscr + NQS; };
    if constexpr (DIM == 3) {
      constexpr int T1 = rowa(L * L);
      TM::template loop<L * L>([&](int pp, int it) { fwd_item<0, INTIN>(in + pp * sin, Rp(pp), it); });
      TM::sync();
      TM::template loop<L * QP>([&](int pp, int it) { fwd_item<1, INTIN>(Rp(pp), Rp(pp) + T1, it); });
      TM::sync();
      // z: interpolate to the Gauss points and differentiate along z in registers;
      // T2 (R + T1) is read while F_2 (R + 2 NQS) is written: 2 NQS >= T1 + T2.
      static_assert(2 * NQS >= rowa(L * L) + rowa(L * QP), "F_2 overlaps the z input");
      TM::template loop<QP * QP>([&](int pp, int it) {
        fwd_der_last_item<INTIN>(Rp(pp) + T1, Vp(pp), Rp(pp) + 2 * NQS, it);
      });
      TM::sync();
      constexpr int ND = QP * QP;           // lines per direction
      dseg_stage<false, false, 2 * ND>([&](int pp, int r2, const T*& src, T*& dst, int& st) {
        const int ax = r2 / ND, r = r2 - ax * ND;
        if (ax == 0) seg<0>(r, Vp(pp), Rp(pp), src, dst, st);
        else seg<1>(r, Vp(pp), Rp(pp) + NQS, src, dst, st);
      });
      TM::sync();
      quad_stage(scr, sscr, gcell);
      TM::sync();
      // transposed derivatives along x and y, each in place on its flux array
      dseg_stage<true, false, 2 * ND>([&](int pp, int r2, const T*& src, T*& dst, int& st) {
        const int ax = r2 / ND, r = r2 - ax * ND;
        if (ax == 0) seg<0>(r, Rp(pp), Rp(pp), src, dst, st);
        else seg<1>(r, Rp(pp) + NQS, Rp(pp) + NQS, src, dst, st);
      });
      TM::sync();
      // z: F_0 + F_1 + D^T F_2 -> B^T along z -> V [Lo][QP][QP]
      static_assert(rowa(Lo * QP) <= NQS, "z output exceeds V");
      TM::template loop<QP * QP>([&](int pp, int it) {
        dert_bwd_last_item(Rp(pp) + 2 * NQS, Rp(pp), Rp(pp) + NQS, Vp(pp), it);
      });
      TM::sync();
      TM::template loop<Lo * QP>([&](int pp, int it) { bwd_item<1, false>(Vp(pp), Rp(pp), it); });
      TM::sync();
      TM::template loop<Lo * Lo>([&](int pp, int it) { bwd0_item(Rp(pp), it, pp, epi); });
      TM::sync();
    } else {
      TM::template loop<L>([&](int pp, int it) { fwd_item<0, INTIN>(in + pp * sin, Rp(pp), it); });
      TM::sync();
      // y: R [L][QP] -> V [QP][QP] and F_1 = R + NQS (R holds rowa(L) <= NQS values)
      static_assert(rowa(L) <= NQS, "F_1 overlaps the y input");
      TM::template loop<QP>([&](int pp, int it) { fwd_der_last_item<INTIN>(Rp(pp), Vp(pp), Rp(pp) + NQS, it); });
      TM::sync();
      constexpr int ND = QP;                // lines per direction
      dseg_stage<false, false, ND>([&](int pp, int r, const T*& src, T*& dst, int& st) {
        seg<0>(r, Vp(pp), Rp(pp), src, dst, st);
      });
      TM::sync();
      quad_stage(scr, sscr, gcell);
      TM::sync();
      dseg_stage<true, false, ND>([&](int pp, int r, const T*& src, T*& dst, int& st) {
        seg<0>(r, Rp(pp), Vp(pp), src, dst, st);
      });
      TM::sync();
      // y: D^T F_1 + V -> B^T along y -> R [Lo][QP] (F_0 = R is dead)
      TM::template loop<QP>([&](int pp, int it) { dert_bwd_last_item(Rp(pp) + NQS, Vp(pp), nullptr, Rp(pp), it); });
      TM::sync();
      TM::template loop<Lo>([&](int pp, int it) { bwd0_item(Rp(pp), it, pp, epi); });
      TM::sync();
    }
  }

  // Full operator A in for PPB blocks, every output value handed to the
  // epilogue epi(pp, index, value) in the final stage (apply: stored, or
  // added, to out); in/scr are per-block base pointers with strides; INTIN:
  // input on interior nodes only.  The input is read in the first stage only,
  // so an epilogue may overwrite it.
  // Not inlined: one copy per (level, input kind) is shared by all call
  // sites, which keeps the patch kernel small for the instruction cache.
  // LINE selects the design of the last direction: false = separate stages
  // with all fluxes in shared memory, true = one thread per line with that
  // direction's gradient and flux in registers.  Ends with __syncthreads().
  // The functors are passed by value and the vectors are re-derived as
  // shared-memory pointers (smem_ptr) on entry, so that nothing of the call
  // goes through local memory or generic addressing.
  template <bool INTIN, typename GF, typename EPI>
  __device__ __noinline__ static void apply_epi(const T* in, int sin, T* scr, int sscr, const GF gcell,
                                                const EPI epi) {
    const T* in_s = smem_ptr(in);
    T* scr_s = smem_ptr(scr);
    const EPI e = epi.rebase();
    if constexpr (LINE) apply_line<INTIN>(in_s, sin, scr_s, sscr, gcell, e);
    else apply_stage<INTIN>(in_s, sin, scr_s, sscr, gcell, e);
  }

  // plain result: out (+)= A in, per block pp at out + pp * sout (shared memory)
  template <bool ACC>
  struct Store {
    T* out;
    int sout;
    __device__ __forceinline__ Store rebase() const { return Store{smem_ptr(out), sout}; }
    __device__ void operator()(int pp, int i, T s) const {
      T* p = out + pp * sout + i;
      *p = ACC ? *p + s : s;
    }
  };

  template <bool INTIN, bool ACC, typename GF>
  __device__ static void apply(const T* in, int sin, T* out, int sout, T* scr, int sscr, const GF& gcell) {
    apply_epi<INTIN>(in, sin, scr, sscr, gcell, Store<ACC>{out, sout});
  }
};

}  // namespace pmg
