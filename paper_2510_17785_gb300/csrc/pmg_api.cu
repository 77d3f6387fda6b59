// C ABI of the library (include/pmg.h): context, structured mesh hierarchy,
// set-up, patch smoother, local p-MG V-cycle, GMG V-cycle and preconditioned
// CG.  Every numerical step runs in the kernels of kern_*.cu; this file holds
// host-side orchestration, the 1D tables and the dense coarse factorisation.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/pmg.h"
#include "basis.h"
#include "device_guard.h"
#include "lanczos_view.h"
#include "umesh.h"
#include "launch.h"
#include "mlp.h"

using namespace pmg;

namespace {

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
};

struct PLevel {
  int q = 0;
  double* G64 = nullptr;
  float* G32 = nullptr;
  float* Gp32 = nullptr;       // the G the FP32 patch kernels read: G32, or G32 rounded to BF16
  unsigned* Gb32 = nullptr;    // geometry_bf16: Gp32 as packed BF16 pairs (what the FP32 patch kernels load)
  double* dinv64 = nullptr;
  float* dinv32 = nullptr;
  double* bounds64 = nullptr;
  float* bounds32 = nullptr;
  double* ritz = nullptr;
  double* dense64 = nullptr;   // small levels: dense patch matrices [patch][Ni][Ni]
  float* dense32 = nullptr;
};

// tabulated local solve of a mesh level (top p-level): [patch][Ni][Ni], (m, k) = (B_j e_m)_k
struct SolveTable {
  double* t64 = nullptr;
  float* t32 = nullptr;
  bool on = false;
};

struct HLevel {
  int N = 0;
  size_t nd = 0;        // (pN+1)^d
  size_t ncells = 0;
  size_t npatch = 0;
  double* coords = nullptr;
  double* kappa = nullptr;
  PLevel pl[8];
  int32_t* colour_list[8] = {nullptr};
  int ncolour[8] = {0};
  std::vector<uint8_t> colours;     // host copy, per patch
  // GMG work vectors
  double *x64 = nullptr, *b64 = nullptr, *r64 = nullptr;
  float *x32 = nullptr, *b32 = nullptr, *r32 = nullptr;
  // transfer tables from level l-1 (fine = this level)
  double* PW = nullptr;
  int* Ps = nullptr;
  double* RW = nullptr;
  int* Rs = nullptr;
  int Rwidth = 0;
};

}  // namespace

struct pmg_ctx {
  int device = 0;
  pmg_options opt{};
  std::string err;
  int dim = 0, N = 0, p = 0, nlev = 0;
  int npl = 0;
  int plevels[8] = {0};
  std::vector<double> h_coords, h_kappa;
  std::vector<std::vector<double>> kappa_level;   // per-level coefficients from pmg_coeff_upload (empty: derived)
  UMesh* um = nullptr;                             // finest unstructured mesh (pmg_mesh_upload), else NULL
  std::vector<UMesh*> umv;                         // unstructured meshes by level (0 = coarsest)
  std::vector<HLevel> L;
  bool mesh_ok = false, setup_ok = false;
  int* d_err = nullptr;
  // coarse solve
  double* Ainv = nullptr;
  int* freeidx = nullptr;
  int nf = 0;
  // transfer temporaries (largest), per precision
  double *t64a = nullptr, *t64b = nullptr;
  float *t32a = nullptr, *t32b = nullptr;
  // user-facing FP32 staging buffers (mixed precision API calls)
  float *s32a = nullptr, *s32b = nullptr;
  // CG
  double *cg_x = nullptr, *cg_r = nullptr, *cg_z = nullptr, *cg_p = nullptr, *cg_Ap = nullptr;
  double *partial = nullptr, *scal = nullptr;
  double* h_rr = nullptr;   // pinned
  double *stage_b = nullptr, *stage_u = nullptr;   // device staging for the host-vector solve
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_caller = nullptr;       // orders the solvers' internal stream after the caller's
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int64_t graph_launches_per_iter = 0;   // kernels recorded in one CG iteration graph
  int64_t launches = 0;                  // kernels launched so far
  int variant = 0;                       // launch shape of the patch-sweep kernel
  float variant_ms[NUM_VARIANTS] = {};   // set-up timings of the finest level (-1: not timed)
  int level_variant[16] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};  // per mesh level
  float level_ms[16][NUM_VARIANTS] = {};  // set-up timings per mesh level (-1: not timed)
  bool level_persist[16] = {};           // sweeps of the level as one persistent launch
  SolveTable solve_table[16];            // tabulated local solves per mesh level
  float dense_ms[16][2] = {};            // set-up: full sweep matrix-free / tabulated (-1: not timed)
  float persist_ms[16][2] = {};          // set-up: full sweep per-colour / persistent (-1: not timed)
  bool any_persist = false;
  unsigned int* d_sync = nullptr;        // grid barrier: count, generation, status
  float* mlp_params = nullptr;           // PMG_BOUNDS_MLP network and normalisation
  float* mlp_norm = nullptr;
  double* add64 = nullptr;               // additive sweeps: correction sums (finest-level size)
  float* add32 = nullptr;
  double* gm_V = nullptr;                // GMRES basis (restart + 1 vectors), grown on demand
  int gm_m = 0;
  double* fdm64[PMG_MAXQ + 1] = {nullptr};   // Cartesian-reinforced tables per degree q (device)
  float* fdm32[PMG_MAXQ + 1] = {nullptr};
  double* lanczos_V = nullptr;           // Lanczos basis scratch, grown on demand, reused
  size_t lanczos_V_n = 0;
  std::vector<void*> allocs;
};

// ---------------------------------------------------------------------------
namespace {

int fail(pmg_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CU(...)                                                                     \
  do {                                                                              \
    cudaError_t e_ = (__VA_ARGS__);                                                 \
    if (e_ != cudaSuccess)                                                          \
      return fail(ctx, PMG_ERR_CUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define ST(...)                                                                   \
  do {                                                                            \
    int s_ = (__VA_ARGS__);                                                       \
    if (s_ != ST_OK) {                                                            \
      if (s_ == ST_CUDA) {                                                        \
        cudaError_t e_ = cudaGetLastError();                                      \
        return fail(ctx, PMG_ERR_CUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)); \
      }                                                                           \
      return fail(ctx, s_, std::string(#__VA_ARGS__) + " failed");                \
    }                                                                             \
  } while (0)

// ST() plus the number of kernels the call launched
#define LK(n, ...)                \
  do {                            \
    ST(__VA_ARGS__);              \
    ctx->launches += (n);         \
  } while (0)

template <typename T>
int dalloc(pmg_ctx* ctx, T** p, size_t n) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess) return fail(ctx, PMG_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  ctx->allocs.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return PMG_OK;
}
#define DALLOC(ptr, n)                        \
  do {                                        \
    int s_ = dalloc(ctx, &(ptr), (n));        \
    if (s_ != PMG_OK) return s_;              \
  } while (0)

// largest coarsest level for the dense FP64 inverse (2 GB matrix; its assembly
// holds nf columns of the coarsest vector, about 2 GB more, during set-up)
constexpr int kMaxCoarseDofs = 16384;

size_t ipow_sz(size_t b, int e) {
  size_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// ---- dispatch on dimension -------------------------------------------------
// launch shape: the one tuned for the mesh level (sweeps), else the context's
template <typename T>
int patch_launch(pmg_ctx* c, int mode, const PatchArgs<T>& a, cudaStream_t s, int level = -1) {
  int v = 0;
  if (mode == MODE_SWEEP)
    v = (level >= 0 && level < 16 && c->level_variant[level] >= 0) ? c->level_variant[level] : c->variant;
  if (c->opt.level_rule == 1 && rules_differ(c->p)) v = VARIANT_PAPER_LEVELS;   // every mode
  return c->dim == 2 ? launch_patch<2, T>(c->p, mode, v, a, s) : launch_patch<3, T>(c->p, mode, v, a, s);
}
template <typename T>
int cell_apply(pmg_ctx* c, int q, const T* u, T* out, const T* G, int N, cudaStream_t s) {
  return c->dim == 2 ? launch_cell_apply<2, T>(q, u, out, G, N, s) : launch_cell_apply<3, T>(q, u, out, G, N, s);
}
template <typename T>
int mask_boundary(pmg_ctx* c, T* x, int M, cudaStream_t s) {
  return c->dim == 2 ? launch_mask_boundary<2, T>(x, M, s) : launch_mask_boundary<3, T>(x, M, s);
}

template <typename T>
const T* Gof(const PLevel& pl);
template <>
const double* Gof<double>(const PLevel& pl) { return pl.G64; }
template <>
const float* Gof<float>(const PLevel& pl) { return pl.G32; }
template <typename T>
const T* GPatchof(const PLevel& pl);
template <>
const double* GPatchof<double>(const PLevel& pl) { return pl.G64; }
template <>
const float* GPatchof<float>(const PLevel& pl) { return pl.Gp32; }
template <typename T>
const unsigned* GPackedof(const PLevel& pl) { return std::is_same<T, float>::value ? pl.Gb32 : nullptr; }
template <typename T>
const T* Dinvof(const PLevel& pl);
template <>
const double* Dinvof<double>(const PLevel& pl) { return pl.dinv64; }
template <>
const float* Dinvof<float>(const PLevel& pl) { return pl.dinv32; }
template <typename T>
const T* Boundsof(const PLevel& pl);
template <>
const double* Boundsof<double>(const PLevel& pl) { return pl.bounds64; }
template <>
const float* Boundsof<float>(const PLevel& pl) { return pl.bounds32; }

template <typename T>
const T* Denseof(const PLevel& pl);
template <>
const double* Denseof<double>(const PLevel& pl) { return pl.dense64; }
template <>
const float* Denseof<float>(const PLevel& pl) { return pl.dense32; }

template <typename T>
const T* Fdmof(const pmg_ctx* c, int q);
template <>
const double* Fdmof<double>(const pmg_ctx* c, int q) { return c->fdm64[q]; }
template <>
const float* Fdmof<float>(const pmg_ctx* c, int q) { return c->fdm32[q]; }

template <typename T>
const T* SolveTableof(const SolveTable& t);
template <>
const double* SolveTableof<double>(const SolveTable& t) { return t.t64; }
template <>
const float* SolveTableof<float>(const SolveTable& t) { return t.t32; }

template <typename T>
PatchArgs<T> patch_args(pmg_ctx* c, int level) {
  PatchArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  HLevel& h = c->L[level];
  a.N = h.N;
  for (int k = 0; k < c->npl; ++k) {
    a.lv[k].fdm = Fdmof<T>(c, c->plevels[k]);
    a.lv[k].G = GPatchof<T>(h.pl[k]);
    a.lv[k].Gb = GPackedof<T>(h.pl[k]);
    a.lv[k].dinv = Dinvof<T>(h.pl[k]);
    a.lv[k].bounds = Boundsof<T>(h.pl[k]);
    a.lv[k].dense = Denseof<T>(h.pl[k]);
  }
  if (level < 16 && c->solve_table[level].on) a.solveop = SolveTableof<T>(c->solve_table[level]);
  a.smoother = c->opt.smoother;
  a.cheb_degree = c->opt.cheb_degree;
  a.omega = c->opt.jacobi_omega;
  a.n_mg = c->opt.n_mg;
  a.err = c->d_err;
  return a;
}

template <typename T>
int sweep_colour(pmg_ctx* ctx, int level, int colour, const T* b, T* u, cudaStream_t s) {
  HLevel& h = ctx->L[level];
  PatchArgs<T> a = patch_args<T>(ctx, level);
  a.list = h.colour_list[colour];
  a.n_items = h.ncolour[colour];
  a.u = u;
  a.b = b;
  LK(1, patch_launch<T>(ctx, MODE_SWEEP, a, s, level));
  return PMG_OK;
}

GridSync grid_sync_of(pmg_ctx* ctx) {
  GridSync g;
  g.count = ctx->d_sync;
  g.gen = ctx->d_sync + 1;
  g.status = reinterpret_cast<int*>(ctx->d_sync + 2);
  g.budget = ctx->opt.sync_budget > 0 ? ctx->opt.sync_budget : (1LL << 31);
  return g;
}

// every colour of the level in one cooperative launch (grid barrier between colours)
template <typename T>
int sweep_persist(pmg_ctx* ctx, int level, const T* b, T* u, bool reverse, cudaStream_t s) {
  HLevel& h = ctx->L[level];
  PersistArgs<T> pa;
  std::memset(&pa, 0, sizeof(pa));
  pa.base = patch_args<T>(ctx, level);
  pa.base.u = u;
  pa.base.b = b;
  const int nc = 1 << ctx->dim;
  for (int c = 0; c < nc; ++c) {
    pa.lists[c] = h.colour_list[c];
    pa.counts[c] = h.ncolour[c];
  }
  pa.n_colours = nc;
  pa.reverse = reverse ? 1 : 0;
  pa.sync = grid_sync_of(ctx);
  int grid = 0;
  LK(1, ctx->dim == 2 ? launch_patch_persist<2, T>(ctx->p, pa, &grid, s)
                      : launch_patch_persist<3, T>(ctx->p, pa, &grid, s));
  return PMG_OK;
}

// bytes of the tabulated local solves of a mesh level
size_t solve_table_bytes(const pmg_ctx* ctx, int level, size_t elem) {
  const size_t ni = ipow_sz(2 * ctx->p - 1, ctx->dim);
  return ctx->L[level].npatch * ni * ni * elem;
}

// tabulate the local solves of a mesh level: one local launch over
// (patch, unit right-hand side) items, whose outputs are the table's rows
template <typename T>
int build_solve_table(pmg_ctx* ctx, int level, T** out) {
  HLevel& h = ctx->L[level];
  const size_t ni = ipow_sz(2 * ctx->p - 1, ctx->dim);
  const size_t items = h.npatch * ni;
  if (items > (size_t)INT32_MAX) return fail(ctx, PMG_ERR_UNSUPPORTED, "local-solve table too large");
  T* B = nullptr;
  CU(cudaMalloc(&B, std::max<size_t>(items * ni, 1) * sizeof(T)));
  PatchArgs<T> a = patch_args<T>(ctx, level);
  a.solveop = nullptr;
  a.unit_rhs = 1;
  a.n_items = (int)items;
  a.d_out = B;
  const int st = patch_launch<T>(ctx, MODE_LOCAL, a, ctx->stream);
  ctx->launches += 1;
  if (st) {
    cudaFree(B);
    return fail(ctx, st == ST_UNSUPPORTED ? PMG_ERR_UNSUPPORTED : PMG_ERR_CUDA, "local-solve table launch failed");
  }
  *out = B;
  return PMG_OK;
}

void free_solve_table(SolveTable& t) {
  if (t.t64) cudaFree(t.t64);
  if (t.t32) cudaFree(t.t32);
  t = SolveTable();
}

// after a synchronisation: a persistent sweep whose barrier wait ran out
int check_sync(pmg_ctx* ctx) {
  if (!ctx->any_persist) return PMG_OK;
  int st = 0;
  CU(cudaMemcpy(&st, ctx->d_sync + 2, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) {
    CU(cudaMemset(ctx->d_sync, 0, 3 * sizeof(unsigned int)));
    return fail(ctx, PMG_ERR_TIMEOUT, "a grid barrier of a persistent sweep ran out of its wait budget");
  }
  return PMG_OK;
}

template <typename T>
T* additive_buffer(pmg_ctx* ctx);
template <>
double* additive_buffer<double>(pmg_ctx* ctx) { return ctx->add64; }
template <>
float* additive_buffer<float>(pmg_ctx* ctx) { return ctx->add32; }

template <typename T>
int sweep(pmg_ctx* ctx, int level, const T* b, T* u, bool reverse, cudaStream_t s) {
  const int nc = 1 << ctx->dim;
  if (ctx->opt.additive) {
    // weighted additive sweep: every colour adds its corrections to `corr`
    // (patches of one colour have disjoint interiors; colours in a fixed
    // order, so the sum is deterministic), all from the residual of the same u
    HLevel& h = ctx->L[level];
    T* corr = additive_buffer<T>(ctx);
    CU(cudaMemsetAsync(corr, 0, h.nd * sizeof(T), s));
    for (int c = 0; c < nc; ++c) {
      PatchArgs<T> a = patch_args<T>(ctx, level);
      a.list = h.colour_list[c];
      a.n_items = h.ncolour[c];
      a.u = u;
      a.b = b;
      a.corr = corr;
      a.weight_residual = reverse ? 1 : 0;
      LK(1, patch_launch<T>(ctx, MODE_SWEEP, a, s, level));
    }
    const int w = reverse ? 0 : 1;
    LK(1, ctx->dim == 2 ? launch_additive_update<2, T>(u, corr, ctx->opt.additive_theta, w, ctx->p, h.N, s)
                        : launch_additive_update<3, T>(u, corr, ctx->opt.additive_theta, w, ctx->p, h.N, s));
    return PMG_OK;
  }
  if (level < 16 && ctx->level_persist[level]) return sweep_persist<T>(ctx, level, b, u, reverse, s);
  for (int i = 0; i < nc; ++i) {
    const int c = reverse ? nc - 1 - i : i;
    int st = sweep_colour<T>(ctx, level, c, b, u, s);
    if (st) return st;
  }
  return PMG_OK;
}

// h-transfers by DIM band sweeps
template <typename T>
int prolongate(pmg_ctx* ctx, int lf, const T* xc, T* xf, T* ta, T* tb, cudaStream_t s) {
  HLevel& f = ctx->L[lf];
  const int p = ctx->p;
  const int Mc = p * ctx->L[lf - 1].N + 1, Mf = p * f.N + 1;
  if (ctx->dim == 2) {
    LK(1, launch_band_sweep<T>(xc, ta, f.PW, f.Ps, p + 1, Mc, Mf, Mc, 1, 1, s));          // x
    LK(1, launch_band_sweep<T>(ta, xf, f.PW, f.Ps, p + 1, Mc, Mf, 1, Mf, 1, s));          // y
  } else {
    LK(1, launch_band_sweep<T>(xc, ta, f.PW, f.Ps, p + 1, Mc, Mf, (size_t)Mc * Mc, 1, 1, s));
    LK(1, launch_band_sweep<T>(ta, tb, f.PW, f.Ps, p + 1, Mc, Mf, Mc, Mf, 1, s));
    LK(1, launch_band_sweep<T>(tb, xf, f.PW, f.Ps, p + 1, Mc, Mf, 1, (size_t)Mf * Mf, 1, s));
  }
  return PMG_OK;
}

template <typename T>
int restrict_(pmg_ctx* ctx, int lf, const T* rf, T* rc, T* ta, T* tb, cudaStream_t s) {
  HLevel& f = ctx->L[lf];
  const int p = ctx->p;
  const int Mc = p * ctx->L[lf - 1].N + 1, Mf = p * f.N + 1;
  const int w = f.Rwidth;
  if (ctx->dim == 2) {
    LK(1, launch_band_sweep<T>(rf, ta, f.RW, f.Rs, w, Mf, Mc, Mf, 1, 1, s));
    LK(1, launch_band_sweep<T>(ta, rc, f.RW, f.Rs, w, Mf, Mc, 1, Mc, 1, s));
  } else {
    LK(1, launch_band_sweep<T>(rf, ta, f.RW, f.Rs, w, Mf, Mc, (size_t)Mf * Mf, 1, 1, s));
    LK(1, launch_band_sweep<T>(ta, tb, f.RW, f.Rs, w, Mf, Mc, Mf, Mc, 1, s));
    LK(1, launch_band_sweep<T>(tb, rc, f.RW, f.Rs, w, Mf, Mc, 1, (size_t)Mc * Mc, 1, s));
  }
  return PMG_OK;
}

template <typename T>
T* Xof(HLevel& h);
template <>
double* Xof<double>(HLevel& h) { return h.x64; }
template <>
float* Xof<float>(HLevel& h) { return h.x32; }
template <typename T>
T* Bof(HLevel& h);
template <>
double* Bof<double>(HLevel& h) { return h.b64; }
template <>
float* Bof<float>(HLevel& h) { return h.b32; }
template <typename T>
T* Rof(HLevel& h);
template <>
double* Rof<double>(HLevel& h) { return h.r64; }
template <>
float* Rof<float>(HLevel& h) { return h.r32; }
template <typename T>
T* TA(pmg_ctx* c);
template <>
double* TA<double>(pmg_ctx* c) { return c->t64a; }
template <>
float* TA<float>(pmg_ctx* c) { return c->t32a; }
template <typename T>
T* TB(pmg_ctx* c);
template <>
double* TB<double>(pmg_ctx* c) { return c->t64b; }
template <>
float* TB<float>(pmg_ctx* c) { return c->t32b; }

// GMG V-cycle on level l: x_l = B_l b_l (both in the level's work vectors)
template <typename T>
int vcycle(pmg_ctx* ctx, int l, cudaStream_t s) {
  HLevel& h = ctx->L[l];
  T* x = Xof<T>(h);
  T* b = Bof<T>(h);
  LK(1, launch_fill<T>(x, h.nd, T(0), s));
  if (l == 0) {
    LK(1, launch_coarse_gemv<T>(ctx->Ainv, ctx->freeidx, ctx->nf, b, x, s));
    return PMG_OK;
  }
  int st = sweep<T>(ctx, l, b, x, false, s);                     // pre-smoothing
  if (st) return st;
  T* r = Rof<T>(h);
  LK(1 + (1 << ctx->dim), cell_apply<T>(ctx, ctx->p, x, r, Gof<T>(h.pl[0]), h.N, s));   // r = b - A x
  LK(1, launch_sub_from<T>(b, r, h.nd, s));
  HLevel& hc = ctx->L[l - 1];
  st = restrict_<T>(ctx, l, r, Bof<T>(hc), TA<T>(ctx), TB<T>(ctx), s);
  if (st) return st;
  st = vcycle<T>(ctx, l - 1, s);
  if (st) return st;
  st = prolongate<T>(ctx, l, Xof<T>(hc), r, TA<T>(ctx), TB<T>(ctx), s);
  if (st) return st;
  LK(1, launch_add_to<T>(r, x, h.nd, s));
  return sweep<T>(ctx, l, b, x, ctx->opt.post_reverse != 0, s);  // post-smoothing
}

// z = M r on the finest level (FP64 in and out)
int precondition(pmg_ctx* ctx, const double* r, double* z, cudaStream_t s) {
  if (ctx->um) return umesh_precondition(ctx->um, r, z, s) ? fail(ctx, PMG_ERR_CUDA, "unstructured V-cycle failed") : PMG_OK;
  const int lf = ctx->nlev - 1;
  HLevel& h = ctx->L[lf];
  if (ctx->opt.precision == PMG_PREC_MIXED) {
    LK(1, launch_cast_d2f(r, h.b32, h.nd, s));
    int st = vcycle<float>(ctx, lf, s);
    if (st) return st;
    LK(1, launch_cast_f2d(h.x32, z, h.nd, s));
  } else {
    CU(cudaMemcpyAsync(h.b64, r, h.nd * sizeof(double), cudaMemcpyDeviceToDevice, s));
    int st = vcycle<double>(ctx, lf, s);
    if (st) return st;
    CU(cudaMemcpyAsync(z, h.x64, h.nd * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  return PMG_OK;
}

// Time every launch-shape variant of the patch-sweep kernel on colour 0 of
// every mesh level (zero vectors; results are discarded) and keep the fastest
// per level: large launches favour occupancy, the small launches of coarse
// levels the latency of one patch.  The finest level's timings are reported.
template <typename T>
int autotune_T(pmg_ctx* ctx) {
  cudaStream_t s = ctx->stream;
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  int st = PMG_OK;
  for (int l = 0; l < 16; ++l)
    for (int v = 0; v < NUM_VARIANTS; ++v) ctx->level_ms[l][v] = -1.f;
  // the paper's level rule has one launch shape, and no persistent form
  const bool paper = ctx->opt.level_rule == 1 && rules_differ(ctx->p);
  for (int l = ctx->nlev - 1; l >= 0 && st == PMG_OK && !paper; --l) {
    HLevel& h = ctx->L[l];
    if (h.npatch == 0 || l >= 16) continue;
    T* u = Xof<T>(h);
    T* b = Bof<T>(h);
    if (cudaMemsetAsync(u, 0, h.nd * sizeof(T), s) != cudaSuccess ||
        cudaMemsetAsync(b, 0, h.nd * sizeof(T), s) != cudaSuccess) {
      st = fail(ctx, PMG_ERR_CUDA, "autotune: memset failed");
      break;
    }
    float best = 1e30f;
    int bestv = 0;
    for (int v = 0; v < NUM_VARIANTS && st == PMG_OK; ++v) {
      size_t sm;
      int ppb, nt;
      if (ctx->dim == 2) patch_config<2, T>(ctx->p, v, &sm, &ppb, &nt);
      else patch_config<3, T>(ctx->p, v, &sm, &ppb, &nt);
      if (sm == 0) continue;
      if (ctx->opt.autotune == 2 && (v == 3 || v == 6)) continue;   // throughput mode: no latency shapes
      ctx->level_variant[l] = v;
      st = sweep_colour<T>(ctx, l, 0, b, u, s);          // warm-up (and kernel attribute)
      float ms = 1e30f;
      for (int rep = 0; rep < 3 && st == PMG_OK; ++rep) {
        float t = 0.f;
        if (cudaEventRecord(e0, s) != cudaSuccess) st = fail(ctx, PMG_ERR_CUDA, "autotune: event");
        if (st == PMG_OK) st = sweep_colour<T>(ctx, l, 0, b, u, s);
        if (st == PMG_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
          st = fail(ctx, PMG_ERR_CUDA, "autotune: event");
        ms = std::min(ms, t);
      }
      if (l == ctx->nlev - 1) ctx->variant_ms[v] = ms;
      ctx->level_ms[l][v] = ms;
      if (ms < best) {
        best = ms;
        bestv = v;
      }
    }
    ctx->level_variant[l] = bestv;
    if (l == ctx->nlev - 1) ctx->variant = bestv;
  }
  // persistent sweeps: one full sweep each way, the faster kept
  for (int l = ctx->nlev - 1; l >= 0 && st == PMG_OK; --l) {
    HLevel& h = ctx->L[l];
    ctx->persist_ms[l][0] = ctx->persist_ms[l][1] = -1.f;
    if (h.npatch == 0 || l >= 16 || ctx->opt.persistent == 0 || ctx->opt.additive || paper) continue;
    if (ctx->opt.persistent == 1 && (h.npatch > 4096 || ctx->opt.autotune == 2)) continue;
    T* u = Xof<T>(h);
    T* b = Bof<T>(h);
    float ms[2] = {1e30f, 1e30f};
    bool ok = true;
    for (int mode = 0; mode < 2 && st == PMG_OK && ok; ++mode) {
      ctx->level_persist[l] = mode == 1;
      ctx->any_persist = ctx->any_persist || mode == 1;
      int r = sweep<T>(ctx, l, b, u, false, s);                // warm-up
      if (r != PMG_OK) {
        if (mode == 1) {                                       // no co-resident grid: per-colour launches
          cudaGetLastError();
          ok = false;
          break;
        }
        st = r;
        break;
      }
      for (int rep = 0; rep < 3 && st == PMG_OK; ++rep) {
        float t = 0.f;
        if (cudaEventRecord(e0, s) != cudaSuccess) st = fail(ctx, PMG_ERR_CUDA, "autotune: event");
        if (st == PMG_OK) st = sweep<T>(ctx, l, b, u, false, s);
        if (st == PMG_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
          st = fail(ctx, PMG_ERR_CUDA, "autotune: event");
        ms[mode] = std::min(ms[mode], t);
      }
    }
    if (st == PMG_OK && ok) st = check_sync(ctx);
    ctx->persist_ms[l][0] = ms[0];
    ctx->persist_ms[l][1] = ok ? ms[1] : -1.f;
    ctx->level_persist[l] = ok && (ctx->opt.persistent == 2 || ms[1] < ms[0]);
  }
  // tabulated local solves: one full sweep each way, the faster kept
  for (int l = ctx->nlev - 1; l >= 0 && st == PMG_OK; --l) {
    HLevel& h = ctx->L[l];
    if (l >= 16) continue;
    ctx->dense_ms[l][0] = ctx->dense_ms[l][1] = -1.f;
    if (h.npatch == 0 || ctx->opt.dense_local == 0 || solve_table_bytes(ctx, l, sizeof(T)) > (size_t(2) << 30))
      continue;
    T* tab = nullptr;
    st = build_solve_table<T>(ctx, l, &tab);
    if (st) break;
    SolveTable& t = ctx->solve_table[l];
    if constexpr (sizeof(T) == 8) t.t64 = reinterpret_cast<double*>(tab);
    else t.t32 = reinterpret_cast<float*>(tab);
    T* u = Xof<T>(h);
    T* b = Bof<T>(h);
    float ms[2] = {1e30f, 1e30f};
    for (int mode = 0; mode < 2 && st == PMG_OK; ++mode) {
      t.on = mode == 1;
      st = sweep<T>(ctx, l, b, u, false, s);                 // warm-up
      for (int rep = 0; rep < 3 && st == PMG_OK; ++rep) {
        float tm = 0.f;
        if (cudaEventRecord(e0, s) != cudaSuccess) st = fail(ctx, PMG_ERR_CUDA, "autotune: event");
        if (st == PMG_OK) st = sweep<T>(ctx, l, b, u, false, s);
        if (st == PMG_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&tm, e0, e1) != cudaSuccess))
          st = fail(ctx, PMG_ERR_CUDA, "autotune: event");
        ms[mode] = std::min(ms[mode], tm);
      }
    }
    if (st == PMG_OK) st = check_sync(ctx);
    ctx->dense_ms[l][0] = ms[0];
    ctx->dense_ms[l][1] = ms[1];
    t.on = ctx->opt.dense_local == 2 || ms[1] < ms[0];
    if (!t.on) free_solve_table(t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

int autotune(pmg_ctx* ctx) {
  for (int v = 0; v < NUM_VARIANTS; ++v) ctx->variant_ms[v] = -1.f;
  for (int l = 0; l < 16; ++l)
    for (int v = 0; v < NUM_VARIANTS; ++v) ctx->level_ms[l][v] = -1.f;
  for (int l = 0; l < 16; ++l) ctx->persist_ms[l][0] = ctx->persist_ms[l][1] = -1.f;
  for (int l = 0; l < 16; ++l) ctx->dense_ms[l][0] = ctx->dense_ms[l][1] = -1.f;
  if (!ctx->opt.autotune) {
    if (ctx->opt.persistent == 2 && !ctx->opt.additive && !(ctx->opt.level_rule == 1 && rules_differ(ctx->p))) {
      for (int l = 0; l < ctx->nlev && l < 16; ++l) ctx->level_persist[l] = ctx->L[l].npatch > 0;
      ctx->any_persist = true;
    }
    if (ctx->opt.dense_local == 2) {
      const bool mixed = ctx->opt.precision == PMG_PREC_MIXED;
      for (int l = 0; l < ctx->nlev && l < 16; ++l) {
        if (ctx->L[l].npatch == 0 || solve_table_bytes(ctx, l, mixed ? 4 : 8) > (size_t(2) << 30)) continue;
        SolveTable& t = ctx->solve_table[l];
        const int st = mixed ? build_solve_table<float>(ctx, l, &t.t32) : build_solve_table<double>(ctx, l, &t.t64);
        if (st) return st;
        t.on = true;
      }
    }
    ctx->variant = ctx->opt.variant;
    size_t sm;
    int ppb, nt;
    const bool mixed = ctx->opt.precision == PMG_PREC_MIXED;     // the sweeps' precision decides
    if (ctx->dim == 2) {
      if (mixed) patch_config<2, float>(ctx->p, ctx->variant, &sm, &ppb, &nt);
      else patch_config<2, double>(ctx->p, ctx->variant, &sm, &ppb, &nt);
    } else {
      if (mixed) patch_config<3, float>(ctx->p, ctx->variant, &sm, &ppb, &nt);
      else patch_config<3, double>(ctx->p, ctx->variant, &sm, &ppb, &nt);
    }
    if (sm == 0) return fail(ctx, PMG_ERR_UNSUPPORTED, "this launch-shape variant does not exist for this degree");
    return PMG_OK;
  }
  if (ctx->opt.precision == PMG_PREC_MIXED) return autotune_T<float>(ctx);
  return autotune_T<double>(ctx);
}

}  // namespace

// ===========================================================================
// Every entry point that touches the device makes the context's device
// current and restores the caller's on return.
#define PMG_GUARD_DEV(dev)                          \
  pmg::DeviceGuard pmg_device_guard_(dev);          \
  if (pmg_device_guard_.err != cudaSuccess) return PMG_ERR_CUDA
#define PMG_GUARD_CTX(ctx) PMG_GUARD_DEV((ctx)->device)

extern "C" {

void pmg_default_options(pmg_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->smoother = PMG_SMOOTHER_CHEBYSHEV;
  o->cheb_degree = 3;
  o->jacobi_omega = 0.5;
  o->n_mg = 1;
  o->bounds = PMG_BOUNDS_LANCZOS;
  o->lanczos_steps = 16;
  o->bound_safety = 1.1;
  o->bound_ratio = 10.0;
  o->fixed_lo = 0.2;
  o->fixed_hi = 2.0;
  o->seed = 0;
  o->precision = PMG_PREC_FP64;
  o->autotune = 1;
  o->variant = 0;
  o->mlp_safety = 1.2;
  o->coarse_kappa = PMG_KAPPA_ARITHMETIC;
  o->post_reverse = 1;
  o->additive = 0;
  o->additive_theta = 1.0;
  o->persistent = 1;
  o->sync_budget = 0;
  o->geometry_bf16 = 0;
  o->dense_local = 1;
  o->level_rule = 0;
}

int pmg_create(int device, const pmg_options* opt, pmg_ctx** out) {
  if (!out) return PMG_ERR_ARG;
  *out = nullptr;
  pmg_ctx* ctx = new pmg_ctx();
  ctx->device = device;
  if (opt) ctx->opt = *opt;
  else pmg_default_options(&ctx->opt);
  const pmg_options& o = ctx->opt;
  if (o.cheb_degree < 1 || o.cheb_degree > 8 || o.n_mg < 1 || o.lanczos_steps < 1 || o.lanczos_steps > 64 ||
      (o.smoother < 0 || o.smoother > 2) || (o.precision != 0 && o.precision != 1) || o.bounds < 0 ||
      (o.additive != 0 && o.additive != 1) || !(o.additive_theta > 0) ||
      o.bounds > 3 || !(o.bound_safety > 0) || !(o.mlp_safety > 0) || o.coarse_kappa < 0 || o.coarse_kappa > 2 || !(o.bound_ratio >= 1) || o.variant < 0 ||
      o.variant >= NUM_VARIANTS || (o.additive != 0 && o.additive != 1) || !(o.additive_theta > 0) ||
      o.persistent < 0 || o.persistent > 2 || o.sync_budget < 0 || o.geometry_bf16 < 0 || o.geometry_bf16 > 1 ||
      (o.geometry_bf16 && o.precision != PMG_PREC_MIXED) || o.dense_local < 0 || o.dense_local > 2 ||
      o.level_rule < 0 || o.level_rule > 1) {
    delete ctx;
    return PMG_ERR_ARG;
  }
  pmg::DeviceGuard guard(device);
  if (guard.err != cudaSuccess) {
    delete ctx;
    return PMG_ERR_CUDA;
  }
  if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&ctx->d_err, sizeof(int)) != cudaSuccess || cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&ctx->d_sync, 3 * sizeof(unsigned int)) != cudaSuccess ||
      cudaMemset(ctx->d_sync, 0, 3 * sizeof(unsigned int)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_rr, sizeof(double)) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_caller, cudaEventDisableTiming) != cudaSuccess) {
    delete ctx;
    return PMG_ERR_CUDA;
  }
  *out = ctx;
  return PMG_OK;
}

int pmg_destroy(pmg_ctx* ctx) {
  if (!ctx) return PMG_ERR_ARG;
  pmg::DeviceGuard guard(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  for (void* p : ctx->allocs) cudaFree(p);
  if (ctx->lanczos_V) cudaFree(ctx->lanczos_V);
  if (ctx->gm_V) cudaFree(ctx->gm_V);
  if (ctx->d_err) cudaFree(ctx->d_err);
  if (ctx->d_sync) cudaFree(ctx->d_sync);
  for (auto& t : ctx->solve_table) free_solve_table(t);
  if (ctx->h_rr) cudaFreeHost(ctx->h_rr);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  if (ctx->ev_caller) cudaEventDestroy(ctx->ev_caller);
  for (UMesh* m : ctx->umv) umesh_destroy(m);
  delete ctx;
  return PMG_OK;
}

const char* pmg_last_error(const pmg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int pmg_mesh_structured(pmg_ctx* ctx, int dim, int N, int p, int n_levels, const double* coords,
                        const double* kappa) {
  if (!ctx) return PMG_ERR_ARG;
  if (dim != 2 && dim != 3) return fail(ctx, PMG_ERR_ARG, "dim must be 2 or 3");
  if (p < 1 || p > 8) return fail(ctx, PMG_ERR_UNSUPPORTED, "degree must be in 1..8");
  if (n_levels < 1 || N < 2 || !coords || !kappa) return fail(ctx, PMG_ERR_ARG, "bad mesh arguments");
  if (N % (1 << (n_levels - 1)) != 0) return fail(ctx, PMG_ERR_ARG, "N must be divisible by 2^(n_levels-1)");
  if (N / (1 << (n_levels - 1)) < 2) return fail(ctx, PMG_ERR_ARG, "coarsest mesh needs at least 2 cells per direction");
  if (ctx->mesh_ok) return fail(ctx, PMG_ERR_ARG, "mesh already uploaded");
  size_t sz, pb;
  int ppb, nt;
  if (dim == 2) patch_config<2, double>(p, 0, &sz, &ppb, &nt);
  else patch_config<3, double>(p, 0, &sz, &ppb, &nt);
  size_t sz32;
  if (dim == 2) patch_config<2, float>(p, 0, &sz32, &ppb, &nt);
  else patch_config<3, float>(p, 0, &sz32, &ppb, &nt);
  (void)pb;
  if ((ctx->opt.precision == PMG_PREC_FP64 && sz == 0) || sz32 == 0)
    return fail(ctx, PMG_ERR_UNSUPPORTED, "patch working set of this degree does not fit in shared memory in this precision");
  ctx->dim = dim;
  ctx->N = N;
  ctx->p = p;
  ctx->nlev = n_levels;
  ctx->npl = 0;
  for (int q = p; q >= 1; q = coarse_degree(q, ctx->opt.level_rule)) ctx->plevels[ctx->npl++] = q;
  if (ctx->opt.level_rule == 1 && rules_differ(p)) {
    size_t s64 = 0, s32 = 0;
    if (dim == 2) {
      patch_config<2, double>(p, VARIANT_PAPER_LEVELS, &s64, &ppb, &nt);
      patch_config<2, float>(p, VARIANT_PAPER_LEVELS, &s32, &ppb, &nt);
    } else {
      patch_config<3, double>(p, VARIANT_PAPER_LEVELS, &s64, &ppb, &nt);
      patch_config<3, float>(p, VARIANT_PAPER_LEVELS, &s32, &ppb, &nt);
    }
    if ((ctx->opt.precision == PMG_PREC_FP64 ? s64 : s32) == 0)
      return fail(ctx, PMG_ERR_UNSUPPORTED, "the paper's level rule is not built for this degree and precision");
  }
  const size_t nv = ipow_sz(N + 1, dim), nc = ipow_sz(N, dim);
  ctx->h_coords.assign(coords, coords + nv * dim);
  ctx->h_kappa.assign(kappa, kappa + nc);
  for (size_t i = 0; i < nc; ++i)
    if (!std::isfinite(kappa[i]) || !(kappa[i] > 0)) return fail(ctx, PMG_ERR_ARG, "kappa must be positive and finite");
  for (size_t i = 0; i < nv * dim; ++i)
    if (!std::isfinite(coords[i])) return fail(ctx, PMG_ERR_ARG, "coordinates must be finite");
  ctx->mesh_ok = true;
  return PMG_OK;
}

int pmg_set_degree(pmg_ctx* ctx, int p) {
  if (!ctx) return PMG_ERR_ARG;
  if (ctx->setup_ok) return fail(ctx, PMG_ERR_ARG, "already set up");
  if (ctx->mesh_ok && !ctx->um) return fail(ctx, PMG_ERR_ARG, "a structured mesh carries its own degree");
  if (p < 1 || p > 8) return fail(ctx, PMG_ERR_UNSUPPORTED, "degree must be in 1..8");
  if (ctx->opt.level_rule != 0)
    return fail(ctx, PMG_ERR_UNSUPPORTED, "unstructured meshes: the halving level rule only");
  ctx->p = p;
  ctx->npl = 0;
  for (int q = p; q >= 1; q >>= 1) ctx->plevels[ctx->npl++] = q;
  return PMG_OK;
}

int pmg_mesh_upload(pmg_ctx* ctx, int level, int dim, int64_t n_vertices, const double* coords, int64_t n_cells,
                    const int64_t* cell_vertices, const uint8_t* vertex_on_boundary, const int64_t* parent_cell,
                    const uint8_t* child_index) {
  if (!ctx) return PMG_ERR_ARG;
  if (ctx->setup_ok) return fail(ctx, PMG_ERR_ARG, "already set up");
  if (ctx->mesh_ok && !ctx->um) return fail(ctx, PMG_ERR_ARG, "a structured mesh was uploaded");
  const int have = (int)ctx->umv.size();
  if (level != have) return fail(ctx, PMG_ERR_ARG, "upload the mesh levels in order, coarsest (level 0) first");
  if (level >= 16) return fail(ctx, PMG_ERR_UNSUPPORTED, "at most 16 mesh levels");
  if ((level == 0) != (parent_cell == nullptr) || (level == 0) != (child_index == nullptr))
    return fail(ctx, PMG_ERR_ARG, "parent_cell and child_index: NULL on level 0, given on finer levels");
  if ((dim != 2 && dim != 3) || n_vertices < 1 || n_cells < 1 || !coords || !cell_vertices)
    return fail(ctx, PMG_ERR_ARG, "bad mesh arguments");
  if (n_vertices > INT32_MAX || n_cells > INT32_MAX) return fail(ctx, PMG_ERR_UNSUPPORTED, "mesh too large");
  if (ctx->opt.additive || ctx->opt.smoother == PMG_SMOOTHER_CARTESIAN)
    return fail(ctx, PMG_ERR_UNSUPPORTED,
                "unstructured meshes: multiplicative sweeps with the Chebyshev or Jacobi local smoother");
  std::string msg;
  UMesh* m = umesh_create(dim, n_vertices, coords, n_cells, cell_vertices, vertex_on_boundary, &msg);
  if (!m) return fail(ctx, PMG_ERR_ARG, msg);
  if (level > 0 && umesh_set_parent(m, ctx->umv[level - 1], parent_cell, child_index, &msg)) {
    umesh_destroy(m);
    return fail(ctx, PMG_ERR_ARG, msg);
  }
  ctx->umv.push_back(m);
  ctx->um = m;
  ctx->dim = dim;
  ctx->nlev = level + 1;
  ctx->N = 0;
  ctx->mesh_ok = true;
  return PMG_OK;
}

int pmg_get_dof_map(pmg_ctx* ctx, int k, int32_t* out) {
  if (!ctx || !out) return PMG_ERR_ARG;
  if (!ctx->um || !ctx->setup_ok) return fail(ctx, PMG_ERR_ARG, "an unstructured mesh after pmg_setup");
  if (umesh_cell_dofs(ctx->um, k, out)) return fail(ctx, PMG_ERR_ARG, "p-level out of range");
  return PMG_OK;
}

int pmg_local_size(const pmg_ctx* ctx, int level, int64_t* n) {
  if (!ctx || !n || !ctx->setup_ok || level < 0 || level >= ctx->nlev) return PMG_ERR_ARG;
  *n = ctx->um ? umesh_interior_max(ctx->umv[level]) : (int64_t)ipow_sz(2 * ctx->p - 1, ctx->dim);
  return PMG_OK;
}

int pmg_coeff_upload(pmg_ctx* ctx, int level, const double* kappa) {
  if (!ctx) return PMG_ERR_ARG;
  if (!ctx->mesh_ok) return fail(ctx, PMG_ERR_ARG, "upload a mesh first");
  if (ctx->setup_ok) return fail(ctx, PMG_ERR_ARG, "coefficients must be uploaded before pmg_setup");
  if (level < 0 || level >= ctx->nlev || !kappa) return fail(ctx, PMG_ERR_ARG, "bad level or null array");
  if (ctx->um) {
    if (umesh_set_kappa(ctx->umv[level], kappa)) return fail(ctx, PMG_ERR_ARG, "kappa must be positive and finite");
    return PMG_OK;
  }
  const size_t nc = ipow_sz(ctx->N >> (ctx->nlev - 1 - level), ctx->dim);
  for (size_t i = 0; i < nc; ++i)
    if (!std::isfinite(kappa[i]) || !(kappa[i] > 0)) return fail(ctx, PMG_ERR_ARG, "kappa must be positive and finite");
  if ((int)ctx->kappa_level.size() < ctx->nlev) ctx->kappa_level.resize(ctx->nlev);
  ctx->kappa_level[level].assign(kappa, kappa + nc);
  return PMG_OK;
}

int pmg_setup(pmg_ctx* ctx) {
  if (!ctx || !ctx->mesh_ok) return fail(ctx, PMG_ERR_ARG, "upload a mesh first");
  if (ctx->setup_ok) return fail(ctx, PMG_ERR_ARG, "already set up");
  PMG_GUARD_CTX(ctx);
  const int d = ctx->dim, p = ctx->p;
  cudaStream_t s = ctx->stream;
  {
    Tables<double> t64;
    Tables<float> t32;
    Rules r;
    build_tables(t64, t32, r);
    const int e = upload_all_tables(t64, t32, r);
    if (e != 0) return fail(ctx, PMG_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString((cudaError_t)e));
  }
  const bool mixed = ctx->opt.precision == PMG_PREC_MIXED;
  if (ctx->um) {
    if (ctx->p < 1) return fail(ctx, PMG_ERR_ARG, "set the degree first (pmg_set_degree)");
    if (ctx->opt.bounds == PMG_BOUNDS_MLP)
      return fail(ctx, PMG_ERR_UNSUPPORTED,
                  "unstructured meshes: Lanczos, fixed or user-given Chebyshev intervals (pmg_set_bounds)");
    if (ctx->opt.bounds == PMG_BOUNDS_LANCZOS && (ctx->opt.lanczos_steps < 1 || ctx->opt.lanczos_steps > 64))
      return fail(ctx, PMG_ERR_ARG, "lanczos_steps must be in 1..64");
    UOptions o;
    o.precision = ctx->opt.precision;
    o.smoother = ctx->opt.smoother;
    o.cheb_degree = ctx->opt.cheb_degree;
    o.omega = ctx->opt.jacobi_omega;
    o.n_mg = ctx->opt.n_mg;
    o.fixed_lo = ctx->opt.fixed_lo;
    o.fixed_hi = ctx->opt.fixed_hi;
    o.seed = ctx->opt.seed;
    // a coarser mesh without a coefficient of its own takes the mean of its children's
    for (int l = ctx->nlev - 2; l >= 0; --l)
      if (!umesh_kappa_given(ctx->umv[l])) umesh_kappa_from_children(ctx->umv[l], ctx->umv[l + 1]);
    for (int l = 0; l < ctx->nlev; ++l) {
      CU(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s));
      std::string msg;
      o.coarse_space = l == 0;                       // the Q1 space of the coarsest mesh only
      int ust = umesh_setup(ctx->umv[l], ctx->p, o, s, ctx->d_err, &msg);
      if (!ust && l > 0) ust = umesh_link(ctx->umv[l], s, &msg);
      if (ust == ST_DEGENERATE) return fail(ctx, PMG_ERR_DEGENERATE, msg);
      if (ust == ST_UNSUPPORTED) return fail(ctx, PMG_ERR_UNSUPPORTED, msg);
      if (ust == ST_ARG) return fail(ctx, PMG_ERR_ARG, msg);
      if (ust) return fail(ctx, PMG_ERR_CUDA, msg.empty() ? "unstructured set-up failed" : msg);
    }
    const size_t n = (size_t)umesh_ndofs(ctx->um);
    DALLOC(ctx->cg_x, n);
    DALLOC(ctx->cg_r, n);
    DALLOC(ctx->cg_z, n);
    DALLOC(ctx->cg_p, n);
    DALLOC(ctx->cg_Ap, n);
    DALLOC(ctx->stage_b, n);
    DALLOC(ctx->stage_u, n);
    DALLOC(ctx->partial, DOT_BLOCKS);
    DALLOC(ctx->scal, S_NSLOT);
    if (ctx->opt.bounds == PMG_BOUNDS_LANCZOS)
      for (UMesh* m : ctx->umv)
        if (umesh_lanczos(m, ctx->opt.lanczos_steps, ctx->opt.seed, ctx->opt.bound_safety, ctx->opt.bound_ratio, s))
          return fail(ctx, PMG_ERR_CUDA, "unstructured Lanczos intervals failed");
    ctx->setup_ok = true;
    CU(cudaStreamSynchronize(s));
    return PMG_OK;
  }
  // ---- levels: coordinates (even-index subsampling), kappa (mean of children)
  ctx->L.assign(ctx->nlev, HLevel());
  std::vector<double> X = ctx->h_coords, K = ctx->h_kappa;
  for (int l = ctx->nlev - 1; l >= 0; --l) {
    HLevel& h = ctx->L[l];
    h.N = ctx->N >> (ctx->nlev - 1 - l);
    const int Nl = h.N;
    if (l < ctx->nlev - 1) {
      const int Nf = 2 * Nl;
      std::vector<double> Xc(ipow_sz(Nl + 1, d) * d), Kc(ipow_sz(Nl, d), 0.0);
      for (size_t v = 0; v < ipow_sz(Nl + 1, d); ++v) {
        size_t rem = v, fid = 0, mul = 1;
        for (int ax = 0; ax < d; ++ax) {
          const size_t i = rem % (Nl + 1);
          rem /= (Nl + 1);
          fid += 2 * i * mul;
          mul *= (Nf + 1);
        }
        for (int k = 0; k < d; ++k) Xc[v * d + k] = X[fid * d + k];
      }
      for (size_t c = 0; c < ipow_sz(Nl, d); ++c) {
        size_t rem = c;
        int ci[3] = {0, 0, 0};
        for (int ax = 0; ax < d; ++ax) { ci[ax] = (int)(rem % Nl); rem /= Nl; }
        double sum = 0.0;
        const int rule = ctx->opt.coarse_kappa;
        for (int ch = 0; ch < (1 << d); ++ch) {
          size_t fid = 0, mul = 1;
          for (int ax = 0; ax < d; ++ax) { fid += (size_t)(2 * ci[ax] + ((ch >> ax) & 1)) * mul; mul *= Nf; }
          sum += rule == PMG_KAPPA_GEOMETRIC ? std::log(K[fid]) : (rule == PMG_KAPPA_HARMONIC ? 1.0 / K[fid] : K[fid]);
        }
        const double m = sum / (1 << d);
        Kc[c] = rule == PMG_KAPPA_GEOMETRIC ? std::exp(m) : (rule == PMG_KAPPA_HARMONIC ? 1.0 / m : m);
      }
      X.swap(Xc);
      K.swap(Kc);
    }
    if (l < (int)ctx->kappa_level.size() && !ctx->kappa_level[l].empty()) K = ctx->kappa_level[l];
    h.nd = ipow_sz((size_t)p * Nl + 1, d);
    h.ncells = ipow_sz(Nl, d);
    h.npatch = ipow_sz(Nl - 1, d);
    DALLOC(h.coords, X.size());
    DALLOC(h.kappa, K.size());
    CU(cudaMemcpy(h.coords, X.data(), X.size() * sizeof(double), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h.kappa, K.data(), K.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  // ---- geometry tensors and level diagonals
  double* diag = nullptr;
  DALLOC(diag, ctx->L.back().nd);
  for (int l = 0; l < ctx->nlev; ++l) {
    HLevel& h = ctx->L[l];
    for (int k = 0; k < ctx->npl; ++k) {
      PLevel& pl = h.pl[k];
      pl.q = ctx->plevels[k];
      const int q = pl.q;
      const size_t ng = h.ncells * (size_t)(d * (d + 1) / 2) * ipow_sz(q + 1, d);
      const size_t ndq = ipow_sz((size_t)q * h.N + 1, d);
      DALLOC(pl.G64, ng);
      DALLOC(pl.dinv64, ndq);
      DALLOC(pl.dinv32, ndq);
      if (d == 2) ST(launch_geometry<2, double>(h.coords, h.kappa, h.N, q, pl.G64, ctx->d_err, s));
      else ST(launch_geometry<3, double>(h.coords, h.kappa, h.N, q, pl.G64, ctx->d_err, s));
      if (mixed) {
        DALLOC(pl.G32, ng);
        if (d == 2) ST(launch_geometry<2, float>(h.coords, h.kappa, h.N, q, pl.G32, ctx->d_err, s));
        else ST(launch_geometry<3, float>(h.coords, h.kappa, h.N, q, pl.G32, ctx->d_err, s));
        pl.Gp32 = pl.G32;
        if (ctx->opt.geometry_bf16) {
          DALLOC(pl.Gp32, ng);
          ST(launch_round_bf16(pl.G32, pl.Gp32, ng, s));
          const int ncomp = d * (d + 1) / 2;
          DALLOC(pl.Gb32, h.ncells * (size_t)((ncomp + 1) / 2) * ipow_sz(q + 1, d));
          ST(launch_pack_bf16(pl.Gp32, pl.Gb32, h.ncells, ncomp, (int)ipow_sz(q + 1, d), s));
        }
      }
      if (d == 2) ST(launch_diag<2>(pl.G64, h.N, q, diag, pl.dinv64, pl.dinv32, s));
      else ST(launch_diag<3>(pl.G64, h.N, q, diag, pl.dinv64, pl.dinv32, s));
      if (dense_level(d, q) && h.npatch > 0) {
        const size_t ni = ipow_sz(2 * q - 1, d);
        DALLOC(pl.dense64, h.npatch * ni * ni);
        if (d == 2) ST(launch_dense_patch<2>(q, pl.G64, h.N, 0, (int)h.npatch, pl.dense64, s));
        else ST(launch_dense_patch<3>(q, pl.G64, h.N, 0, (int)h.npatch, pl.dense64, s));
        if (mixed) {
          DALLOC(pl.dense32, h.npatch * ni * ni);
          ST(launch_cast_d2f(pl.dense64, pl.dense32, h.npatch * ni * ni, s));
        }
      }
      DALLOC(pl.bounds64, 2 * std::max<size_t>(h.npatch, 1));
      DALLOC(pl.bounds32, 2 * std::max<size_t>(h.npatch, 1));
      DALLOC(pl.ritz, 2 * std::max<size_t>(h.npatch, 1));
      CU(cudaMemsetAsync(pl.ritz, 0, 2 * std::max<size_t>(h.npatch, 1) * sizeof(double), s));
    }
  }
  int herr = 0;
  CU(cudaMemcpyAsync(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (herr) return fail(ctx, PMG_ERR_DEGENERATE, "det J <= 0 at a Gauss point of some cell");
  // ---- patches and colours (colour bit k = parity of the vertex index k)
  for (int l = 0; l < ctx->nlev; ++l) {
    HLevel& h = ctx->L[l];
    const int Nv = h.N - 1;
    std::vector<std::vector<int32_t>> lists(1 << d);
    h.colours.assign(h.npatch, 0);
    for (size_t j = 0; j < h.npatch; ++j) {
      size_t rem = j;
      int c = 0;
      for (int ax = 0; ax < d; ++ax) {
        const int v = 1 + (int)(rem % Nv);
        rem /= Nv;
        c |= (v & 1) << ax;
      }
      h.colours[j] = (uint8_t)c;
      lists[c].push_back((int32_t)j);
    }
    for (int c = 0; c < (1 << d); ++c) {
      h.ncolour[c] = (int)lists[c].size();
      DALLOC(h.colour_list[c], lists[c].size());
      if (!lists[c].empty())
        CU(cudaMemcpy(h.colour_list[c], lists[c].data(), lists[c].size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
  }
  // ---- work vectors and transfer tables
  size_t tmax = 1;
  for (int l = 0; l < ctx->nlev; ++l) {
    HLevel& h = ctx->L[l];
    DALLOC(h.x64, h.nd);
    DALLOC(h.b64, h.nd);
    DALLOC(h.r64, h.nd);
    if (mixed) {
      DALLOC(h.x32, h.nd);
      DALLOC(h.b32, h.nd);
      DALLOC(h.r32, h.nd);
    }
    if (l > 0) {
      const int Mc = p * ctx->L[l - 1].N + 1, Mf = p * h.N + 1;
      tmax = std::max(tmax, ipow_sz(Mf, d - 1) * Mc);
      tmax = std::max(tmax, ipow_sz(Mc, d - 1) * Mf);
      std::vector<double> W, RW;
      std::vector<int> S, RS;
      h_prolongation_band(p, ctx->L[l - 1].N, W, S);
      h_restriction_band(p, ctx->L[l - 1].N, RW, RS, h.Rwidth);
      DALLOC(h.PW, W.size());
      DALLOC(h.Ps, S.size());
      DALLOC(h.RW, RW.size());
      DALLOC(h.Rs, RS.size());
      CU(cudaMemcpy(h.PW, W.data(), W.size() * sizeof(double), cudaMemcpyHostToDevice));
      CU(cudaMemcpy(h.Ps, S.data(), S.size() * sizeof(int), cudaMemcpyHostToDevice));
      CU(cudaMemcpy(h.RW, RW.data(), RW.size() * sizeof(double), cudaMemcpyHostToDevice));
      CU(cudaMemcpy(h.Rs, RS.data(), RS.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
  }
  DALLOC(ctx->t64a, tmax);
  DALLOC(ctx->t64b, tmax);
  if (mixed) {
    DALLOC(ctx->t32a, tmax);
    DALLOC(ctx->t32b, tmax);
  }
  {
    const size_t nfin = ctx->L.back().nd;
    size_t nloc = 0;
    for (int l = 0; l < ctx->nlev; ++l)
      nloc = std::max(nloc, ctx->L[l].npatch * ipow_sz(2 * p - 1, d));
    DALLOC(ctx->s32a, std::max(nfin, nloc));
    DALLOC(ctx->s32b, std::max(nfin, nloc));
  }
  // ---- Cartesian-reinforced smoother: reference-patch fast-diagonalisation tables
  for (int k = 0; k < ctx->npl; ++k) {
    const int q = ctx->plevels[k];
    if (q < 2 || ctx->fdm64[q]) continue;
    const std::vector<double> t = fdm_table(q);
    const std::vector<float> t32(t.begin(), t.end());
    DALLOC(ctx->fdm64[q], t.size());
    DALLOC(ctx->fdm32[q], t.size());
    CU(cudaMemcpy(ctx->fdm64[q], t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(ctx->fdm32[q], t32.data(), t32.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  // ---- coarse matrix by applying the coarsest operator to unit vectors
  {
    HLevel& h = ctx->L[0];
    const int M = p * h.N + 1;
    std::vector<int> fidx;
    for (size_t i = 0; i < h.nd; ++i) {
      size_t rem = i;
      bool bnd = false;
      for (int ax = 0; ax < d; ++ax) {
        const int k = (int)(rem % M);
        rem /= M;
        bnd = bnd || k == 0 || k == M - 1;
      }
      if (!bnd) fidx.push_back((int)i);
    }
    const int nf = (int)fidx.size();
    if (nf > kMaxCoarseDofs)
      return fail(ctx, PMG_ERR_UNSUPPORTED,
                  "the coarsest level has " + std::to_string(nf) + " free DoFs; the dense coarse solver takes at most " +
                      std::to_string(kMaxCoarseDofs) + ": use more h-levels");
    ctx->nf = nf;
    DALLOC(ctx->Ainv, (size_t)nf * nf);
    DALLOC(ctx->freeidx, fidx.size());
    CU(cudaMemcpy(ctx->freeidx, fidx.data(), fidx.size() * sizeof(int), cudaMemcpyHostToDevice));
    // all columns of the operator at once (nf unit vectors), then the free rows
    double* cols = nullptr;
    CU(cudaMalloc(&cols, (size_t)nf * h.nd * sizeof(double)));
    int st = PMG_OK;
    for (int j = 0; j < nf && st == PMG_OK; ++j) {
      if (cudaMemsetAsync(h.x64, 0, h.nd * sizeof(double), s) != cudaSuccess ||
          launch_unit(h.x64, (size_t)fidx[j], s) != ST_OK) {
        st = fail(ctx, PMG_ERR_CUDA, "coarse matrix assembly failed");
        break;
      }
      ctx->launches += 1;
      if (cell_apply<double>(ctx, p, h.x64, cols + (size_t)j * h.nd, h.pl[0].G64, h.N, s) != ST_OK)
        st = fail(ctx, PMG_ERR_CUDA, "coarse matrix assembly failed");
      ctx->launches += 1 + (1 << ctx->dim);
    }
    if (st == PMG_OK && launch_gather_coarse(cols, ctx->freeidx, nf, h.nd, ctx->Ainv, s) != ST_OK)
      st = fail(ctx, PMG_ERR_CUDA, "coarse matrix gather failed");
    if (st == PMG_OK && cudaStreamSynchronize(s) != cudaSuccess) st = fail(ctx, PMG_ERR_CUDA, "coarse matrix assembly failed");
    cudaFree(cols);
    if (st) return st;
    std::string msg;
    const int ci = coarse_inverse(ctx->Ainv, nf, s, &msg);
    if (ci == ST_NOT_SPD) return fail(ctx, PMG_ERR_NUMERIC, msg);
    if (ci != ST_OK) return fail(ctx, PMG_ERR_CUDA, msg);
  }
  // ---- CG vectors
  {
    const size_t n = ctx->L.back().nd;
    DALLOC(ctx->cg_x, n);
    if (ctx->opt.additive) {
      DALLOC(ctx->add64, n);
      if (mixed) DALLOC(ctx->add32, n);
    }
    DALLOC(ctx->cg_r, n);
    DALLOC(ctx->cg_z, n);
    DALLOC(ctx->cg_p, n);
    DALLOC(ctx->cg_Ap, n);
    DALLOC(ctx->stage_b, n);
    DALLOC(ctx->stage_u, n);
    DALLOC(ctx->partial, DOT_BLOCKS);
    DALLOC(ctx->scal, S_NSLOT);
  }
  ctx->setup_ok = true;
  // ---- Chebyshev bounds
  int st = pmg_compute_bounds(ctx, ctx->opt.bounds);
  if (st) {
    ctx->setup_ok = false;
    return st;
  }
  st = autotune(ctx);
  if (st) {
    ctx->setup_ok = false;
    return st;
  }
  // warm-up V-cycle on a zero vector: every kernel of the preconditioner runs
  // once (and gets its shared-memory attribute) before any graph capture
  CU(cudaMemsetAsync(ctx->cg_r, 0, ctx->L.back().nd * sizeof(double), s));
  st = precondition(ctx, ctx->cg_r, ctx->cg_z, s);
  if (st) {
    ctx->setup_ok = false;
    return st;
  }
  CU(cudaStreamSynchronize(s));
  return PMG_OK;
}

int pmg_compute_bounds(pmg_ctx* ctx, int source) {
  if (!ctx || !ctx->setup_ok) return fail(ctx, PMG_ERR_ARG, "not set up");
  PMG_GUARD_CTX(ctx);
  if (ctx->um) {
    if (source == PMG_BOUNDS_USER) return PMG_OK;
    if (source == PMG_BOUNDS_LANCZOS) {
      if (ctx->opt.lanczos_steps < 1 || ctx->opt.lanczos_steps > 64)
        return fail(ctx, PMG_ERR_ARG, "lanczos_steps must be in 1..64");
      for (UMesh* m : ctx->umv)
        if (umesh_lanczos(m, ctx->opt.lanczos_steps, ctx->opt.seed, ctx->opt.bound_safety, ctx->opt.bound_ratio,
                          ctx->stream))
          return fail(ctx, PMG_ERR_CUDA, "unstructured Lanczos intervals failed");
      return PMG_OK;
    }
    if (source != PMG_BOUNDS_FIXED)
      return fail(ctx, PMG_ERR_UNSUPPORTED, "unstructured meshes: Lanczos, fixed or user-given Chebyshev intervals");
    for (UMesh* m : ctx->umv) {
      const size_t np = (size_t)umesh_npatch(m);
      std::vector<double> v(2 * np);
      for (size_t j = 0; j < np; ++j) { v[2 * j] = ctx->opt.fixed_lo; v[2 * j + 1] = ctx->opt.fixed_hi; }
      for (int k = 0; k < ctx->npl; ++k)
        if (ctx->plevels[k] > 1 && umesh_set_bounds(m, k, v.data())) return fail(ctx, PMG_ERR_CUDA, "bounds");
    }
    return PMG_OK;
  }
  cudaStream_t s = ctx->stream;
  const int d = ctx->dim;
  if (source == PMG_BOUNDS_USER) return PMG_OK;
  for (int l = 0; l < ctx->nlev; ++l) {
    HLevel& h = ctx->L[l];
    if (h.npatch == 0) continue;
    for (int k = 0; k < ctx->npl; ++k) {
      PLevel& pl = h.pl[k];
      if (pl.q == 1) continue;
      if (source == PMG_BOUNDS_FIXED) {
        std::vector<double> v(2 * h.npatch);
        for (size_t j = 0; j < h.npatch; ++j) { v[2 * j] = ctx->opt.fixed_lo; v[2 * j + 1] = ctx->opt.fixed_hi; }
        CU(cudaMemcpy(pl.bounds64, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice));
        LK(1, launch_cast_d2f(pl.bounds64, pl.bounds32, v.size(), s));
        continue;
      }
      if (source == PMG_BOUNDS_MLP) {
        if (!ctx->mlp_params) return fail(ctx, PMG_ERR_ARG, "no network installed (pmg_set_mlp)");
        float *X = nullptr, *Y = nullptr;
        CU(cudaMalloc(&X, h.npatch * 16 * sizeof(float)));
        CU(cudaMalloc(&Y, h.npatch * 2 * sizeof(float)));
        ST(features_launch(d, h.coords, h.kappa, h.N, pl.q, ctx->npl - 1 - k, (int)h.npatch, X, s));
        ST(mlp_infer_launch(ctx->mlp_params, ctx->mlp_norm, X, (int64_t)h.npatch, 1, Y, s));
        ST(bounds_from_logs_launch(Y, (int64_t)h.npatch, ctx->opt.mlp_safety, ctx->opt.bound_ratio, pl.bounds32,
                                   pl.bounds64, s));
        CU(cudaStreamSynchronize(s));
        cudaFree(X);
        cudaFree(Y);
        continue;
      }
      if (source != PMG_BOUNDS_LANCZOS) return fail(ctx, PMG_ERR_ARG, "unknown bounds source");
      const size_t ni = ipow_sz(2 * pl.q - 1, d);
      const size_t chunk = std::max<size_t>(1, std::min<size_t>(h.npatch, (size_t)(512u << 20) / (ctx->opt.lanczos_steps * ni * 8)));
      const size_t need = chunk * ctx->opt.lanczos_steps * ni;
      if (ctx->lanczos_V_n < need) {
        if (ctx->lanczos_V) CU(cudaFree(ctx->lanczos_V));
        ctx->lanczos_V = nullptr;
        ctx->lanczos_V_n = 0;
        CU(cudaMalloc(&ctx->lanczos_V, need * sizeof(double)));
        ctx->lanczos_V_n = need;
      }
      double* V = ctx->lanczos_V;
      for (size_t j0 = 0; j0 < h.npatch; j0 += chunk) {
        const int n = (int)std::min(chunk, h.npatch - j0);
        LanczosArgs<double> a;
        a.N = h.N;
        a.n_items = n;
        a.first_patch = (int)j0;
        a.G = pl.G64;
        a.dinv = pl.dinv64;
        a.V = V;
        a.ksteps = ctx->opt.lanczos_steps;
        a.seed = ctx->opt.seed;
        a.safety = ctx->opt.bound_safety;
        a.ratio = ctx->opt.bound_ratio;
        a.ritz = pl.ritz;
        a.bounds = pl.bounds64;
        a.bounds_f64 = nullptr;
        a.out_offset = 0;
        int r = d == 2 ? launch_lanczos<2, double>(pl.q, a, s) : launch_lanczos<3, double>(pl.q, a, s);
        if (r == ST_UNSUPPORTED) {
          // the FP64 working set does not fit: FP32 operator, FP64 Lanczos vectors
          LanczosArgs<float> b;
          b.N = a.N;
          b.n_items = a.n_items;
          b.first_patch = a.first_patch;
          b.G = pl.G32;
          b.dinv = pl.dinv32;
          b.V = V;
          b.ksteps = a.ksteps;
          b.seed = a.seed;
          b.safety = a.safety;
          b.ratio = a.ratio;
          b.ritz = pl.ritz;
          b.bounds = pl.bounds32;
          b.bounds_f64 = nullptr;
          b.out_offset = 0;
          if (!pl.G32) {   // FP64 contexts: an FP32 copy of the geometry for the interval estimates only
            const size_t ng = h.ncells * (size_t)(d * (d + 1) / 2) * ipow_sz(pl.q + 1, d);
            DALLOC(pl.G32, ng);
            if (d == 2) ST(launch_geometry<2, float>(h.coords, h.kappa, h.N, pl.q, pl.G32, ctx->d_err, s));
            else ST(launch_geometry<3, float>(h.coords, h.kappa, h.N, pl.q, pl.G32, ctx->d_err, s));
            b.G = pl.G32;
          }
          ST(d == 2 ? launch_lanczos<2, float>(pl.q, b, s) : launch_lanczos<3, float>(pl.q, b, s));
          LK(1, launch_cast_f2d(pl.bounds32, pl.bounds64, 2 * h.npatch, s));
        } else {
          ST(r);
        }
      }
      CU(cudaStreamSynchronize(s));
      LK(1, launch_cast_d2f(pl.bounds64, pl.bounds32, 2 * h.npatch, s));
    }
  }
  CU(cudaStreamSynchronize(s));
  return PMG_OK;
}

int pmg_num_dofs(const pmg_ctx* ctx, int level, int64_t* total, int64_t* n_free) {
  if (!ctx || !ctx->mesh_ok || level < 0 || level >= ctx->nlev) return PMG_ERR_ARG;
  if (ctx->um) {
    if (!ctx->setup_ok) return PMG_ERR_ARG;
    if (total) *total = umesh_ndofs(ctx->umv[level]);
    if (n_free) *n_free = umesh_nfree(ctx->umv[level]);
    return PMG_OK;
  }
  const int Nl = ctx->N >> (ctx->nlev - 1 - level);
  if (total) *total = (int64_t)ipow_sz((size_t)ctx->p * Nl + 1, ctx->dim);
  if (n_free) *n_free = (int64_t)ipow_sz((size_t)ctx->p * Nl - 1, ctx->dim);
  return PMG_OK;
}

int pmg_num_patches(const pmg_ctx* ctx, int level, int64_t* n_patches, int* n_colours) {
  if (!ctx || !ctx->mesh_ok || level < 0 || level >= ctx->nlev) return PMG_ERR_ARG;
  if (ctx->um) {
    if (!ctx->setup_ok) return PMG_ERR_ARG;
    if (n_patches) *n_patches = umesh_npatch(ctx->umv[level]);
    if (n_colours) *n_colours = umesh_ncolours(ctx->umv[level]);
    return PMG_OK;
  }
  const int Nl = ctx->N >> (ctx->nlev - 1 - level);
  if (n_patches) *n_patches = (int64_t)ipow_sz(Nl - 1, ctx->dim);
  if (n_colours) *n_colours = 1 << ctx->dim;
  return PMG_OK;
}

int pmg_p_levels(const pmg_ctx* ctx, int* degrees, int* n) {
  if (!ctx || !ctx->mesh_ok || !n) return PMG_ERR_ARG;
  *n = ctx->npl;
  if (degrees)
    for (int k = 0; k < ctx->npl; ++k) degrees[k] = ctx->plevels[k];
  return PMG_OK;
}

static int check_level(pmg_ctx* ctx, int level) {
  if (!ctx) return PMG_ERR_ARG;
  if (!ctx->setup_ok) return fail(ctx, PMG_ERR_ARG, "call pmg_setup first");
  if (level < 0 || level >= ctx->nlev) return fail(ctx, PMG_ERR_ARG, "level out of range");
  return PMG_OK;
}

int pmg_apply(pmg_ctx* ctx, int level, const double* u, double* Au, void* stream) {
  int st = check_level(ctx, level);
  if (st) return st;
  PMG_GUARD_CTX(ctx);
  if (!u || !Au) return fail(ctx, PMG_ERR_ARG, "null vector");
  if (ctx->um) return umesh_apply(ctx->umv[level], u, Au, (cudaStream_t)stream) ? fail(ctx, PMG_ERR_CUDA, "apply failed") : PMG_OK;
  HLevel& h = ctx->L[level];
  LK(1 + (1 << ctx->dim), cell_apply<double>(ctx, ctx->p, u, Au, h.pl[0].G64, h.N, (cudaStream_t)stream));
  return PMG_OK;
}

int pmg_patch_smooth_colour(pmg_ctx* ctx, int level, int colour, const double* b, double* u, void* stream) {
  int st = check_level(ctx, level);
  if (st) return st;
  PMG_GUARD_CTX(ctx);
  if (!b || !u) return fail(ctx, PMG_ERR_ARG, "null vector");
  if (ctx->um) {
    if (colour < 0 || colour >= umesh_ncolours(ctx->umv[level])) return fail(ctx, PMG_ERR_ARG, "colour out of range");
    return umesh_sweep_colour(ctx->umv[level], colour, b, u, (cudaStream_t)stream) ? fail(ctx, PMG_ERR_CUDA, "sweep failed")
                                                                           : PMG_OK;
  }
  if (colour < 0 || colour >= (1 << ctx->dim)) return fail(ctx, PMG_ERR_ARG, "colour out of range");
  if (ctx->opt.additive) return fail(ctx, PMG_ERR_UNSUPPORTED, "an additive sweep runs all colours (pmg_patch_smooth)");
  cudaStream_t s = (cudaStream_t)stream;
  HLevel& h = ctx->L[level];
  if (ctx->opt.precision == PMG_PREC_MIXED) {
    LK(1, launch_cast_d2f(b, ctx->s32a, h.nd, s));
    LK(1, launch_cast_d2f(u, ctx->s32b, h.nd, s));
    st = sweep_colour<float>(ctx, level, colour, ctx->s32a, ctx->s32b, s);
    if (st) return st;
    LK(1, launch_cast_f2d(ctx->s32b, u, h.nd, s));
    return PMG_OK;
  }
  return sweep_colour<double>(ctx, level, colour, b, u, s);
}

int pmg_patch_smooth(pmg_ctx* ctx, int level, const double* b, double* u, int n_sweeps, int reverse, void* stream) {
  int st = check_level(ctx, level);
  if (st) return st;
  PMG_GUARD_CTX(ctx);
  if (!b || !u || n_sweeps < 0) return fail(ctx, PMG_ERR_ARG, "bad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  if (ctx->um)
    return umesh_sweep(ctx->umv[level], b, u, n_sweeps, reverse != 0, s) ? fail(ctx, PMG_ERR_CUDA, "sweep failed") : PMG_OK;
  HLevel& h = ctx->L[level];
  // a persistent level's barrier status is read here, so the call waits for its stream
  const bool wait = level < 16 && ctx->level_persist[level] && n_sweeps > 0;
  if (ctx->opt.precision == PMG_PREC_MIXED) {
    LK(1, launch_cast_d2f(b, ctx->s32a, h.nd, s));
    LK(1, launch_cast_d2f(u, ctx->s32b, h.nd, s));
    for (int i = 0; i < n_sweeps; ++i) {
      st = sweep<float>(ctx, level, ctx->s32a, ctx->s32b, reverse != 0, s);
      if (st) return st;
    }
    LK(1, launch_cast_f2d(ctx->s32b, u, h.nd, s));
  } else {
    for (int i = 0; i < n_sweeps; ++i) {
      st = sweep<double>(ctx, level, b, u, reverse != 0, s);
      if (st) return st;
    }
  }
  if (wait) {
    CU(cudaStreamSynchronize(s));
    return check_sync(ctx);
  }
  return PMG_OK;
}

int pmg_local_vcycle(pmg_ctx* ctx, int level, int64_t n, const int64_t* ids, const double* r, double* dout,
                     int n_cycles, void* stream) {
  int st = check_level(ctx, level);
  if (st) return st;
  PMG_GUARD_CTX(ctx);
  if (n < 0 || (n > 0 && (!ids || !r || !dout)) || n_cycles < 1) return fail(ctx, PMG_ERR_ARG, "bad arguments");
  if (n == 0) return PMG_OK;
  if (ctx->um) {
    if (n > umesh_npatch(ctx->umv[level])) return fail(ctx, PMG_ERR_ARG, "more patches than the level has");
    return umesh_local(ctx->umv[level], n, ids, r, dout, n_cycles, (cudaStream_t)stream) ? fail(ctx, PMG_ERR_CUDA, "local solve failed")
                                                                                 : PMG_OK;
  }
  HLevel& h = ctx->L[level];
  if ((size_t)n > h.npatch) return fail(ctx, PMG_ERR_ARG, "more patches than the level has");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ni = ipow_sz(2 * ctx->p - 1, ctx->dim);
  if (ctx->opt.precision == PMG_PREC_MIXED) {
    PatchArgs<float> a = patch_args<float>(ctx, level);
    a.n_mg = n_cycles;
    a.ids64 = ids;
    a.n_items = (int)n;
    LK(1, launch_cast_d2f(r, ctx->s32a, (size_t)n * ni, s));
    a.r_in = ctx->s32a;
    a.d_out = ctx->s32b;
    LK(1, patch_launch<float>(ctx, MODE_LOCAL, a, s));
    LK(1, launch_cast_f2d(ctx->s32b, dout, (size_t)n * ni, s));
    return PMG_OK;
  }
  PatchArgs<double> a = patch_args<double>(ctx, level);
  a.n_mg = n_cycles;
  a.ids64 = ids;
  a.n_items = (int)n;
  a.r_in = r;
  a.d_out = dout;
  LK(1, patch_launch<double>(ctx, MODE_LOCAL, a, s));
  return PMG_OK;
}

int pmg_get_bounds(pmg_ctx* ctx, int level, double* lohi) {
  int st = check_level(ctx, level);
  if (st) return st;
  PMG_GUARD_CTX(ctx);
  if (ctx->um) {
    const size_t np = (size_t)umesh_npatch(ctx->umv[level]);
    std::vector<double> out(2 * np * ctx->npl, 0.0), tmp(2 * np);
    CU(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < ctx->npl; ++k) {
      if (ctx->plevels[k] == 1 || np == 0) continue;
      if (umesh_get_bounds(ctx->umv[level], k, tmp.data())) return fail(ctx, PMG_ERR_CUDA, "bounds copy failed");
      for (size_t j = 0; j < np; ++j) {
        out[(j * ctx->npl + k) * 2] = tmp[2 * j];
        out[(j * ctx->npl + k) * 2 + 1] = tmp[2 * j + 1];
      }
    }
    std::memcpy(lohi, out.data(), out.size() * sizeof(double));
    return PMG_OK;
  }
  HLevel& h = ctx->L[level];
  std::vector<double> out(2 * h.npatch * ctx->npl, 0.0), tmp(2 * h.npatch);
  CU(cudaStreamSynchronize(ctx->stream));
  for (int k = 0; k < ctx->npl; ++k) {
    if (h.pl[k].q == 1 || h.npatch == 0) continue;
    CU(cudaMemcpy(tmp.data(), h.pl[k].bounds64, tmp.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (size_t j = 0; j < h.npatch; ++j) {
      out[(j * ctx->npl + k) * 2] = tmp[2 * j];
      out[(j * ctx->npl + k) * 2 + 1] = tmp[2 * j + 1];
    }
  }
  std::memcpy(lohi, out.data(), out.size() * sizeof(double));
  return PMG_OK;
}

int pmg_get_ritz(pmg_ctx* ctx, int level, double* tm) {
  int st = check_level(ctx, level);
  if (st) return st;
  PMG_GUARD_CTX(ctx);
  if (ctx->um) {
    const size_t np = (size_t)umesh_npatch(ctx->umv[level]);
    std::vector<double> out(2 * np * ctx->npl, 0.0), tmp(2 * np);
    CU(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < ctx->npl; ++k) {
      if (ctx->plevels[k] == 1 || np == 0) continue;
      if (umesh_get_ritz(ctx->umv[level], k, tmp.data())) return fail(ctx, PMG_ERR_CUDA, "copy failed");
      for (size_t j = 0; j < np; ++j) {
        out[(j * ctx->npl + k) * 2] = tmp[2 * j];
        out[(j * ctx->npl + k) * 2 + 1] = tmp[2 * j + 1];
      }
    }
    std::memcpy(tm, out.data(), out.size() * sizeof(double));
    return PMG_OK;
  }
  HLevel& h = ctx->L[level];
  std::vector<double> out(2 * h.npatch * ctx->npl, 0.0), tmp(2 * h.npatch);
  CU(cudaStreamSynchronize(ctx->stream));
  for (int k = 0; k < ctx->npl; ++k) {
    if (h.pl[k].q == 1 || h.npatch == 0) continue;
    CU(cudaMemcpy(tmp.data(), h.pl[k].ritz, tmp.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (size_t j = 0; j < h.npatch; ++j) {
      out[(j * ctx->npl + k) * 2] = tmp[2 * j];
      out[(j * ctx->npl + k) * 2 + 1] = tmp[2 * j + 1];
    }
  }
  std::memcpy(tm, out.data(), out.size() * sizeof(double));
  return PMG_OK;
}

int pmg_set_bounds(pmg_ctx* ctx, int level, const double* lohi) {
  int st = check_level(ctx, level);
  if (st) return st;
  PMG_GUARD_CTX(ctx);
  if (ctx->um) {
    const size_t np = (size_t)umesh_npatch(ctx->umv[level]);
    std::vector<double> tmp(2 * np);
    CU(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < ctx->npl; ++k) {
      if (ctx->plevels[k] == 1 || np == 0) continue;
      for (size_t j = 0; j < np; ++j) {
        const double lo = lohi[(j * ctx->npl + k) * 2], hi = lohi[(j * ctx->npl + k) * 2 + 1];
        if (!(lo > 0) || !(hi > lo)) return fail(ctx, PMG_ERR_ARG, "bounds must satisfy 0 < lo < hi");
        tmp[2 * j] = lo;
        tmp[2 * j + 1] = hi;
      }
      if (umesh_set_bounds(ctx->umv[level], k, tmp.data())) return fail(ctx, PMG_ERR_CUDA, "bounds copy failed");
    }
    return PMG_OK;
  }
  HLevel& h = ctx->L[level];
  std::vector<double> tmp(2 * h.npatch);
  for (int k = 0; k < ctx->npl; ++k) {
    if (h.pl[k].q == 1 || h.npatch == 0) continue;
    for (size_t j = 0; j < h.npatch; ++j) {
      const double lo = lohi[(j * ctx->npl + k) * 2], hi = lohi[(j * ctx->npl + k) * 2 + 1];
      if (!(lo > 0) || !(hi > lo)) return fail(ctx, PMG_ERR_ARG, "bounds must satisfy 0 < lo < hi");
      tmp[2 * j] = lo;
      tmp[2 * j + 1] = hi;
    }
    CU(cudaMemcpy(h.pl[k].bounds64, tmp.data(), tmp.size() * sizeof(double), cudaMemcpyHostToDevice));
    LK(1, launch_cast_d2f(h.pl[k].bounds64, h.pl[k].bounds32, tmp.size(), ctx->stream));
  }
  CU(cudaStreamSynchronize(ctx->stream));
  return PMG_OK;
}

int pmg_gmg_vcycle(pmg_ctx* ctx, const double* b, double* x, void* stream) {
  int st = check_level(ctx, ctx ? ctx->nlev - 1 : 0);
  if (st) return st;
  PMG_GUARD_CTX(ctx);
  if (!b || !x) return fail(ctx, PMG_ERR_ARG, "null vector");
  return precondition(ctx, b, x, (cudaStream_t)stream);
}

// One CG iteration body (captured into a CUDA graph): z = M r, rz = (r, z),
// p = z + beta p, Ap = A p, alpha = rz / (p, Ap), x += alpha p, r -= alpha Ap,
// rr = (r, r) copied to pinned host memory.
// vector length of the finest level
static size_t fine_n(const pmg_ctx* ctx) { return ctx->um ? (size_t)umesh_ndofs(ctx->um) : ctx->L.back().nd; }

// Ax = A x on the finest level (FP64)
static int fine_apply(pmg_ctx* ctx, const double* x, double* Ax, cudaStream_t s) {
  if (ctx->um) return umesh_apply(ctx->um, x, Ax, s) ? fail(ctx, PMG_ERR_CUDA, "apply failed") : PMG_OK;
  HLevel& h = ctx->L.back();
  LK(1 + (1 << ctx->dim), cell_apply<double>(ctx, ctx->p, x, Ax, h.pl[0].G64, h.N, s));
  return PMG_OK;
}

static int fine_mask(pmg_ctx* ctx, double* x, cudaStream_t s) {
  if (ctx->um) return umesh_mask(ctx->um, x, s) ? fail(ctx, PMG_ERR_CUDA, "mask failed") : PMG_OK;
  LK(1, mask_boundary<double>(ctx, x, ctx->p * ctx->L.back().N + 1, s));
  return PMG_OK;
}

static int cg_body(pmg_ctx* ctx, cudaStream_t s) {
  const size_t n = fine_n(ctx);
  int st = precondition(ctx, ctx->cg_r, ctx->cg_z, s);
  if (st) return st;
  LK(2, launch_dot(ctx->cg_r, ctx->cg_z, n, ctx->partial, ctx->scal, S_RZ, 1, s));
  LK(1, launch_cg_update_p(ctx->cg_z, ctx->cg_p, ctx->scal, n, s));
  st = fine_apply(ctx, ctx->cg_p, ctx->cg_Ap, s);
  if (st) return st;
  LK(2, launch_dot(ctx->cg_p, ctx->cg_Ap, n, ctx->partial, ctx->scal, S_PAP, 2, s));
  LK(1, launch_cg_update_xr(ctx->cg_x, ctx->cg_r, ctx->cg_p, ctx->cg_Ap, ctx->scal, n, s));
  LK(2, launch_dot(ctx->cg_r, ctx->cg_r, n, ctx->partial, ctx->scal, S_RR, 0, s));
  CU(cudaMemcpyAsync(ctx->h_rr, ctx->scal + S_RR, sizeof(double), cudaMemcpyDeviceToHost, s));
  return PMG_OK;
}

// ---- CG in three steps, so that several contexts can interleave their
// iterations (pmg_batch_solve_cg): start (x = 0, r = b, (r, r) copied to the
// host), graph (capture of one iteration body, once per context), step (one
// iteration launched; (r, r) copied to the host at its end).  All are
// asynchronous on the context's stream.
static int cg_start(pmg_ctx* ctx, const double* b) {
  cudaStream_t s = ctx->stream;
  const size_t n = fine_n(ctx);
  CU(cudaMemsetAsync(ctx->cg_x, 0, n * sizeof(double), s));
  CU(cudaMemsetAsync(ctx->cg_p, 0, n * sizeof(double), s));
  CU(cudaMemcpyAsync(ctx->cg_r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  const int stm = fine_mask(ctx, ctx->cg_r, s);
  if (stm) return stm;
  {
    static const double init[S_NSLOT] = {0.0, 1.0, 0.0, 0.0, 0.0, 0.0};
    CU(cudaMemcpyAsync(ctx->scal, init, sizeof(init), cudaMemcpyHostToDevice, s));
  }
  LK(2, launch_dot(ctx->cg_r, ctx->cg_r, n, ctx->partial, ctx->scal, S_RR, 0, s));
  CU(cudaMemcpyAsync(ctx->h_rr, ctx->scal + S_RR, sizeof(double), cudaMemcpyDeviceToHost, s));
  return PMG_OK;
}

static int cg_graph(pmg_ctx* ctx) {
  if (ctx->graph_exec) return PMG_OK;
  cudaStream_t s = ctx->stream;
  cudaGraph_t g = nullptr;
  const int64_t before = ctx->launches;
  const int64_t ubefore = ctx->um ? umesh_kernel_launches(ctx->um) : 0;
  CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  int st = cg_body(ctx, s);
  // the capture launched nothing: what the body counted is one replay's launches
  const int64_t ucount = ctx->um ? umesh_kernel_launches(ctx->um) - ubefore : 0;
  ctx->graph_launches_per_iter = ctx->launches - before + ucount;
  ctx->launches = before - ucount;
  cudaError_t ce = cudaStreamEndCapture(s, &g);
  if (st || ce != cudaSuccess) {           // no graph: iterations launch the body directly
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    ctx->graph_exec = nullptr;
  } else {
    ctx->graph = g;
    if (cudaGraphInstantiate(&ctx->graph_exec, g, 0) != cudaSuccess) {
      cudaGetLastError();
      ctx->graph_exec = nullptr;
    }
  }
  return PMG_OK;
}

static int cg_step(pmg_ctx* ctx) {
  if (ctx->graph_exec) {
    CU(cudaGraphLaunch(ctx->graph_exec, ctx->stream));
    ctx->launches += ctx->graph_launches_per_iter;
    return PMG_OK;
  }
  return cg_body(ctx, ctx->stream);
}

int pmg_solve_cg(pmg_ctx* ctx, const double* b, double* u, double rtol, int maxit, int* iters, double* relres,
                 void* stream) {
  int st = check_level(ctx, ctx ? ctx->nlev - 1 : 0);
  if (st) return st;
  PMG_GUARD_CTX(ctx);
  if (!b || !u || maxit < 0 || !(rtol >= 0)) return fail(ctx, PMG_ERR_ARG, "bad arguments");
  cudaStream_t us = (cudaStream_t)stream;
  cudaStream_t s = ctx->stream;
  // the solve runs on the context's stream, after the work already queued
  // on the caller's stream (an event wait; the caller's stream is not synchronised)
  CU(cudaEventRecord(ctx->ev_caller, us));
  CU(cudaStreamWaitEvent(ctx->stream, ctx->ev_caller, 0));
  const size_t n = fine_n(ctx);
  st = cg_start(ctx, b);
  if (st) return st;
  CU(cudaStreamSynchronize(s));
  const double r0 = std::sqrt(*ctx->h_rr);
  int it = 0;
  double rel = 1.0;
  int result = PMG_OK;
  if (!std::isfinite(r0)) result = fail(ctx, PMG_ERR_NUMERIC, "non-finite right-hand side");
  if (result == PMG_OK && r0 == 0.0) rel = 0.0;
  if (result == PMG_OK && r0 > 0.0) {
    st = cg_graph(ctx);
    if (st) return st;
    while (it < maxit) {
      ++it;
      st = cg_step(ctx);
      if (st) return st;
      CU(cudaStreamSynchronize(s));
      if ((result = check_sync(ctx)) != PMG_OK) break;
      rel = std::sqrt(*ctx->h_rr) / r0;
      if (!std::isfinite(rel)) {
        result = fail(ctx, PMG_ERR_NUMERIC, "non-finite residual");
        break;
      }
      if (rel <= rtol) break;
    }
    if (result == PMG_OK && rel > rtol) result = fail(ctx, PMG_ERR_NOT_CONVERGED, "maxit reached");
  }
  CU(cudaMemcpyAsync(u, ctx->cg_x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CU(cudaStreamSynchronize(s));
  if (iters) *iters = it;
  if (relres) *relres = rel;
  return result;
}

int pmg_batch_solve_cg(pmg_ctx* const* ctxs, int n_problems, const double* const* b, double* const* u, double rtol,
                       int maxit, int* iters, double* relres, int* status) {
  if (n_problems < 0 || (n_problems > 0 && (!ctxs || !b || !u)) || maxit < 0 || !(rtol >= 0)) return PMG_ERR_ARG;
  const int K = n_problems;
  for (int k = 0; k < K; ++k) {
    if (!ctxs[k] || !b[k] || !u[k]) return PMG_ERR_ARG;
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) return fail(ctxs[k], PMG_ERR_ARG, "a context appears twice in the batch");
    const int st = check_level(ctxs[k], ctxs[k]->nlev - 1);
    if (st) return st;
    if (ctxs[k]->device != ctxs[0]->device)
      return fail(ctxs[k], PMG_ERR_ARG, "all problems of a batch must be on one device");
  }
  if (K == 0) return PMG_OK;
  PMG_GUARD_DEV(ctxs[0]->device);
  std::vector<double> r0(K, 0.0), rel(K, 1.0);
  std::vector<int> it(K, 0), res(K, PMG_OK);
  std::vector<char> active(K, 0);
  // on an error, no problem's work may still be running when we return
  auto drain = [&](int code) {
    for (int k = 0; k < K; ++k) cudaStreamSynchronize(ctxs[k]->stream);
    return code;
  };
  for (int k = 0; k < K; ++k) {                      // every start in flight before the first wait
    const int st = cg_start(ctxs[k], b[k]);
    if (st) return drain(st);
  }
  for (int k = 0; k < K; ++k) {
    pmg_ctx* ctx = ctxs[k];
    CU(cudaStreamSynchronize(ctx->stream));
    r0[k] = std::sqrt(*ctx->h_rr);
    if (!std::isfinite(r0[k])) res[k] = fail(ctx, PMG_ERR_NUMERIC, "non-finite right-hand side");
    else if (r0[k] == 0.0) rel[k] = 0.0;
    else if (maxit > 0) active[k] = 1;
    if (active[k]) {
      const int st = cg_graph(ctx);
      if (st) return drain(st);
    }
  }
  for (;;) {
    bool any = false;
    for (int k = 0; k < K; ++k) {                    // one iteration of every unfinished problem
      if (!active[k]) continue;
      any = true;
      ++it[k];
      const int st = cg_step(ctxs[k]);
      if (st) return drain(st);
    }
    if (!any) break;
    for (int k = 0; k < K; ++k) {
      if (!active[k]) continue;
      pmg_ctx* ctx = ctxs[k];
      CU(cudaStreamSynchronize(ctx->stream));
      rel[k] = std::sqrt(*ctx->h_rr) / r0[k];
      const int sy = check_sync(ctx);
      if (sy != PMG_OK) {
        res[k] = sy;
        active[k] = 0;
      } else if (!std::isfinite(rel[k])) {
        res[k] = fail(ctx, PMG_ERR_NUMERIC, "non-finite residual");
        active[k] = 0;
      } else if (rel[k] <= rtol) {
        active[k] = 0;
      } else if (it[k] >= maxit) {
        res[k] = fail(ctx, PMG_ERR_NOT_CONVERGED, "maxit reached");
        active[k] = 0;
      }
    }
  }
  for (int k = 0; k < K; ++k) {
    pmg_ctx* ctx = ctxs[k];
    if (res[k] == PMG_OK && rel[k] > rtol) res[k] = fail(ctx, PMG_ERR_NOT_CONVERGED, "maxit reached");
    CU(cudaMemcpyAsync(u[k], ctx->cg_x, fine_n(ctx) * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
  }
  int result = PMG_OK;
  for (int k = 0; k < K; ++k) {
    pmg_ctx* ctx = ctxs[k];
    CU(cudaStreamSynchronize(ctx->stream));
    if (iters) iters[k] = it[k];
    if (relres) relres[k] = rel[k];
    if (status) status[k] = res[k];
    if (res[k] != PMG_OK && result == PMG_OK) result = res[k];
  }
  return result;
}

// (x, y) in FP64, deterministic, result on the host
static int dot_host(pmg_ctx* ctx, const double* x, const double* y, size_t n, double* out, cudaStream_t s) {
  LK(2, launch_dot(x, y, n, ctx->partial, ctx->scal, S_RR, 0, s));
  CU(cudaMemcpyAsync(ctx->h_rr, ctx->scal + S_RR, sizeof(double), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  *out = *ctx->h_rr;
  return PMG_OK;
}

int pmg_solve_gmres(pmg_ctx* ctx, const double* b, double* u, double rtol, int maxit, int restart, int left,
                    int* iters, double* relres, void* stream) {
  int st = check_level(ctx, ctx ? ctx->nlev - 1 : 0);
  if (st) return st;
  PMG_GUARD_CTX(ctx);
  if (!b || !u || maxit < 0 || restart < 1 || restart > 1000 || !(rtol >= 0)) return fail(ctx, PMG_ERR_ARG, "bad arguments");
  cudaStream_t us = (cudaStream_t)stream;
  cudaStream_t s = ctx->stream;
  // the solve runs on the context's stream, after the work already queued
  // on the caller's stream (an event wait; the caller's stream is not synchronised)
  CU(cudaEventRecord(ctx->ev_caller, us));
  CU(cudaStreamWaitEvent(ctx->stream, ctx->ev_caller, 0));
  const size_t n = fine_n(ctx);
  if (ctx->gm_m < restart) {
    if (ctx->gm_V) CU(cudaFree(ctx->gm_V));
    ctx->gm_V = nullptr;
    ctx->gm_m = 0;
    CU(cudaMalloc(&ctx->gm_V, (size_t)(restart + 1) * n * sizeof(double)));
    ctx->gm_m = restart;
  }
  double* V = ctx->gm_V;
  double *x = ctx->cg_x, *r = ctx->cg_r, *w = ctx->cg_Ap, *z = ctx->cg_z, *t = ctx->cg_p;
  CU(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  CU(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  st = fine_mask(ctx, r, s);
  if (st) return st;
  if (left) {                                                           // r = M b
    st = precondition(ctx, r, z, s);
    if (st) return st;
    CU(cudaMemcpyAsync(r, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  double rr;
  st = dot_host(ctx, r, r, n, &rr, s);
  if (st) return st;
  const double r0 = std::sqrt(rr);
  int it = 0;
  double rel = r0 > 0 ? 1.0 : 0.0;
  int result = PMG_OK;
  if (!std::isfinite(r0)) result = fail(ctx, PMG_ERR_NUMERIC, "non-finite right-hand side");
  std::vector<double> H((size_t)(restart + 1) * restart), cs(restart), sn(restart), g(restart + 1), y(restart);
  while (result == PMG_OK && r0 > 0 && rel > rtol && it < maxit) {
    double beta;
    st = dot_host(ctx, r, r, n, &beta, s);
    if (st) return st;
    beta = std::sqrt(beta);
    LK(1, launch_scale(1.0 / beta, r, V, n, s));
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < restart && it < maxit; ++j) {
      if (left) {                                                       // w = M A v_j
        st = fine_apply(ctx, V + (size_t)j * n, z, s);
        if (st) break;
        st = precondition(ctx, z, w, s);
      } else {                                                          // w = A M v_j
        st = precondition(ctx, V + (size_t)j * n, z, s);
        if (!st) st = fine_apply(ctx, z, w, s);
      }
      if (st) return st;
      for (int i = 0; i <= j; ++i) {                                    // modified Gram-Schmidt
        double hij;
        st = dot_host(ctx, w, V + (size_t)i * n, n, &hij, s);
        if (st) return st;
        H[(size_t)i * restart + j] = hij;
        LK(1, launch_axpy(-hij, V + (size_t)i * n, w, n, s));
      }
      double hn;
      st = dot_host(ctx, w, w, n, &hn, s);
      if (st) return st;
      hn = std::sqrt(hn);
      H[(size_t)(j + 1) * restart + j] = hn;
      if (hn > 0) LK(1, launch_scale(1.0 / hn, w, V + (size_t)(j + 1) * n, n, s));
      for (int i = 0; i < j; ++i) {                                     // previous rotations
        const double a = H[(size_t)i * restart + j], c = H[(size_t)(i + 1) * restart + j];
        H[(size_t)i * restart + j] = cs[i] * a + sn[i] * c;
        H[(size_t)(i + 1) * restart + j] = -sn[i] * a + cs[i] * c;
      }
      const double a = H[(size_t)j * restart + j], c = H[(size_t)(j + 1) * restart + j];
      const double den = std::hypot(a, c);
      cs[j] = a / den;
      sn[j] = c / den;
      H[(size_t)j * restart + j] = den;
      H[(size_t)(j + 1) * restart + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++it;
      k = j + 1;
      rel = std::fabs(g[j + 1]) / r0;
      if (!std::isfinite(rel)) {
        result = fail(ctx, PMG_ERR_NUMERIC, "non-finite residual");
        break;
      }
      if (rel <= rtol) break;
    }
    if (result != PMG_OK) break;
    for (int i = k - 1; i >= 0; --i) {                                  // H y = g (upper triangular)
      double v = g[i];
      for (int c2 = i + 1; c2 < k; ++c2) v -= H[(size_t)i * restart + c2] * y[c2];
      y[i] = v / H[(size_t)i * restart + i];
    }
    if (left) {                                                         // x += V y
      for (int i = 0; i < k; ++i) LK(1, launch_axpy(y[i], V + (size_t)i * n, x, n, s));
    } else {                                                            // x += M (V y)
      CU(cudaMemsetAsync(t, 0, n * sizeof(double), s));
      for (int i = 0; i < k; ++i) LK(1, launch_axpy(y[i], V + (size_t)i * n, t, n, s));
      st = precondition(ctx, t, z, s);
      if (st) return st;
      LK(1, launch_axpy(1.0, z, x, n, s));
    }
    st = fine_apply(ctx, x, w, s);   // r = b - A x
    if (st) return st;
    CU(cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    st = fine_mask(ctx, r, s);
    if (st) return st;
    LK(1, launch_axpy(-1.0, w, r, n, s));
    if (left) {                                                         // r = M (b - A x)
      st = precondition(ctx, r, z, s);
      if (st) return st;
      CU(cudaMemcpyAsync(r, z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
  }
  if (result == PMG_OK && rel > rtol) result = fail(ctx, PMG_ERR_NOT_CONVERGED, "maxit reached");
  CU(cudaMemcpyAsync(u, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CU(cudaStreamSynchronize(s));
  if (iters) *iters = it;
  if (relres) *relres = rel;
  const int sy = check_sync(ctx);
  return sy != PMG_OK ? sy : result;
}

int pmg_solve_cg_host(pmg_ctx* ctx, const double* b_host, double* u_host, double rtol, int maxit, int* iters,
                      double* relres, void* stream) {
  int st = check_level(ctx, ctx ? ctx->nlev - 1 : 0);
  if (st) return st;
  PMG_GUARD_CTX(ctx);
  if (!b_host || !u_host) return fail(ctx, PMG_ERR_ARG, "null vector");
  const size_t n = fine_n(ctx);
  cudaStream_t s = ctx->stream;
  CU(cudaMemcpyAsync(ctx->stage_b, b_host, n * sizeof(double), cudaMemcpyHostToDevice, s));
  CU(cudaStreamSynchronize(s));
  st = pmg_solve_cg(ctx, ctx->stage_b, ctx->stage_u, rtol, maxit, iters, relres, stream);
  CU(cudaMemcpyAsync(u_host, ctx->stage_u, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  return st;
}

int pmg_rhs_manufactured(pmg_ctx* ctx, double* b, void* stream) {
  int st = check_level(ctx, ctx ? ctx->nlev - 1 : 0);
  if (st) return st;
  PMG_GUARD_CTX(ctx);
  if (ctx->um) return fail(ctx, PMG_ERR_UNSUPPORTED, "not available on unstructured meshes");
  if (!b) return fail(ctx, PMG_ERR_ARG, "null vector");
  HLevel& h = ctx->L.back();
  if (ctx->dim == 2) ST(launch_rhs_manufactured<2>(h.coords, h.N, ctx->p, b, (cudaStream_t)stream));
  else ST(launch_rhs_manufactured<3>(h.coords, h.N, ctx->p, b, (cudaStream_t)stream));
  return PMG_OK;
}

int pmg_get_colours(const pmg_ctx* ctx, int level, uint8_t* out) {
  if (!ctx || !ctx->setup_ok || level < 0 || level >= ctx->nlev || !out) return PMG_ERR_ARG;
  if (ctx->um) return umesh_colours(ctx->umv[level], out) ? PMG_ERR_ARG : PMG_OK;
  const HLevel& h = ctx->L[level];
  std::memcpy(out, h.colours.data(), h.npatch);
  return PMG_OK;
}

int pmg_get_patch_map(const pmg_ctx* ctx, int level, int64_t* out) {
  if (!ctx || !ctx->setup_ok || level < 0 || level >= ctx->nlev || !out) return PMG_ERR_ARG;
  if (ctx->um) return umesh_patches(ctx->umv[level], out, 1 + PMG_UMAXC) ? PMG_ERR_ARG : PMG_OK;
  const HLevel& h = ctx->L[level];
  const int d = ctx->dim, Nl = h.N, Nv = Nl - 1;
  const size_t Mg = (size_t)ctx->p * Nl + 1;
  for (size_t j = 0; j < h.npatch; ++j) {
    int v[3] = {0, 0, 0};
    size_t rem = j;
    for (int ax = 0; ax < d; ++ax) { v[ax] = 1 + (int)(rem % Nv); rem /= Nv; }
    int64_t* o = out + j * ((1 << d) + 1);
    for (int s2 = 0; s2 < (1 << d); ++s2) {
      int64_t id = 0, mul = 1;
      for (int ax = 0; ax < d; ++ax) { id += (v[ax] - 1 + ((s2 >> ax) & 1)) * mul; mul *= Nl; }
      o[s2] = id;
    }
    int64_t g = 0, mul = 1;
    for (int ax = 0; ax < d; ++ax) { g += (int64_t)ctx->p * (v[ax] - 1) * mul; mul *= (int64_t)Mg; }
    o[1 << d] = g;
  }
  return PMG_OK;
}

int pmg_get_inv_diag(pmg_ctx* ctx, int level, int k, double* out, void* stream) {
  int st = check_level(ctx, level);
  if (st) return st;
  PMG_GUARD_CTX(ctx);
  if (ctx->um) return fail(ctx, PMG_ERR_UNSUPPORTED, "not available on unstructured meshes");
  if (k < 0 || k >= ctx->npl || !out) return fail(ctx, PMG_ERR_ARG, "bad p-level");
  HLevel& h = ctx->L[level];
  const size_t ndq = ipow_sz((size_t)h.pl[k].q * h.N + 1, ctx->dim);
  CU(cudaMemcpyAsync(out, h.pl[k].dinv64, ndq * sizeof(double), cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return PMG_OK;
}

double pmg_sweep_flops(const pmg_ctx* ctx, int level) {
  if (!ctx || !ctx->mesh_ok || level < 0 || level >= ctx->nlev || ctx->um) return 0.0;
  const int d = ctx->dim;
  const int Nl = ctx->N >> (ctx->nlev - 1 - level);
  const double npatch = (double)ipow_sz(Nl - 1, d);
  auto fcell = [d](int n) { return 8.0 * d * std::pow(n, d + 1) + (2.0 * d * d - d) * std::pow(n, d); };
  auto fpatch = [&](int q) { return (double)(1 << d) * fcell(q + 1); };
  const int k = ctx->opt.cheb_degree;
  const bool jac = ctx->opt.smoother == PMG_SMOOTHER_JACOBI || ctx->opt.smoother == PMG_SMOOTHER_CARTESIAN;
  const bool fdm = ctx->opt.smoother == PMG_SMOOTHER_CARTESIAN;
  double per = fpatch(ctx->p);   // Evaluate
  for (int cyc = 0; cyc < ctx->opt.n_mg; ++cyc) {
    for (int lv = 0; lv < ctx->npl; ++lv) {
      const int q = ctx->plevels[lv];
      if (q == 1) continue;
      const bool zero = (lv > 0) || (cyc == 0);
      const int pre = jac ? (zero ? 0 : 1) : (zero ? k - 1 : k);
      const int post = jac ? 1 : k;
      per += (pre + 1 + post) * fpatch(q);
      if (fdm)   // pre and post: 2d one-dimensional contractions of (2q-1)^(d+1) FMAs each
        per += 2.0 * 2.0 * (2.0 * d) * std::pow(2 * q - 1, d + 1);
      const int qc = coarse_degree(q, ctx->opt.level_rule);
      // restriction + prolongation: d sweeps per cell, each at most n_f^d * n_c FMAs
      per += 2.0 * (1 << d) * 2.0 * d * std::pow(q + 1, d) * (qc + 1);
    }
  }
  return per * npatch;
}

int pmg_tuning_level(const pmg_ctx* ctx, int level, int* variant, float* ms_per_variant) {
  if (!ctx || !ctx->setup_ok || level < 0 || level >= ctx->nlev) return PMG_ERR_ARG;
  const int v = (level < 16 && ctx->level_variant[level] >= 0) ? ctx->level_variant[level] : ctx->variant;
  if (variant) *variant = v;
  if (ms_per_variant)
    for (int k = 0; k < NUM_VARIANTS; ++k) ms_per_variant[k] = level < 16 ? ctx->level_ms[level][k] : -1.f;
  return PMG_OK;
}

int pmg_level_persistent(const pmg_ctx* ctx, int level, int* on, float* ms_per_colour, float* ms_persistent) {
  if (!ctx || !ctx->setup_ok || level < 0 || level >= ctx->nlev) return PMG_ERR_ARG;
  const bool in = level < 16 && !ctx->um;
  if (on) *on = in && ctx->level_persist[level] ? 1 : 0;
  if (ms_per_colour) *ms_per_colour = in ? ctx->persist_ms[level][0] : -1.f;
  if (ms_persistent) *ms_persistent = in ? ctx->persist_ms[level][1] : -1.f;
  return PMG_OK;
}

int pmg_level_dense_local(const pmg_ctx* ctx, int level, int* on, float* ms_matrix_free, float* ms_tabulated) {
  if (!ctx || !ctx->setup_ok || level < 0 || level >= ctx->nlev) return PMG_ERR_ARG;
  const bool in = level < 16 && !ctx->um;
  if (on) *on = in && ctx->solve_table[level].on ? 1 : 0;
  if (ms_matrix_free) *ms_matrix_free = in ? ctx->dense_ms[level][0] : -1.f;
  if (ms_tabulated) *ms_tabulated = in ? ctx->dense_ms[level][1] : -1.f;
  return PMG_OK;
}

int pmg_tuning(const pmg_ctx* ctx, int* variant, int* threads, int* ppb_out, float* ms) {
  if (!ctx || !ctx->setup_ok) return PMG_ERR_ARG;
  size_t sm;
  int ppb, nt;
  const bool mixed = ctx->opt.precision == PMG_PREC_MIXED;
  if (ctx->dim == 2) {
    if (mixed) patch_config<2, float>(ctx->p, ctx->variant, &sm, &ppb, &nt);
    else patch_config<2, double>(ctx->p, ctx->variant, &sm, &ppb, &nt);
  } else {
    if (mixed) patch_config<3, float>(ctx->p, ctx->variant, &sm, &ppb, &nt);
    else patch_config<3, double>(ctx->p, ctx->variant, &sm, &ppb, &nt);
  }
  if (variant) *variant = ctx->variant;
  if (threads) *threads = nt;
  if (ppb_out) *ppb_out = ppb;
  if (ms)
    for (int v = 0; v < NUM_VARIANTS; ++v) ms[v] = ctx->variant_ms[v];
  return PMG_OK;
}

int pmg_features(pmg_ctx* ctx, int level, int k, float* X, void* stream) {
  int st = check_level(ctx, level);
  if (st) return st;
  PMG_GUARD_CTX(ctx);
  if (ctx->um) return fail(ctx, PMG_ERR_UNSUPPORTED, "not available on unstructured meshes");
  if (k < 0 || k >= ctx->npl || !X) return fail(ctx, PMG_ERR_ARG, "bad p-level or null output");
  HLevel& h = ctx->L[level];
  ST(features_launch(ctx->dim, h.coords, h.kappa, h.N, h.pl[k].q, ctx->npl - 1 - k, (int)h.npatch, X,
                     (cudaStream_t)stream));
  return PMG_OK;
}

int pmg_set_mlp(pmg_ctx* ctx, const float* params, const float* norm) {
  if (!ctx || !params || !norm) return PMG_ERR_ARG;
  PMG_GUARD_CTX(ctx);
  if (!ctx->mlp_params) DALLOC(ctx->mlp_params, PMG_MLP_NPARAM);
  if (!ctx->mlp_norm) DALLOC(ctx->mlp_norm, PMG_MLP_NNORM);
  for (int i = 0; i < 16; ++i)
    if (!(norm[16 + i] > 0)) return fail(ctx, PMG_ERR_ARG, "feature standard deviations must be positive");
  if (!(norm[34] > 0) || !(norm[35] > 0)) return fail(ctx, PMG_ERR_ARG, "target standard deviations must be positive");
  CU(cudaMemcpy(ctx->mlp_params, params, PMG_MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(ctx->mlp_norm, norm, PMG_MLP_NNORM * sizeof(float), cudaMemcpyHostToDevice));
  return PMG_OK;
}

int pmg_mlp_targets(pmg_ctx* ctx, int level, int k, float* T, void* stream) {
  int st = check_level(ctx, level);
  if (st) return st;
  PMG_GUARD_CTX(ctx);
  if (ctx->um) return fail(ctx, PMG_ERR_UNSUPPORTED, "not available on unstructured meshes");
  if (k < 0 || k >= ctx->npl || !T) return fail(ctx, PMG_ERR_ARG, "bad p-level or null output");
  const HLevel& h = ctx->L[level];
  if (h.pl[k].q < 2) return fail(ctx, PMG_ERR_ARG, "the p = 1 level has no Lanczos estimates");
  ST(targets_launch(h.pl[k].ritz, (int64_t)h.npatch, T, (cudaStream_t)stream));
  return PMG_OK;
}

// file layout: 8-byte magic "PMGMLP1", uint32 parameter count, uint32
// normalisation count, the parameters, the normalisation floats (host byte order)
static const char kMlpMagic[8] = {'P', 'M', 'G', 'M', 'L', 'P', '1', 0};

int pmg_mlp_save(pmg_ctx* ctx, const char* path) {
  if (!ctx || !path) return PMG_ERR_ARG;
  if (!ctx->mlp_params) return fail(ctx, PMG_ERR_ARG, "no network installed (pmg_set_mlp or pmg_mlp_load)");
  PMG_GUARD_CTX(ctx);
  std::vector<float> prm(PMG_MLP_NPARAM), nrm(PMG_MLP_NNORM);
  CU(cudaMemcpy(prm.data(), ctx->mlp_params, prm.size() * sizeof(float), cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(nrm.data(), ctx->mlp_norm, nrm.size() * sizeof(float), cudaMemcpyDeviceToHost));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(ctx, PMG_ERR_ARG, "cannot open the file for writing");
  const uint32_t counts[2] = {PMG_MLP_NPARAM, PMG_MLP_NNORM};
  bool ok = std::fwrite(kMlpMagic, 1, 8, f) == 8 && std::fwrite(counts, sizeof(uint32_t), 2, f) == 2 &&
            std::fwrite(prm.data(), sizeof(float), prm.size(), f) == prm.size() &&
            std::fwrite(nrm.data(), sizeof(float), nrm.size(), f) == nrm.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? PMG_OK : fail(ctx, PMG_ERR_ARG, "short write");
}

int pmg_mlp_load(pmg_ctx* ctx, const char* path) {
  if (!ctx || !path) return PMG_ERR_ARG;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(ctx, PMG_ERR_ARG, "cannot open the file");
  char magic[8] = {};
  uint32_t counts[2] = {0, 0};
  std::vector<float> prm(PMG_MLP_NPARAM), nrm(PMG_MLP_NNORM);
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMlpMagic, 8) == 0 &&
            std::fread(counts, sizeof(uint32_t), 2, f) == 2 && counts[0] == PMG_MLP_NPARAM &&
            counts[1] == PMG_MLP_NNORM && std::fread(prm.data(), sizeof(float), prm.size(), f) == prm.size() &&
            std::fread(nrm.data(), sizeof(float), nrm.size(), f) == nrm.size();
  std::fclose(f);
  if (!ok) return fail(ctx, PMG_ERR_ARG, "not a network file of this library (magic, sizes or length)");
  return pmg_set_mlp(ctx, prm.data(), nrm.data());
}

int pmg_launch_count(const pmg_ctx* ctx, int64_t* n) {
  if (!ctx || !n) return PMG_ERR_ARG;
  *n = ctx->launches + (ctx->um ? umesh_kernel_launches(ctx->um) : 0);
  return PMG_OK;
}

int pmg_fma_peak(pmg_ctx* ctx, int precision, double* flops) {
  if (!ctx || !flops) return PMG_ERR_ARG;
  PMG_GUARD_CTX(ctx);
  int nsm = 0;
  CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
  const int block = 256, grid = nsm * 8;
  cudaStream_t s = ctx->stream;
  void* out = nullptr;
  CU(cudaMalloc(&out, (size_t)grid * block * sizeof(double)));
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  double best = 0.0;
  int iters = precision == PMG_PREC_FP64 ? 2000 : 20000;
  for (int rep = 0; rep < 4; ++rep) {
    CU(cudaEventRecord(e0, s));
    if (precision == PMG_PREC_FP64) ST(launch_fma_chain<double>((double*)out, grid, block, iters, s));
    else ST(launch_fma_chain<float>((float*)out, grid, block, iters, s));
    CU(cudaEventRecord(e1, s));
    CU(cudaEventSynchronize(e1));
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, e0, e1));
    const double f = 2.0 * 32.0 * iters * (double)grid * block / (ms * 1e-3);
    best = std::max(best, f);
    if (ms < 50.f) iters = (int)std::min<double>(iters * (60.0 / std::max(ms, 0.01f)), 2e8);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  *flops = best;
  return PMG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// internal accessors (lanczos_view.h)
namespace pmg {

int lanczos_view(const pmg_ctx* ctx, int level, int k, LanczosView* v) {
  if (!ctx || !v || !ctx->setup_ok || level < 0 || level >= ctx->nlev || k < 0 || k >= ctx->npl) return PMG_ERR_ARG;
  const HLevel& h = ctx->L[level];
  v->device = ctx->device;
  v->dim = ctx->dim;
  v->N = h.N;
  v->q = h.pl[k].q;
  v->ksteps = ctx->opt.lanczos_steps;
  v->npatch = (int64_t)h.npatch;
  v->G64 = h.pl[k].G64;
  v->dinv64 = h.pl[k].dinv64;
  v->G32 = h.pl[k].G32;
  v->dinv32 = h.pl[k].dinv32;
  v->seed = ctx->opt.seed;
  v->safety = ctx->opt.bound_safety;
  v->ratio = ctx->opt.bound_ratio;
  return PMG_OK;
}

int set_last_error(pmg_ctx* ctx, int code, const char* msg) { return fail(ctx, code, msg); }

}  // namespace pmg
