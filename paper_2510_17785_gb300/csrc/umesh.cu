// Host side of the unstructured-mesh path: set-up (topology, DoF maps,
// patches, colours, geometry, diagonals, Q1 coarse space), the sweeps, the
// local solves, the Lanczos intervals and the two-level preconditioner.  The
// kernels and the design notes are in umesh_kern.cuh.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "basis.h"
#include "umesh_kern.cuh"
#include "umesh.h"
#include "utopo.h"

namespace pmg {

// ------------------------------------------------------ h-transfers between meshes
// The fine mesh is the uniform refinement of the coarse one and a fine cell
// lies in its parent's reference frame, so the embedding is, per fine cell,
// the tensor product of the 1D half-interval interpolations
// H[b][a][m] = l_m((b + xi_a) / 2) (degree q, Gauss-Lobatto nodes xi), b the
// child's bit along the axis: d one-dimensional passes over the cell.

// one pass along axis `ax` of the (q+1)^d cell array: out = H_b (TRANS: H_b^T) in
template <int DIM, bool TRANS, typename T>
__device__ void uh_pass(const T* in, T* out, const double* __restrict__ H, int child, int ax, int n) {
  int s = 1;
  for (int k = 0; k < ax; ++k) s *= n;
  int nl = 1;
  for (int k = 0; k < DIM; ++k) nl *= n;
  const double* Hb = H + ((child >> ax) & 1) * n * n;
  for (int e = threadIdx.x; e < nl; e += blockDim.x) {
    const int lo = e % s, o = (e / s) % n, hi = e / (s * n);
    T acc = T(0);
    for (int j = 0; j < n; ++j) {
      const T h = TRANS ? T(Hb[j * n + o]) : T(Hb[o * n + j]);
      acc += h * in[lo + s * (j + n * hi)];
    }
    out[e] = acc;
  }
  __syncthreads();
}

// Y[c][l] = (embedded parent values) at fine node l of cell c
template <int DIM, typename T>
__global__ void __launch_bounds__(128) k_uh_prolong_cells(const T* __restrict__ xc, const int32_t* __restrict__ cdofs_c,
                                                          const int32_t* __restrict__ parent,
                                                          const uint8_t* __restrict__ child, int64_t nc, int q,
                                                          const double* __restrict__ H, T* __restrict__ Y) {
  const int n = q + 1;
  const int nl = DIM == 3 ? n * n * n : n * n;
  T* a = reinterpret_cast<T*>(pmg_smem);
  T* b = a + nl;
  for (int64_t c = blockIdx.x; c < nc; c += gridDim.x) {
    const int32_t P = parent[c];
    const int k = child[c];
    for (int e = threadIdx.x; e < nl; e += blockDim.x) a[e] = xc[cdofs_c[(size_t)P * nl + e]];
    __syncthreads();
    uh_pass<DIM, false>(a, b, H, k, 0, n);
    uh_pass<DIM, false>(b, a, H, k, 1, n);
    const T* res = a;
    if (DIM == 3) {
      uh_pass<DIM, false>(a, b, H, k, 2, n);
      res = b;
    }
    for (int e = threadIdx.x; e < nl; e += blockDim.x) Y[(size_t)c * nl + e] = res[e];
    __syncthreads();
  }
}

// Yc[c][m] = sum_l H^T (fine residual at l / number of cells holding it)
template <int DIM, typename T>
__global__ void __launch_bounds__(128) k_uh_restrict_cells(const T* __restrict__ rf, const int32_t* __restrict__ cdofs_f,
                                                           const int32_t* __restrict__ dstart_f,
                                                           const uint8_t* __restrict__ bnd_f,
                                                           const uint8_t* __restrict__ child, int64_t nc, int q,
                                                           const double* __restrict__ H, T* __restrict__ Yc) {
  const int n = q + 1;
  const int nl = DIM == 3 ? n * n * n : n * n;
  T* a = reinterpret_cast<T*>(pmg_smem);
  T* b = a + nl;
  for (int64_t c = blockIdx.x; c < nc; c += gridDim.x) {
    const int k = child[c];
    for (int e = threadIdx.x; e < nl; e += blockDim.x) {
      const int32_t g = cdofs_f[(size_t)c * nl + e];
      a[e] = bnd_f[g] ? T(0) : rf[g] / T(dstart_f[g + 1] - dstart_f[g]);
    }
    __syncthreads();
    uh_pass<DIM, true>(a, b, H, k, 0, n);
    uh_pass<DIM, true>(b, a, H, k, 1, n);
    const T* res = a;
    if (DIM == 3) {
      uh_pass<DIM, true>(a, b, H, k, 2, n);
      res = b;
    }
    for (int e = threadIdx.x; e < nl; e += blockDim.x) Yc[(size_t)c * nl + e] = res[e];
    __syncthreads();
  }
}

// xf[g] += Y at the first (cell, node) entry of fine DoF g (0 on Dirichlet DoFs)
template <typename T>
__global__ void k_uh_add_first(const T* __restrict__ Y, const int32_t* __restrict__ dstart,
                               const int32_t* __restrict__ dlist, const uint8_t* __restrict__ bnd, int64_t n,
                               T* __restrict__ xf) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    if (!bnd[g]) xf[g] += Y[dlist[dstart[g]]];
}

// rc[G] = sum over the (coarse cell, node) entries of G and the cell's children
// of Yc (fixed order); 0 on Dirichlet DoFs
template <typename T>
__global__ void k_uh_assemble_coarse(const T* __restrict__ Yc, const int32_t* __restrict__ dstart_c,
                                     const int32_t* __restrict__ dlist_c, const int32_t* __restrict__ children,
                                     const uint8_t* __restrict__ bnd_c, int64_t n, int nl, int nch,
                                     T* __restrict__ rc) {
  for (int64_t G = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; G < n; G += (int64_t)gridDim.x * blockDim.x) {
    T s = T(0);
    if (!bnd_c[G])
      for (int e = dstart_c[G]; e < dstart_c[G + 1]; ++e) {
        const int32_t P = dlist_c[e] / nl, m = dlist_c[e] - P * nl;
        for (int j = 0; j < nch; ++j) s += Yc[(size_t)children[(size_t)P * nch + j] * nl + m];
      }
    rc[G] = s;
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
  double *dinv64 = nullptr, *bounds64 = nullptr, *ritz64 = nullptr;
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
  bool kappa_given = false;
  // mesh hierarchy: this mesh refines `coarser` (NULL on the coarsest mesh)
  UMesh* coarser = nullptr;
  std::vector<int32_t> h_parent, h_children;   // [nc] parents; [coarser->nc][2^d] children
  std::vector<uint8_t> h_child;
  int32_t *d_parent = nullptr, *d_children = nullptr;
  uint8_t* d_child = nullptr;
  double* d_H = nullptr;                        // [2][q+1][q+1] half-interval interpolation, degree p
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
  m->kappa_given = true;
  return ST_OK;
}

bool umesh_kappa_given(const UMesh* m) { return m->kappa_given; }
int64_t umesh_ncells(const UMesh* m) { return m->nc; }

int umesh_set_parent(UMesh* fine, UMesh* coarse, const int64_t* parent, const uint8_t* child, std::string* msg) {
  const int nch = 1 << fine->dim;
  if (coarse->dim != fine->dim) {
    *msg = "the meshes of a hierarchy have one dimension";
    return ST_ARG;
  }
  if (fine->nc != coarse->nc * nch) {
    *msg = "a refined mesh has 2^dim cells per coarse cell";
    return ST_ARG;
  }
  std::vector<int32_t> ch((size_t)coarse->nc * nch, -1);
  for (int64_t c = 0; c < fine->nc; ++c) {
    const int64_t P = parent[c];
    const int k = child[c];
    if (P < 0 || P >= coarse->nc || k >= nch || ch[(size_t)P * nch + k] >= 0) {
      *msg = "parent_cell / child_index: every coarse cell needs its 2^dim children, each child index once";
      return ST_ARG;
    }
    ch[(size_t)P * nch + k] = (int32_t)c;
  }
  fine->coarser = coarse;
  fine->h_parent.assign(fine->nc, 0);
  fine->h_child.assign(child, child + fine->nc);
  for (int64_t c = 0; c < fine->nc; ++c) fine->h_parent[c] = (int32_t)parent[c];
  fine->h_children = ch;
  return ST_OK;
}

int umesh_kappa_from_children(UMesh* coarse, const UMesh* fine) {
  const int nch = 1 << fine->dim;
  std::vector<double> k(coarse->nc, 0.0);
  for (int64_t P = 0; P < coarse->nc; ++P) {
    double s = 0.0;
    for (int j = 0; j < nch; ++j) s += fine->h_kappa[fine->h_children[(size_t)P * nch + j]];
    k[P] = s / nch;
  }
  coarse->h_kappa = k;
  return ST_OK;
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

// dynamic shared memory of the patch kernel without its workspace, degree p
template <int DIM, typename T>
static size_t upatch_base_bytes(int p) {
  switch (p) {
    case 1: return upatch_smem_aligned<DIM, 1, T>();
    case 2: return upatch_smem_aligned<DIM, 2, T>();
    case 3: return upatch_smem_aligned<DIM, 3, T>();
    case 4: return upatch_smem_aligned<DIM, 4, T>();
    case 5: return upatch_smem_aligned<DIM, 5, T>();
    case 6: return upatch_smem_aligned<DIM, 6, T>();
    case 7: return upatch_smem_aligned<DIM, 7, T>();
    default: return upatch_smem_aligned<DIM, 8, T>();
  }
}

template <typename T>
static void fill_args(UMesh* m, UPatchArgs<T>& a) {
  std::memset(&a, 0, sizeof(a));
  a.p_cells = m->p_cells;
  a.p_ncell = m->p_ncell;
  a.p_vertex = m->p_vertex;
  a.n_patches = (int)m->pverts.size();
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
  // the workspace slice moves into shared memory when CTA and slice fit 100 KB (two CTAs per SM)
  const size_t base = m->dim == 2 ? upatch_base_bytes<2, T>(m->p) : upatch_base_bytes<3, T>(m->p);
  a.ws_shared = base + m->ws_stride * sizeof(T) <= 100 * 1024 ? 1 : 0;
  a.yoff = m->yoff;
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
    UCK(m->upload(&L.ritz64, std::vector<double>(2 * np, 0.0)));
    ymax = std::max(ymax, (size_t)umesh_max_valence(m) * L.nloc);   // cell outputs of the largest patch
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
  if (o.coarse_space) {
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
int64_t umesh_kernel_launches(const UMesh* m) {
  int64_t n = 0;
  for (const UMesh* x = m; x; x = x->coarser) n += x->launches;   // the chain's V-cycle launches them all
  return n;
}
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


template <int DIM>
static int ulanczos_launch_p(int p, const UPatchArgs<double>& a, const ULanczos& z, int grid, cudaStream_t s) {
  switch (p) {
    case 2: return ulanczos_launch<DIM, 2>(a, z, grid, s);
    case 3: return ulanczos_launch<DIM, 3>(a, z, grid, s);
    case 4: return ulanczos_launch<DIM, 4>(a, z, grid, s);
    case 5: return ulanczos_launch<DIM, 5>(a, z, grid, s);
    case 6: return ulanczos_launch<DIM, 6>(a, z, grid, s);
    case 7: return ulanczos_launch<DIM, 7>(a, z, grid, s);
    case 8: return ulanczos_launch<DIM, 8>(a, z, grid, s);
    default: return ST_UNSUPPORTED;
  }
}

int umesh_lanczos(UMesh* m, int ksteps, uint64_t seed, double safety, double ratio, cudaStream_t s) {
  const int64_t np = (int64_t)m->pverts.size();
  if (np == 0 || m->p < 2) return ST_OK;
  if (ksteps < 1 || ksteps > 64) return ST_ARG;
  UPatchArgs<double> a;
  fill_args(m, a);
  a.ws_shared = 0;                                   // the Lanczos kernel keeps its slices in global memory
  const int grid = (int)std::min<int64_t>(np, std::min<int64_t>(m->ws_grid, 152 * 2));
  ULanczos z{};
  z.stride = ((size_t)(ksteps + 3) * m->L[0].nimax + 31) & ~size_t(31);
  if (cudaMalloc(&z.V, z.stride * grid * sizeof(double)) != cudaSuccess) return ST_CUDA;
  z.ksteps = ksteps;
  z.seed = seed;
  z.safety = safety;
  z.ratio = ratio;
  int st = ST_OK;
  for (int k = 0; k < m->npl && !st; ++k) {
    if (m->L[k].q == 1) continue;
    z.level = k;
    z.ritz = m->L[k].ritz64;
    z.b64 = m->L[k].bounds64;
    z.b32 = m->L[k].bounds32;
    st = m->dim == 2 ? ulanczos_launch_p<2>(m->p, a, z, grid, s) : ulanczos_launch_p<3>(m->p, a, z, grid, s);
    ++m->launches;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) st = ST_CUDA;
  cudaFree(z.V);
  return st;
}

int umesh_get_ritz(const UMesh* m, int k, double* out) {
  if (k < 0 || k >= m->npl) return ST_ARG;
  const size_t np = m->pverts.size();
  if (np && cudaMemcpy(out, m->L[k].ritz64, 2 * np * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return ST_CUDA;
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

// the work vectors of a mesh in precision T
template <typename T>
struct UVec {
  T *x, *b, *r, *Y, *r1, *x1;
};
template <typename T>
UVec<T> uvec(UMesh* m);
template <>
UVec<double> uvec<double>(UMesh* m) { return {m->x64, m->b64, m->r64, m->Y64, m->r1_64, m->x1_64}; }
template <>
UVec<float> uvec<float>(UMesh* m) { return {m->x32, m->b32, m->r32, m->Y32, m->r1_32, m->x1_32}; }

int umesh_link(UMesh* m, cudaStream_t s, std::string* msg) {
  if (!m->coarser) return ST_OK;
  const UMesh* c = m->coarser;
  if (c->p != m->p || c->opt.precision != m->opt.precision) {
    *msg = "the meshes of a hierarchy share the degree and the precision";
    return ST_ARG;
  }
  const int q = m->p, n = q + 1;
  const std::vector<double> xi = gauss_lobatto(q);
  std::vector<double> H(2 * n * n);
  for (int b = 0; b < 2; ++b) {
    std::vector<double> pts(n);
    for (int a = 0; a < n; ++a) pts[a] = 0.5 * (b + xi[a]);
    const auto L = lagrange_matrix(xi, pts);          // L[a][mm] = l_mm(pts_a)
    for (int a = 0; a < n; ++a)
      for (int mm = 0; mm < n; ++mm) H[(b * n + a) * n + mm] = L[a][mm];
  }
  UCK(m->upload(&m->d_H, H));
  UCK(m->upload(&m->d_parent, m->h_parent));
  UCK(m->upload(&m->d_child, m->h_child));
  UCK(m->upload(&m->d_children, m->h_children));
  (void)s;
  return ST_OK;
}

// the V-cycle over the chain of meshes ending at m: x = B b in precision T
template <typename T>
static int uvcycle_chain_T(UMesh* m, const T* b, T* x, cudaStream_t s) {
  UVec<T> v = uvec<T>(m);
  if (!m->coarser) return uvcycle_T<T>(m, b, x, v.r, v.Y, v.r1, v.x1, s);
  UMesh* c = m->coarser;
  UVec<T> vc = uvec<T>(c);
  const ULevelD& L0 = m->L[0];
  const ULevelD& C0 = c->L[0];
  const size_t n = (size_t)L0.ndofs;
  const int q = L0.q, nl = L0.nloc, nch = 1 << m->dim;
  const int grid = (int)std::min<int64_t>(m->nc, 152 * 16);
  const size_t sm = 2 * (size_t)nl * sizeof(T);
  UCK(launch_fill<T>(x, n, T(0), s));
  UCK(usweep_T<T>(m, b, x, false, s));                     // pre-smoothing on this mesh
  UCK(uglobal_apply<T>(m, 0, x, v.r, v.Y, s));              // r = b - A x
  UCK(launch_sub_from<T>(b, v.r, n, s));
  if (m->dim == 2)                                          // restriction to the coarser mesh
    k_uh_restrict_cells<2, T><<<grid, 128, sm, s>>>(v.r, L0.cdofs, L0.dstart, L0.bnd, m->d_child, m->nc, q, m->d_H, v.Y);
  else
    k_uh_restrict_cells<3, T><<<grid, 128, sm, s>>>(v.r, L0.cdofs, L0.dstart, L0.bnd, m->d_child, m->nc, q, m->d_H, v.Y);
  k_uh_assemble_coarse<T><<<grid_for((size_t)C0.ndofs, 256), 256, 0, s>>>(v.Y, C0.dstart, C0.dlist, m->d_children,
                                                                          C0.bnd, C0.ndofs, nl, nch, vc.b);
  UCU(cudaPeekAtLastError());
  UCK(uvcycle_chain_T<T>(c, vc.b, vc.x, s));                // the coarser meshes
  if (m->dim == 2)                                          // prolongation of the correction
    k_uh_prolong_cells<2, T><<<grid, 128, sm, s>>>(vc.x, C0.cdofs, m->d_parent, m->d_child, m->nc, q, m->d_H, v.Y);
  else
    k_uh_prolong_cells<3, T><<<grid, 128, sm, s>>>(vc.x, C0.cdofs, m->d_parent, m->d_child, m->nc, q, m->d_H, v.Y);
  k_uh_add_first<T><<<grid_for(n, 256), 256, 0, s>>>(v.Y, L0.dstart, L0.dlist, L0.bnd, L0.ndofs, x);
  UCU(cudaPeekAtLastError());
  m->launches += 4;
  return usweep_T<T>(m, b, x, true, s);                     // post-smoothing, colours reversed
}

int umesh_precondition(UMesh* m, const double* r, double* z, cudaStream_t s) {
  const size_t n = (size_t)m->L[0].ndofs;
  if (m->opt.precision == PMG_PREC_MIXED) {
    UCK(launch_cast_d2f(r, m->b32, n, s));
    UCK(uvcycle_chain_T<float>(m, m->b32, m->x32, s));
    UCK(launch_cast_f2d(m->x32, z, n, s));
    m->launches += 2;
    return ST_OK;
  }
  UCU(cudaMemcpyAsync(m->b64, r, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  UCK(uvcycle_chain_T<double>(m, m->b64, m->x64, s));
  UCU(cudaMemcpyAsync(z, m->x64, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  return ST_OK;
}

}  // namespace pmg
