// Internal interface of the unstructured-mesh path (umesh.cu): the vertex-
// patch smoother with the local p-multigrid solver on quadrilateral /
// hexahedral meshes of arbitrary topology, the global operator, and a
// two-level preconditioner (patch sweeps on Q_p, the Q1 space of the same
// mesh as coarse space, dense Cholesky) for CG.  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace pmg {

struct UMesh;

struct UOptions {
  int precision;         // PMG_PREC_*
  int smoother;          // 0 Chebyshev, 1 Jacobi
  int cheb_degree;
  double omega;
  int n_mg;
  double fixed_lo, fixed_hi;
  uint64_t seed;         // colouring priority
  bool coarse_space = true;  // build the Q1 coarse space (the coarsest mesh of a hierarchy only)
};

// host mesh (copied); kappa may be empty (1 everywhere)
UMesh* umesh_create(int dim, int64_t nv, const double* coords, int64_t nc, const int64_t* cells,
                    const uint8_t* vertex_on_boundary, std::string* msg);
void umesh_destroy(UMesh* m);
int umesh_set_kappa(UMesh* m, const double* kappa);     // nc values
// `fine` is the uniform refinement of `coarse`: fine cell c is child child[c]
// (corner bits in the parent's reference frame) of coarse cell parent[c]
int umesh_set_parent(UMesh* fine, UMesh* coarse, const int64_t* parent, const uint8_t* child, std::string* msg);
// kappa of a coarse mesh not given by the user: arithmetic mean of its children's
int umesh_kappa_from_children(UMesh* coarse, const UMesh* fine);
bool umesh_kappa_given(const UMesh* m);
int64_t umesh_ncells(const UMesh* m);
// after both meshes are set up: the h-transfer tables (degree p)
int umesh_link(UMesh* fine, cudaStream_t s, std::string* msg);
// build everything for degree p (p-levels p, p/2, ..., 1); ST_* codes, msg on error
int umesh_setup(UMesh* m, int p, const UOptions& o, cudaStream_t s, int* err_dev, std::string* msg);

int64_t umesh_ndofs(const UMesh* m);
int64_t umesh_nfree(const UMesh* m);
int64_t umesh_npatch(const UMesh* m);
int umesh_ncolours(const UMesh* m);
int umesh_nplevels(const UMesh* m, int* q);
int64_t umesh_kernel_launches(const UMesh* m);
// host copies of the integer structures
int umesh_cell_dofs(const UMesh* m, int k, int32_t* out);             // [nc][(q+1)^d]
int umesh_patches(const UMesh* m, int64_t* out, int width);           // [npatch][width]: vertex, cells (-1)
int umesh_colours(const UMesh* m, uint8_t* out);
int umesh_get_bounds(const UMesh* m, int k, double* out);             // [npatch][2]
int umesh_set_bounds(UMesh* m, int k, const double* lohi);            // [npatch][2]
int umesh_max_valence(const UMesh* m);
// Lanczos intervals of every p-level q > 1 (FP64 operator; synchronises s)
int umesh_lanczos(UMesh* m, int ksteps, uint64_t seed, double safety, double ratio, cudaStream_t s);
int umesh_get_ritz(const UMesh* m, int k, double* out);              // [npatch][2] (theta_min, theta_max)

// FP64 vectors of length umesh_ndofs (caller's device memory)
int umesh_apply(UMesh* m, const double* u, double* Au, cudaStream_t s);
int umesh_sweep(UMesh* m, const double* b, double* u, int n_sweeps, bool reverse, cudaStream_t s);
int umesh_sweep_colour(UMesh* m, int colour, const double* b, double* u, cudaStream_t s);
// local solves of patches ids[0..n): r, d are [n][n_interior_max] (rows padded)
int umesh_local(UMesh* m, int64_t n, const int64_t* ids_dev, const double* r, double* d, int n_cycles,
                cudaStream_t s);
int64_t umesh_interior_max(const UMesh* m);
// z = M r: the V-cycle over the mesh chain ending at m (fine sweeps, h-restriction,
// ..., the coarsest mesh's two-level cycle, ...), FP64 in and out
int umesh_precondition(UMesh* m, const double* r, double* z, cudaStream_t s);
// zero the Dirichlet DoFs of x
int umesh_mask(UMesh* m, double* x, cudaStream_t s);

}  // namespace pmg
