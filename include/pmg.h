/*
 * pmg.h -- C ABI of the GB300 vertex-patch smoother with a nested matrix-free
 * p-multigrid local solver (M. Wichrowski, "Local Solvers for High-Order Patch
 * Smoothers via p-Multigrid", arXiv 2510.17785).
 *
 * The library discretises a(u, v) = int kappa grad u . grad v (Section 2,
 * eq. bilinear-form) with continuous Q_p Lagrange elements on Gauss-Lobatto
 * support points over a structured (N^d cells, d = 2 or 3) mesh of the unit
 * square/cube whose vertices may be displaced arbitrarily (Q1 cell geometry),
 * with homogeneous Dirichlet conditions on the boundary.  Integrals use the
 * (q+1)-point Gauss rule per direction at degree q.
 *
 * Conventions shared by every entry point
 *  - Every function returns an int status (PMG_OK = 0 or a PMG_ERR_* code);
 *    pmg_last_error() returns a message for the last failure on a context.
 *  - Host arrays passed in are caller-owned and copied before the call returns.
 *  - Vector arguments named *_dev are caller-owned DEVICE pointers to FP64
 *    arrays of length (p*N_l+1)^d in the global lexicographic DoF order of
 *    level l (x fastest).  Entries on Dirichlet DoFs are ignored on input and
 *    written as 0 on output.  The library never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Calls are asynchronous on that stream unless stated otherwise.
 *  - Mesh level l = 0 is the coarsest mesh, l = n_levels-1 the finest.
 *  - The context owns every derived structure (geometry tensors, diagonals,
 *    patch lists, eigenvalue bounds, coarse factor, work vectors).
 *  - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef PMG_H
#define PMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
enum {
  PMG_OK = 0,
  PMG_ERR_ARG = 1,           /* invalid argument (size, pointer, state)        */
  PMG_ERR_CUDA = 2,          /* a CUDA runtime call failed                     */
  PMG_ERR_DEGENERATE = 3,    /* det J <= 0 at a Gauss point or vertex of a cell */
  PMG_ERR_NOT_CONVERGED = 4, /* the solver hit maxit before rtol              */
  PMG_ERR_NUMERIC = 5,       /* NaN or Inf in a residual norm                  */
  PMG_ERR_TIMEOUT = 6,       /* a bounded device wait gave up                  */
  PMG_ERR_UNSUPPORTED = 7    /* e.g. p > 8, or a precision/degree combination  */
};

/* Largest number of cells around a vertex (the valence of a vertex patch)
 * that the unstructured-mesh kernels accept. */
#define PMG_UMAXC 32

/* Number of launch-shape variants of the patch-sweep kernel (pmg_tuning). */
#define PMG_NUM_VARIANTS 16

/* ---- options ----------------------------------------------------------- */
enum { PMG_SMOOTHER_CHEBYSHEV = 0, PMG_SMOOTHER_JACOBI = 1, PMG_SMOOTHER_CARTESIAN = 2 };
enum { PMG_BOUNDS_LANCZOS = 0, PMG_BOUNDS_FIXED = 1, PMG_BOUNDS_USER = 2,
       PMG_BOUNDS_MLP = 3   /* learned intervals (pmg_set_mlp), see below      */ };
enum { PMG_PREC_FP64 = 0,  /* everything in FP64                               */
       PMG_PREC_MIXED = 1  /* patch smoother, local p-MG and GMG levels in FP32;
                              outer CG, its residuals and dots, and the coarse
                              solve in FP64                                   */ };

typedef struct pmg_options {
  int smoother;          /* PMG_SMOOTHER_*: smoother on every local p-level:
                            Chebyshev iteration on D^-1 A; damped Jacobi
                            d += omega D^-1 (r - A d); Cartesian-reinforced
                            d += omega D^-1 diag(A_b) A_b^-1 (r - A d), A_b the
                            reference Cartesian patch operator inverted by fast
                            diagonalisation (Section 3.1).  The last is not a
                            symmetric step: precondition GMRES with it, as the
                            paper does, not CG                              */
  int cheb_degree;       /* Chebyshev polynomial degree (k), >= 1              */
  double jacobi_omega;   /* damping omega of the Jacobi and Cartesian-reinforced
                            steps (paper: 1/2)                                 */
  int n_mg;              /* local V-cycles per patch solve (N_MG, >= 1)        */
  int bounds;            /* PMG_BOUNDS_*: source of the Chebyshev intervals    */
  int lanczos_steps;     /* Lanczos steps per (patch, p-level)                 */
  double bound_safety;   /* hi = safety * theta_max                            */
  double bound_ratio;    /* lo = max(theta_min, hi / ratio)                    */
  double fixed_lo, fixed_hi; /* interval used with PMG_BOUNDS_FIXED           */
  uint64_t seed;         /* seed of the Lanczos start vectors                  */
  int precision;         /* PMG_PREC_*                                         */
  int autotune;          /* 1: pmg_setup times the launch-shape variants of the
                            patch sweep on one colour of every mesh level and
                            keeps the fastest per level; 2: the same without
                            the latency-oriented shapes (variants 3 and 6),
                            for problems that share the GPU (batched solves);
                            0: use `variant` everywhere                       */
  int variant;           /* launch-shape variant when autotune = 0 (0 = default) */
  double mlp_safety;     /* PMG_BOUNDS_MLP: hi = mlp_safety * predicted theta_max */
  int coarse_kappa;      /* coefficient of a coarse cell from its 2^d children:
                            PMG_KAPPA_ARITHMETIC, _GEOMETRIC or _HARMONIC mean  */
  int post_reverse;      /* 1: post-smoothing sweeps the colours in reverse
                            order (symmetric V-cycle, for CG; default);
                            0: same order as pre-smoothing (Section 4; GMRES) */
  int additive;          /* 0: multiplicative sweep (Algorithm 1, default);
                            1: weighted additive sweep: every patch solves with
                            the residual of the same u and
                            u += theta W sum_j Pi_j^T d_j, W = diag(1/m), m the
                            number of patches whose interior holds the DoF; a
                            reversed sweep (post-smoothing) applies W to the
                            residual instead, so the V-cycle stays symmetric  */
  double additive_theta; /* theta of the additive sweep (default 1)          */
  int persistent;        /* multiplicative sweeps of a mesh level as ONE
                            cooperative launch over all its colours, CTAs
                            meeting at a grid barrier between colours:
                            1 (default): pmg_setup times it against the
                            per-colour launches on every level with at most
                            4096 patches and keeps the faster (not with
                            autotune = 2, whose problems share the GPU);
                            2: on every level; 0: never                     */
  long long sync_budget; /* clock64 cycles a CTA waits at one grid barrier of
                            a persistent sweep before it gives up: the sweep
                            stops and the call that synchronises next
                            (pmg_solve_cg, pmg_solve_cg_host, pmg_solve_gmres,
                            pmg_batch_solve_cg, pmg_patch_smooth) returns
                            PMG_ERR_TIMEOUT; 0 = 2^31                         */
  int geometry_bf16;     /* PMG_PREC_MIXED only, 1: the patch kernels (local
                            p-MG and the Evaluate step) read the geometry
                            tensors G rounded to BF16 (8-bit significand,
                            round to nearest even); the GMG level operators
                            keep FP32 G.  The patch kernels load them as
                            packed pairs of BF16 components (half the bytes
                            and load instructions of FP32 G); launch shapes
                            that stage G in shared memory read an FP32 copy
                            of the same rounded values, so every shape gives
                            the same bits                                    */
  int dense_local;       /* tabulated local solves: the local solve of a patch
                            (N_MG V-cycles from zero with fixed intervals) is
                            a fixed linear map, tabulated at set-up by
                            applying it to unit vectors; a sweep then does
                            one dense matrix-vector product per patch instead
                            of the V-cycles.  1 (default): pmg_setup times it
                            against the matrix-free V-cycles on every level
                            whose table takes at most 2 GiB and keeps the
                            faster; 2: on every such level; 0: never.  The
                            result equals the V-cycles' up to rounding;
                            pmg_local_vcycle always runs the V-cycles       */
  int level_rule;        /* p-levels of the local V-cycle (Section 3.1):
                            0 (default): p, p/2, ..., 1; 1: the paper's
                            nested sequence 1, 3, 7, 15, ... below p with p
                            on top (p = 8: 8, 7, 3, 1; they differ for
                            p = 4, 5 and 8).  Rule 1 runs one launch shape
                            (no autotuned shapes, no persistent sweeps);
                            structured meshes only                          */
} pmg_options;
enum { PMG_KAPPA_ARITHMETIC = 0, PMG_KAPPA_GEOMETRIC = 1, PMG_KAPPA_HARMONIC = 2 };

typedef struct pmg_ctx pmg_ctx;

/* Fill `opt` with the defaults: Chebyshev degree 3, N_MG = 1, Lanczos bounds
 * with 16 steps, safety 1.1, ratio 10, omega 0.5, seed 0, FP64, autotune on,
 * MLP safety 1.2, persistent sweeps where faster, wait budget 2^31 cycles. */
void pmg_default_options(pmg_options* opt);

/* Create a context on CUDA device `device`; `opt` may be NULL (defaults).
 * On success *out owns the context; release it with pmg_destroy. */
int pmg_create(int device, const pmg_options* opt, pmg_ctx** out);
int pmg_destroy(pmg_ctx* ctx);
const char* pmg_last_error(const pmg_ctx* ctx);

/* ---- mesh and coefficient (Section 2: mesh hierarchy M_1 c ... c M_L) ---
 * Upload the finest mesh of a structured hierarchy: `dim` in {2,3}; N cells
 * per direction on the finest level; degree p in 1..8; n_levels >= 1 h-levels
 * with N_l = N / 2^(n_levels-1-l) cells per direction (N must be divisible by
 * 2^(n_levels-1)).  coords: ((N+1)^dim x dim) FP64 vertex coordinates in
 * lexicographic vertex order (x fastest); vertices of coarser levels are the
 * finest-level vertices with even indices.  kappa: N^dim FP64 cell values of
 * the coefficient (paper: mu); a coarse cell takes the mean of its
 * 2^dim children (options.coarse_kappa: arithmetic, geometric or harmonic).
 * Boundary vertices must lie on the boundary of the unit
 * square/cube for the Dirichlet data to mean what it says (not checked). */
int pmg_mesh_structured(pmg_ctx* ctx, int dim, int N, int p, int n_levels,
                        const double* coords, const double* kappa);

/* ---- unstructured meshes ---------------------------------------------------
 * Quadrilateral (dim 2) or hexahedral (dim 3) meshes of any topology, the
 * setting of Section 2 without the Cartesian structure (the paper's vertex
 * patches on general meshes and its simplicial patches of 3 quadrilaterals /
 * 4 hexahedra, Section 3.2).  One mesh level: the patch smoother and the local
 * p-multigrid of Sections 2.1 and 3 act on degree p.  Mesh levels are
 * uploaded coarsest first (level 0, 1, ...); level l > 0 is the uniform
 * refinement of level l - 1: parent_cell[c] is the level-(l-1) cell that fine
 * cell c subdivides, child_index[c] its position (bit a: the upper half along
 * reference axis a), and corner k of the child lies at the parent's reference
 * point (bits(child) + bits(k)) / 2 (its frame is the parent's); every parent
 * has its 2^dim children.  The preconditioner of pmg_solve_cg /
 * pmg_solve_gmres / pmg_gmg_vcycle is the V-cycle over the levels (Section 2):
 * a patch sweep, the residual restricted by the transposed h-embedding
 * (per fine cell, through the reference cells), the next coarser level, the
 * correction prolongated, a reverse sweep; on level 0 the coarse space is the
 * Q1 space of that mesh (operator re-evaluated with the 2-point Gauss rule,
 * dense Cholesky, at most 16384 free vertices).
 *
 * coords: n_vertices x dim doubles.  cell_vertices: n_cells x 2^dim vertex
 * ids, lexicographic corner order (corner c at the reference point whose k-th
 * coordinate is bit k of c), every cell positively oriented.
 * vertex_on_boundary: n_vertices flags or NULL (derived: the vertices of the
 * facets that belong to one cell).  parent_cell and child_index are NULL on
 * level 0 and given on finer levels (PMG_ERR_ARG otherwise).  Host arrays are
 * copied.  Call pmg_set_degree before pmg_setup; kappa by pmg_coeff_upload
 * per level (default: 1 on the finest level, the mean of the children on a
 * coarser one).  DoF numbering (pmg_get_dof_map, finest level): vertices by id; edges sorted
 * by (smaller id, larger id), q - 1 nodes each from the smaller-id end; faces
 * sorted by their sorted vertex ids, (q - 1)^2 nodes in the frame of the
 * face's smallest-id corner (first axis toward its smaller-id face neighbour,
 * fastest); cell interiors by cell, x fastest.  Patches: the interior vertices
 * in increasing id, each with its cells; colours: greedy in decreasing
 * (splitmix64(id ^ seed), id), the smallest colour not used by a patch that
 * shares a cell.  Chebyshev intervals: PMG_BOUNDS_LANCZOS (FP64 operator in
 * both precisions; start-vector counter (vertex id << 20) | (q << 16) | i),
 * FIXED or USER (pmg_set_bounds); the smoother Chebyshev or Jacobi;
 * multiplicative sweeps.
 * Local vectors of pmg_local_vcycle: one row of pmg_local_size values per patch
 * (its interior DoFs in increasing global id, zero padded). */
int pmg_mesh_upload(pmg_ctx* ctx, int level, int dim, int64_t n_vertices, const double* coords,
                    int64_t n_cells, const int64_t* cell_vertices, const uint8_t* vertex_on_boundary,
                    const int64_t* parent_cell, const uint8_t* child_index);
/* Polynomial degree p (1..8) of an unstructured mesh (p-levels p, p/2, ..., 1). */
int pmg_set_degree(pmg_ctx* ctx, int p);
/* [n_cells][(q+1)^dim] global DoF ids of every cell's nodes at p-level index k
 * (local order lexicographic, x fastest); unstructured meshes, after set-up. */
int pmg_get_dof_map(pmg_ctx* ctx, int k, int32_t* out_host);
/* Row length of the local vectors of pmg_local_vcycle on a level: (2p-1)^d on
 * structured meshes, the largest patch interior on unstructured ones. */
int pmg_local_size(const pmg_ctx* ctx, int level, int64_t* n);

/* Coefficient of every cell of mesh level `level` (0 = coarsest; host array
 * of N_l^d doubles, cell index lexicographic with x fastest, copied), in
 * place of the one the set-up derives from the finer level with the
 * `coarse_kappa` rule (Section 2 defines kappa on the domain only; a coarse
 * level's coefficient is the user's choice).  On the finest level it
 * replaces the mesh's coefficient; a coarser level not uploaded is derived
 * from the level above it, uploaded or not.  Call after the mesh upload and
 * before pmg_setup; PMG_ERR_ARG otherwise or if a value is not positive and
 * finite. */
int pmg_coeff_upload(pmg_ctx* ctx, int level, const double* kappa_host);

/* Build everything the solver needs (geometry tensors on every level and
 * p-level, level diagonals, patch and colour lists, Chebyshev bounds, coarse
 * Cholesky factor).  The coarsest level may have at most 16384 free DoFs
 * (dense coarse solve), else PMG_ERR_UNSUPPORTED.  Returns PMG_ERR_DEGENERATE if a cell has det J <= 0 at
 * any Gauss point or vertex (Section 3.2 excludes such degenerate cells).
 * Synchronises the device. */
int pmg_setup(pmg_ctx* ctx);

/* DoF counts of mesh level l: total (p N_l + 1)^d and free (p N_l - 1)^d. */
int pmg_num_dofs(const pmg_ctx* ctx, int level, int64_t* total, int64_t* n_free);
/* Number of vertex patches (interior vertices, (N_l - 1)^d) and colours (2^d). */
int pmg_num_patches(const pmg_ctx* ctx, int level, int64_t* n_patches, int* n_colours);
/* Levels of the local p-hierarchy (Section 3.1): writes up to 8 degrees,
 * p, floor(p/2), ..., 1, into degrees[], their count into *n. */
int pmg_p_levels(const pmg_ctx* ctx, int* degrees, int* n);

/* ---- operator (eq. matrix) --------------------------------------------
 * Au = A_l u on mesh level l at degree p; rows of Dirichlet DoFs are 0.
 * Deterministic (cells are processed in 2^d parity classes). */
int pmg_apply(pmg_ctx* ctx, int level, const double* u_dev, double* Au_dev, void* stream);

/* ---- patch smoother (Section 2.1, Algorithm 1) --------------------------
 * Multiplicative vertex-patch sweep on mesh level l: for every colour c in
 * 0..2^d-1 (reversed if `reverse`), every patch j of colour c computes
 *   Gather    u_j = Pi_j-bar u, b_j = Pi_j b            (eq. gather)
 *   Evaluate  r_j = b_j - Pi_j A_j-bar u_j             (eq. main:4)
 *   Solve     d_j = N_MG local p-MG V-cycles on r_j    (eq. main:5, Alg. 2)
 *   Scatter   u += Pi_j^T d_j                          (eq. scatter)
 * Patches of one colour share no cell, so they run concurrently and the
 * result equals the sequential sweep in colour-major order.  u_dev is
 * updated in place; n_sweeps sweeps are applied.  Asynchronous on `stream`,
 * except on a level swept by the persistent launch (pmg_level_persistent):
 * there the call waits for the stream and returns PMG_ERR_TIMEOUT if a grid
 * barrier ran out of its budget. */
int pmg_patch_smooth(pmg_ctx* ctx, int level, const double* b_dev, double* u_dev,
                     int n_sweeps, int reverse, void* stream);
/* One colour of the sweep above (colour in 0..2^d-1). */
int pmg_patch_smooth_colour(pmg_ctx* ctx, int level, int colour, const double* b_dev,
                            double* u_dev, void* stream);

/* ---- local solver (Section 3, Algorithm 2) ------------------------------
 * For n patches of mesh level l given by patch_ids_dev (device int64, patch
 * numbering lexicographic over interior vertices, x fastest), apply n_cycles
 * V-cycles (the first from d = 0) to the local right-hand sides r_dev and
 * write the corrections d_dev.  r_dev and d_dev are device FP64 arrays of
 * n x (2p-1)^d values, patch-interior DoFs in lexicographic order (x fastest)
 * (unstructured meshes: n x pmg_local_size values, each row the patch's
 * interior DoFs in increasing global id, zero padded).  An id outside
 * 0 .. n_patches - 1 gives a row of zeros (the call stays asynchronous). */
int pmg_local_vcycle(pmg_ctx* ctx, int level, int64_t n, const int64_t* patch_ids_dev,
                     const double* r_dev, double* d_dev, int n_cycles, void* stream);

/* ---- Chebyshev intervals -----------------------------------------------
 * Per (mesh level, p-level q > 1, patch) interval [lo, hi] for D^-1 A_{j,q}.
 * pmg_get_bounds writes n_patches x n_plevels pairs (lo, hi) as FP64, p-level
 * index fastest (index 0 = degree p), into host memory; entries of q = 1 are 0.
 * pmg_set_bounds uploads such an array (used with PMG_BOUNDS_USER, or to
 * override).  pmg_compute_bounds recomputes them with the configured source.
 * Lanczos: k steps on D^-1/2 A D^-1/2 with full reorthogonalisation,
 * start vector 1 + (u - 1/2), u from counter-based SplitMix64. */
int pmg_get_bounds(pmg_ctx* ctx, int level, double* lohi_host);
int pmg_set_bounds(pmg_ctx* ctx, int level, const double* lohi_host);
int pmg_compute_bounds(pmg_ctx* ctx, int source);
/* Raw Lanczos extreme Ritz values (theta_min, theta_max) per (patch, p-level),
 * same layout as pmg_get_bounds. */
int pmg_get_ritz(pmg_ctx* ctx, int level, double* tminmax_host);

/* ---- global solver (Section 2; GMG preconditioned CG) ------------------
 * One GMG V-cycle on the finest level: x = B b with one forward patch sweep
 * before and one reversed sweep after the coarse-grid correction, dense
 * Cholesky on level 0.  Symmetric, so it preconditions CG. */
int pmg_gmg_vcycle(pmg_ctx* ctx, const double* b_dev, double* x_dev, void* stream);

/* Preconditioned CG on the finest level from u = 0 until
 * ||r_k||_2 <= rtol ||b||_2 or maxit iterations.  Writes *iters and *relres
 * (host).  The solve runs on the context's own stream, ordered after the work
 * already queued on `stream` (an event wait: `stream` itself is not
 * synchronised); the host reads one 8-byte residual per iteration, and the
 * call returns when the solve, including the write of u_dev, has finished.
 * Returns PMG_ERR_NOT_CONVERGED at maxit, PMG_ERR_NUMERIC on NaN/Inf. */
int pmg_solve_cg(pmg_ctx* ctx, const double* b_dev, double* u_dev, double rtol, int maxit,
                 int* iters, double* relres, void* stream);

/* Restarted GMRES(restart) on the finest level from u = 0 with the GMG V-cycle
 * as preconditioner M (the paper's outer solver, Section 4), modified
 * Gram-Schmidt Arnoldi, Givens rotations.  left = 0: right preconditioning,
 * u = M y, stops when ||b - A u||_2 <= rtol ||b||_2; left = 1: the Krylov space
 * of M A, stops when ||M (b - A u)||_2 <= rtol ||M b||_2.  Runs on the
 * context's own stream after the work queued on `stream` (event wait), and
 * synchronises that internal stream once per inner product (the Hessenberg
 * least-squares problem lives on the host); returns when finished.
 * Returns PMG_ERR_NOT_CONVERGED at maxit. */
int pmg_solve_gmres(pmg_ctx* ctx, const double* b_dev, double* u_dev, double rtol, int maxit,
                    int restart, int left, int* iters, double* relres, void* stream);

/* Several independent problems solved together (no counterpart in the paper;
 * the batched-solve layer of this library).  Each context is set up on its own
 * mesh, degree and options (degrees and sizes may differ); problem k solves
 * A_k u_k = b_k by the GMG-preconditioned CG of pmg_solve_cg, with the same
 * stopping rule and the same iterates as a call of pmg_solve_cg on that context
 * alone.  One host thread interleaves the problems: every iteration of every
 * unfinished problem is launched (a captured CUDA graph on the context's own
 * stream) before any is waited for, so the problems run concurrently on the
 * GPU and small ones fill the SMs that large ones leave idle.
 * ctxs[n_problems]: distinct contexts after pmg_setup, on the same device.
 * b[k], u[k]: device vectors of context k (layout of pmg_solve_cg).
 * iters, relres, status: host arrays of n_problems entries, or NULL; status[k]
 * is problem k's code.  Returns PMG_OK if every problem converged, else the
 * first failing problem's code (messages in each context's pmg_last_error).
 * Synchronises; every problem's work is finished on return. */
int pmg_batch_solve_cg(pmg_ctx* const* ctxs, int n_problems, const double* const* b, double* const* u,
                       double rtol, int maxit, int* iters, double* relres, int* status);

/* Same solve with host vectors: copies b in, solves, copies u out. */
int pmg_solve_cg_host(pmg_ctx* ctx, const double* b_host, double* u_host, double rtol,
                      int maxit, int* iters, double* relres, void* stream);

/* Load vector b_i = int f phi_i on the finest level for the manufactured
 * solution u = prod_k sin(pi x_k) (f = d pi^2 u), Gauss rule with p+2 points
 * per direction; Dirichlet entries 0. */
int pmg_rhs_manufactured(pmg_ctx* ctx, double* b_dev, void* stream);

/* ---- integer structures (bit-exact tests) -------------------------------
 * Colour of every patch of level l (uint8, patch order as above). */
int pmg_get_colours(const pmg_ctx* ctx, int level, uint8_t* colours_host);
/* Patch map of level l: for each patch its 2^d cells (int64, cell order
 * lexicographic inside the patch, x fastest) followed by the global DoF id of
 * its closure origin (lowest corner node). Writes n_patches x (2^d + 1).
 * Unstructured meshes: n_patches x (1 + PMG_UMAXC): the patch's vertex id,
 * then its cells in increasing id, -1 padded. */
int pmg_get_patch_map(const pmg_ctx* ctx, int level, int64_t* map_host);

/* Inverse level diagonal 1/diag(A_{l,q}) of mesh level l at p-level index k
 * (degree p >> k), device FP64 output of (q N_l + 1)^d entries (Dirichlet 0). */
int pmg_get_inv_diag(pmg_ctx* ctx, int level, int k, double* out_dev, void* stream);

/* Algorithmic flop count of one forward patch sweep on mesh level l (the
 * operator applies of Evaluate, smoothing and residuals, by the
 * sum-factorisation count 4d 1D sweeps + the quadrature-point product per
 * cell, plus the p-transfers). */
double pmg_sweep_flops(const pmg_ctx* ctx, int level);

/* Launch shape chosen for the patch-sweep kernel: variant index, threads per
 * CTA, patches per CTA, and the set-up timings of the candidate variants
 * (ms for one colour of the finest level, ms_per_variant[PMG_NUM_VARIANTS], -1 where a
 * variant does not exist or was not timed).  Any output may be NULL.
 * Every variant computes bit-identical results. */
int pmg_tuning(const pmg_ctx* ctx, int* variant, int* threads, int* patches_per_cta,
               float* ms_per_variant);
/* Launch shape used on mesh level `level` (the set-up autotuner times every
 * variant on one colour of every level: large launches favour occupancy, the
 * small launches of coarse levels the latency of one patch) and its timings
 * (ms_per_variant[PMG_NUM_VARIANTS], -1 where not timed).  Either output may be NULL. */
int pmg_tuning_level(const pmg_ctx* ctx, int level, int* variant, float* ms_per_variant);
/* Persistent sweeps of mesh level `level`: *on = 1 if its sweeps run as one
 * cooperative launch; the set-up's timings of one full sweep with per-colour
 * launches and with the persistent launch (ms; -1 if not timed). */
int pmg_level_persistent(const pmg_ctx* ctx, int level, int* on, float* ms_per_colour, float* ms_persistent);
/* Tabulated local solves on mesh level `level`: *on = 1 if its sweeps use
 * them; the set-up's timings of one full sweep with the matrix-free V-cycles
 * and with the tables (ms; -1 if not timed). */
int pmg_level_dense_local(const pmg_ctx* ctx, int level, int* on, float* ms_matrix_free, float* ms_tabulated);

/* ---- learned Chebyshev intervals ------------------------------------------
 * No counterpart in the paper (its smoother is damped Jacobi).  A small MLP
 * predicts (log theta_max, log theta_min) of the Lanczos run of a patch from
 * 16 features of its cells' geometry and coefficient; Lanczos stays the
 * reference estimate.  Network 16 -> 64 -> 64 -> 2 with ReLU on standardised inputs and
 * targets; PMG_MLP_NPARAM parameters (W1 64x16 row-major, b1, W2 64x64, b2,
 * W3 2x64, b3) and PMG_MLP_NNORM normalisation floats (mean and std of the 16
 * features, then mean and std of the 2 targets).  Training is FP32 (Adam),
 * inference BF16 with FP32 accumulation.  Loss per sample: sum_o w_o (y_o -
 * t_o)^2 / 2, w_0 = asym when theta_max is underestimated, averaged. */
#define PMG_MLP_NPARAM 5378
#define PMG_MLP_NNORM 36

typedef struct pmg_train_opts {
  int epochs;
  int batch;
  float lr, beta1, beta2, eps;
  float asym;            /* weight of underestimated theta_max               */
  uint64_t seed;         /* shuffling                                        */
} pmg_train_opts;
void pmg_default_train_options(pmg_train_opts* opt);

/* Features of every patch of mesh level l at p-level index k: device float
 * array of n_patches x 16 (layout and definitions in the implementation). */
int pmg_features(pmg_ctx* ctx, int level, int k, float* X_dev, void* stream);
/* Loss and gradient of the loss on n samples (X: n x 16 raw features, T:
 * n x 2 raw targets; all device pointers; one batch of all n). */
int pmg_mlp_grad(int device, const float* params_dev, const float* norm_dev, const float* X_dev,
                 const float* T_dev, int n, float asym, float* loss_dev, float* grad_dev, void* stream);
/* Train in place (params_dev: initial -> trained) on n samples; writes the
 * mean batch loss of every epoch to loss_hist_host (may be NULL). */
int pmg_mlp_train(int device, float* params_dev, const float* norm_dev, const float* X_dev,
                  const float* T_dev, int64_t n, const pmg_train_opts* opt, float* loss_hist_host);
/* Y (n x 2 device) = predicted (log theta_max, log theta_min); bf16 != 0:
 * BF16 weights, biases, inputs and hidden activations, the three layers as
 * tensor-core products (warp-level m16n8k16) with FP32 accumulation; bf16 = 0:
 * FP32 throughout.  Any n >= 0 (a last tile of fewer than 16 samples is
 * padded internally, nothing is written past Y_dev[2n - 1]). */
int pmg_mlp_predict(int device, const float* params_dev, const float* norm_dev, const float* X_dev,
                    int64_t n, int bf16, float* Y_dev, void* stream);
/* Install a trained network (host arrays) for PMG_BOUNDS_MLP. */
int pmg_set_mlp(pmg_ctx* ctx, const float* params_host, const float* norm_host);
/* Initial parameters (host array of PMG_MLP_NPARAM floats): weights uniform in
 * +-sqrt(6 / fan_in) from the SplitMix64 counter stream of `seed`, biases 0. */
void pmg_mlp_init(uint64_t seed, float* params_host);
/* Training targets of mesh level `level`, p-level index k (degree > 1): the
 * context's Lanczos estimates as T_dev (n_patches x 2 device floats) =
 * (log theta_max, log theta_min).  Asynchronous on `stream`. */
int pmg_mlp_targets(pmg_ctx* ctx, int level, int k, float* T_dev, void* stream);
/* Normalisation of a training set (X_dev n x 16 features, T_dev n x 2 targets,
 * device): the PMG_MLP_NNORM floats (column means, then population standard
 * deviations + 1e-6, of X and then of T) to norm_host.  Synchronises. */
int pmg_mlp_norm(int device, const float* X_dev, const float* T_dev, int64_t n, float* norm_host);
/* Write the installed network (parameters and normalisation) to a file, or
 * read one written by pmg_mlp_save and install it (as pmg_set_mlp).  File:
 * 8-byte magic, two uint32 counts, the floats; PMG_ERR_ARG on any mismatch. */
int pmg_mlp_save(pmg_ctx* ctx, const char* path);
int pmg_mlp_load(pmg_ctx* ctx, const char* path);

/* ---- measurement ----------------------------------------------------------
 * Number of kernels this context has launched so far (kernel nodes of a CUDA
 * graph count once per graph launch). */
int pmg_launch_count(const pmg_ctx* ctx, int64_t* n);

/* FMA-pipe peak microbenchmark on the context's device: a grid of
 * independent FMA chains in FP64 (precision = PMG_PREC_FP64) or FP32
 * (PMG_PREC_MIXED), sized to fill every SM; writes the achieved FLOP/s
 * (2 flops per FMA).  Synchronises the device. */
int pmg_fma_peak(pmg_ctx* ctx, int precision, double* flops_per_s);

/* ---- allocation-free bounds ----------------------------------------------
 * No counterpart in the paper: an engineering entry point for callers that
 * must not allocate device memory at this point (for instance inside a
 * framework that owns the device memory through its own allocator, or in a
 * solver that refreshes its Chebyshev intervals mid-run and must not stall on
 * cudaMalloc/cudaFree, which synchronise the device).
 *
 * Computes the same Lanczos estimates as pmg_compute_bounds (the context's
 * Lanczos options) for patches first_patch .. first_patch + n_patches - 1 of
 * mesh level `level` at p-level index k (degree p >> k, must be > 1) and
 * writes n_patches x (theta_min, theta_max) to ritz_dev and n_patches x
 * (lo, hi) to bounds_dev: caller-owned device FP64 arrays of at least
 * 2 * n_patches values each, on the context's device.  The context's own
 * intervals are not changed.  Asynchronous on `stream`.  The operator is
 * applied in FP64, except at degrees whose FP64 working set exceeds shared
 * memory (3D q >= 7), where, like pmg_compute_bounds, it is applied in FP32
 * with FP64 Lanczos vectors and the intervals are rounded to FP32; that needs
 * the context's FP32 geometry (always present in mixed precision; in FP64
 * contexts made by pmg_compute_bounds with Lanczos bounds), else
 * PMG_ERR_UNSUPPORTED.
 *
 * Allocates no device memory: the Lanczos basis lives in one fixed 16 MiB
 * device array inside the library (held by every GPU that loads it until the
 * process exits).  Limit: n_patches * lanczos_steps * (2q-1)^d <= 2^21
 * doubles, else PMG_ERR_ARG (split the range).  The first call on a device
 * also uploads this entry point's tables and looks up the array's device
 * address; make that first call before any stream capture.  All calls share
 * the array: calls whose kernels overlap on the GPU race, so serialise them.
 * The caller's current device is restored before the call returns. */
int pmg_lanczos_bounds_noalloc(pmg_ctx* ctx, int level, int k, int64_t first_patch,
                               int64_t n_patches, double* ritz_dev, double* bounds_dev,
                               void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PMG_H */
