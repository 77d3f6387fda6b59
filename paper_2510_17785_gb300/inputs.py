"""Seeded synthetic inputs for the patch-smoother workloads.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests.  It holds none of the method's arithmetic: it only produces
vertex coordinates of structured hexahedral/quadrilateral meshes of the unit
square/cube (with seeded vertex perturbations), per-cell coefficients and
right-hand-side vectors in the global lexicographic DoF layout.

Layouts (all lexicographic, x fastest):
  * vertices: ``(N+1)**dim`` rows of ``dim`` coordinates;
  * cells:    ``N**dim`` entries;
  * DoFs:     ``(p*N+1)**dim`` entries (Dirichlet DoFs included, set to 0).

The workloads follow the paper's test problems (Section 4: unit square/cube
refined uniformly, interior vertices displaced; Section 3.3: coefficient
jumps) with the sizes of the five benchmark configurations.  One
``numpy.random.default_rng(seed)`` stream draws, in this order: vertex
perturbation, coefficient, right-hand side.  Vertices of cells with a
non-positive corner volume are redrawn from a side stream seeded by
(seed, attempt) until every corner is positive.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic problem: mesh size, degree, perturbation, coefficient, RHS."""
    name: str
    dim: int
    N: int                 # cells per direction on the finest mesh
    p: int                 # polynomial degree
    perturb: float         # vertex displacement as a fraction of h = 1/N
    law: str               # "uniform": each component U(-perturb*h, perturb*h);
                           # "sphere": length perturb*h, direction uniform on S^{d-1};
                           # "kershaw": Kershaw-type mesh with parameter eps = perturb
                           # (three blended segments); "kershaw6": the six-layer
                           # Kershaw mesh, eps = perturb
    kappa: tuple           # ("const", value) or ("loguniform", log10_lo, log10_hi)
    rhs: str               # "uniform" (U[-1,1] on free DoFs) or "manufactured"
    seed: int
    coarse_N: int = 2      # cells per direction on the coarsest h-level

    @property
    def n_dofs(self) -> int:
        return (self.p * self.N + 1) ** self.dim

    @property
    def n_free(self) -> int:
        return (self.p * self.N - 1) ** self.dim

    @property
    def n_patches(self) -> int:
        return (self.N - 1) ** self.dim

    def with_(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


# The five benchmark workloads (seed 1000 + index).
C1 = Workload("c1_2d_q4_n16", 2, 16, 4, 0.0, "uniform", ("const", 1.0), "uniform", 1001)
C2 = Workload("c2_3d_q4_n32_perturbed", 3, 32, 4, 0.25, "uniform", ("const", 1.0),
              "manufactured", 1002, coarse_N=2)
C3 = Workload("c3_3d_q7_n48_varcoef", 3, 48, 7, 0.25, "uniform", ("loguniform", -3.0, 3.0),
              "uniform", 1003, coarse_N=3)
C5 = Workload("c5_3d_q8_n64_varcoef", 3, 64, 8, 0.25, "uniform", ("loguniform", -2.0, 2.0),
              "uniform", 1005, coarse_N=2)
WORKLOADS = {w.name: w for w in (C1, C2, C3, C5)}


def grid_vertices(dim: int, N: int) -> np.ndarray:
    """Unperturbed vertices of the N^dim grid on the unit square/cube."""
    t = np.arange(N + 1, dtype=np.float64) / N
    axes = np.meshgrid(*([t] * dim), indexing="ij")  # axes[k] varies along index k
    # lexicographic with x fastest: reverse the 'ij' order
    cols = [axes[dim - 1 - k].reshape(-1) for k in range(dim)]
    # axes[0] is the slowest index; for x fastest, x must come from the last axis
    return np.stack(cols, axis=1).copy()


def interior_vertex_mask(dim: int, N: int) -> np.ndarray:
    idx = np.indices((N + 1,) * dim).reshape(dim, -1)  # idx[0] slowest
    inner = np.all((idx > 0) & (idx < N), axis=0)
    return inner


def perturbation(rng: np.random.Generator, dim: int, N: int, frac: float, law: str) -> np.ndarray:
    """Displacements of all vertices (zero on the boundary)."""
    nv = (N + 1) ** dim
    h = 1.0 / N
    if law == "uniform":
        disp = rng.uniform(-frac * h, frac * h, size=(nv, dim))
    elif law == "sphere":
        g = rng.standard_normal(size=(nv, dim))
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        disp = frac * h * g
    else:
        raise ValueError(law)
    disp[~interior_vertex_mask(dim, N)] = 0.0
    return disp


def corner_volumes(x: np.ndarray, dim: int, N: int) -> np.ndarray:
    """Signed corner volumes (N^dim cells x 2^dim corners): at each corner the
    determinant of the dim cell edges leaving it along +x, +y(, +z) in the
    cell's own index directions.  All positive <=> no inverted or non-convex
    corner (the paper excludes such degenerate cells, Section 3.2)."""
    X = x.reshape(*([N + 1] * dim), dim)                 # array axes [z][y][x] (or [y][x])
    out = []
    for v in range(2 ** dim):
        cols = []
        for k in range(dim):
            lo = [((v >> a) & 1) if a != k else 0 for a in range(dim)]
            hi = [((v >> a) & 1) if a != k else 1 for a in range(dim)]
            sl_lo = tuple(slice(lo[dim - 1 - a], lo[dim - 1 - a] + N) for a in range(dim))
            sl_hi = tuple(slice(hi[dim - 1 - a], hi[dim - 1 - a] + N) for a in range(dim))
            cols.append(X[sl_hi] - X[sl_lo])
        out.append(np.linalg.det(np.stack(cols, axis=-1)).reshape(-1))
    return np.stack(out, axis=1)


def valid_perturbation(rng, dim: int, N: int, frac: float, law: str, seed: int, max_attempts: int = 64):
    """Perturbed vertices with every corner volume positive: vertices of cells
    with a non-positive corner are redrawn (from a separate stream seeded by
    (seed, attempt), so the main stream is consumed the same way every time)."""
    x = grid_vertices(dim, N)
    disp = perturbation(rng, dim, N, frac, law)
    inner = interior_vertex_mask(dim, N)
    for attempt in range(1, max_attempts + 1):
        bad = corner_volumes(x + disp, dim, N).min(axis=1) <= 0.0
        if not bad.any():
            return x + disp
        cells = np.nonzero(bad)[0]
        verts = set()
        for c in cells:
            ci = [(c // N ** a) % N for a in range(dim)]
            for v in range(2 ** dim):
                verts.add(sum((ci[a] + ((v >> a) & 1)) * (N + 1) ** a for a in range(dim)))
        verts = np.array(sorted(v for v in verts if inner[v]), dtype=np.int64)
        sub = np.random.default_rng([seed, attempt])
        fresh = perturbation(sub, dim, N, frac, law)
        disp[verts] = fresh[verts]
    raise RuntimeError("could not draw a valid perturbed mesh")


def kershaw_squeeze(t: np.ndarray, eps: float) -> np.ndarray:
    """A piecewise-linear bijection of [0, 1] with a kink at 1/2: the left half
    is stretched onto [0, 1 - eps/2], the right half squeezed onto
    [1 - eps/2, 1] (eps in (0, 1]; eps = 1 is the identity)."""
    return np.where(t <= 0.5, (2.0 - eps) * t, 1.0 - eps * (1.0 - t))


def kershaw_vertices(dim: int, N: int, eps: float = 0.3) -> np.ndarray:
    """Vertices of a Kershaw-type mesh of the unit square/cube (Kershaw 1981,
    "Differencing of the diffusion equation in Lagrangian hydrodynamic codes":
    a logically Cartesian grid whose mesh lines zig-zag).  x is kept; y is
    mapped by a blend, linear in x, between the left-fine map
    l(t) = 1 - s(1 - t) and the right-fine map r(t) = s(t) (s =
    kershaw_squeeze): l -> r on x in [0, 1/3], r -> l on [1/3, 2/3] and
    l -> r on [2/3, 1]; in 3D z is mapped the same way in the opposite phase.
    Every map is monotone in its own coordinate and the x-faces stay planes
    x = const, so every cell has det J > 0.  N must be a multiple of 3 (the
    kinks of the blend lie on mesh lines)."""
    if N % 3 != 0:
        raise ValueError("a Kershaw-type mesh needs N divisible by 3")
    x = grid_vertices(dim, N)
    s = lambda t: kershaw_squeeze(t, eps)
    left = lambda t: 1.0 - s(1.0 - t)
    seg = np.minimum((x[:, 0] * 3.0).astype(int), 2)        # x segment 0, 1, 2
    lam = x[:, 0] * 3.0 - seg                                 # position inside the segment
    lam = np.where(seg == 1, 1.0 - lam, lam)                  # r -> l on the middle segment
    out = x.copy()
    out[:, 1] = (1.0 - lam) * left(x[:, 1]) + lam * s(x[:, 1])
    if dim == 3:
        out[:, 2] = lam * left(x[:, 2]) + (1.0 - lam) * s(x[:, 2])
    return out


def kershaw6_vertices(dim: int, N: int, eps: float = 0.3) -> np.ndarray:
    """Vertices of the six-layer Kershaw mesh of the unit square/cube (the
    construction of the high-order benchmark literature, e.g. Fischer et al.,
    "Scalability of high-performance PDE solvers", 2020): x is kept and cut
    into six layers of width 1/6; y (and z, in the same phase) is mapped by
    the left-fine profile l(t) = 1 - s(1 - t) on layer 0 and the right-fine
    profile r(t) = s(t) on layer 5 (s = kershaw_squeeze), by a blend linear in
    x from l to r across layer 1 and across layer 4, and from r back to l
    across layers 2 and 3 together.  N must be a multiple of 6 (layer
    boundaries on mesh lines)."""
    if N % 6 != 0:
        raise ValueError("the six-layer Kershaw mesh needs N divisible by 6")
    x = grid_vertices(dim, N)
    s = lambda t: kershaw_squeeze(t, eps)
    left = lambda t: 1.0 - s(1.0 - t)
    layer = np.minimum((x[:, 0] * 6.0 + 1e-12).astype(int), 5)
    t = x[:, 0] * 6.0 - layer                                  # position inside the layer
    lam = np.select([layer == 0, layer == 1, layer == 2, layer == 3, layer == 4],
                    [np.zeros_like(t), t, 1.0 - 0.5 * t, 0.5 - 0.5 * t, t], default=np.ones_like(t))
    out = x.copy()
    for k in range(1, dim):
        out[:, k] = (1.0 - lam) * left(x[:, k]) + lam * s(x[:, k])
    return out


def kappa_cells(rng: np.random.Generator, dim: int, N: int, spec: tuple) -> np.ndarray:
    nc = N ** dim
    if spec[0] == "const":
        return np.full(nc, float(spec[1]))
    if spec[0] == "loguniform":
        return 10.0 ** rng.uniform(spec[1], spec[2], size=nc)
    raise ValueError(spec)


def free_dof_mask(dim: int, p: int, N: int) -> np.ndarray:
    M = p * N + 1
    idx = np.indices((M,) * dim).reshape(dim, -1)
    return np.all((idx > 0) & (idx < M - 1), axis=0)


def rhs_uniform(rng: np.random.Generator, dim: int, p: int, N: int) -> np.ndarray:
    b = rng.uniform(-1.0, 1.0, size=(p * N + 1) ** dim)
    b[~free_dof_mask(dim, p, N)] = 0.0
    return b


@dataclasses.dataclass
class Problem:
    workload: Workload
    coords: np.ndarray          # ((N+1)^d, d) float64
    kappa: np.ndarray           # (N^d,) float64
    rhs: Optional[np.ndarray]   # ((pN+1)^d,) float64, or None for "manufactured"


def make_problem(w: Workload) -> Problem:
    rng = np.random.default_rng(w.seed)
    x = grid_vertices(w.dim, w.N)
    if w.law == "kershaw":
        x = kershaw_vertices(w.dim, w.N, w.perturb)       # perturb holds the Kershaw parameter eps
    elif w.law == "kershaw6":
        x = kershaw6_vertices(w.dim, w.N, w.perturb)
    elif w.perturb > 0.0:
        x = valid_perturbation(rng, w.dim, w.N, w.perturb, w.law, w.seed)
    kap = kappa_cells(rng, w.dim, w.N, w.kappa)
    b = rhs_uniform(rng, w.dim, w.p, w.N) if w.rhs == "uniform" else None
    return Problem(w, x, kap, b)


def random_vector(seed: int, dim: int, p: int, N: int, free_only: bool = True) -> np.ndarray:
    """A seeded U[-1,1] vector in the DoF layout (zero on Dirichlet DoFs)."""
    rng = np.random.default_rng(seed)
    v = rng.uniform(-1.0, 1.0, size=(p * N + 1) ** dim)
    if free_only:
        v[~free_dof_mask(dim, p, N)] = 0.0
    return v


def sample_patches(seed: int, n_patches: int, k: int) -> np.ndarray:
    """k distinct patch ids drawn without replacement (sorted)."""
    rng = np.random.default_rng(seed)
    k = min(k, n_patches)
    return np.sort(rng.choice(n_patches, size=k, replace=False)).astype(np.int64)


def single_patch_vertices(dim: int, delta: float, direction: np.ndarray) -> np.ndarray:
    """Vertices of a 2^d-cell patch of unit cells ([0,2]^d) with the centre vertex moved
    by delta * (patch width 2) along ``direction`` (normalised here)."""
    x = grid_vertices(dim, 2) * 2.0
    c = (3 ** dim) // 2
    u = np.asarray(direction, dtype=np.float64)
    x[c] += delta * 2.0 * u / np.linalg.norm(u)
    return x


# ---------------------------------------------------------------------------
# Unstructured quadrilateral / hexahedral meshes.  A cell is its 2^d vertex
# ids in lexicographic corner order (corner c at the reference point whose
# k-th coordinate is bit k of c).
def triangulated_square(n: int, seed: int, perturb: float = 0.2):
    """A seeded triangulation of the unit square: n x n squares, each cut along
    a random diagonal, interior vertices moved by U(-perturb h, perturb h) per
    component (h = 1/n).  Returns (points, triangles), triangles
    counter-clockwise."""
    rng = np.random.default_rng(seed)
    pts = grid_vertices(2, n)
    inner = interior_vertex_mask(2, n)
    pts[inner] += rng.uniform(-perturb / n, perturb / n, size=(int(inner.sum()), 2))
    tris = []
    for j in range(n):
        for i in range(n):
            a, b = j * (n + 1) + i, j * (n + 1) + i + 1
            c, d = a + (n + 1), b + (n + 1)
            if rng.integers(2):
                tris += [(a, b, d), (a, d, c)]
            else:
                tris += [(a, b, c), (b, d, c)]
    return pts, np.array(tris, dtype=np.int64)


def triangles_to_quads(points: np.ndarray, tris: np.ndarray):
    """Each triangle split into 3 quadrilaterals through its edge midpoints and
    centroid (the centroid has valence 3, an edge midpoint 4 in the interior,
    an original vertex as many as its triangles).  Returns (coords, cells)."""
    pts = [tuple(p) for p in points]
    coords = list(map(np.array, pts))
    mid = {}

    def midpoint(a, b):
        key = (min(a, b), max(a, b))
        if key not in mid:
            mid[key] = len(coords)
            coords.append(0.5 * (points[a] + points[b]))
        return mid[key]

    cells = []
    for a, b, c in tris:
        mab, mbc, mca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
        g = len(coords)
        coords.append((points[a] + points[b] + points[c]) / 3.0)
        for p0, p1, p2, p3 in ((a, mab, g, mca), (b, mbc, g, mab), (c, mca, g, mbc)):
            cells.append((p0, p1, p3, p2))            # cyclic (counter-clockwise) -> lexicographic
    return np.array(coords), np.array(cells, dtype=np.int64)


def extrude(coords2: np.ndarray, quads: np.ndarray, nz: int):
    """Quadrilateral mesh of the unit square x nz layers of [0, 1]: hexahedra
    with the quad's corners at the bottom (bit 2 = 0) and top (bit 2 = 1)."""
    nv2 = len(coords2)
    z = np.arange(nz + 1, dtype=np.float64) / nz
    coords = np.concatenate([np.column_stack([coords2, np.full(nv2, zk)]) for zk in z])
    cells = [tuple(list(q + k * nv2) + list(q + (k + 1) * nv2)) for k in range(nz) for q in quads]
    return coords, np.array(cells, dtype=np.int64)


def cube_tetrahedra(n: int, seed: int, perturb: float = 0.15):
    """n^3 cubes of the unit cube, each cut into 6 tetrahedra around its main
    diagonal (consistent across faces), interior vertices moved by
    U(-perturb h, perturb h) per component.  Returns (points, tets), each tet
    positively oriented."""
    rng = np.random.default_rng(seed)
    pts = grid_vertices(3, n)
    inner = interior_vertex_mask(3, n)
    pts[inner] += rng.uniform(-perturb / n, perturb / n, size=(int(inner.sum()), 3))
    vid = lambda i, j, k: (k * (n + 1) + j) * (n + 1) + i
    tets = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                v = [vid(i + (c & 1), j + ((c >> 1) & 1), k + ((c >> 2) & 1)) for c in range(8)]
                for path in ((1, 3), (1, 5), (2, 3), (2, 6), (4, 5), (4, 6)):
                    t = [v[0], v[path[0]], v[path[1]], v[7]]
                    x = pts[t]
                    if np.linalg.det(np.array([x[1] - x[0], x[2] - x[0], x[3] - x[0]])) < 0:
                        t[1], t[2] = t[2], t[1]
                    tets.append(tuple(t))
    return pts, np.array(tets, dtype=np.int64)


def tetrahedra_to_hexes(points: np.ndarray, tets: np.ndarray):
    """Each tetrahedron split into 4 hexahedra through its edge midpoints, face
    centroids and centroid (valence 4 at the centroid, 6 at an interior face
    centroid).  Returns (coords, cells)."""
    coords = [np.array(p) for p in points]
    cache = {}

    def point(key, fn):
        if key not in cache:
            cache[key] = len(coords)
            coords.append(fn())
        return cache[key]

    cells = []
    for t in tets:
        t = [int(x) for x in t]
        g = len(coords)
        coords.append(points[t].mean(axis=0))
        for ia in range(4):
            a = t[ia]
            o = [t[j] for j in range(4) if j != ia]
            b, c, d = o
            if ia % 2 == 1:                            # keep (b - a, c - a, d - a) right-handed
                b, c = c, b
            m = lambda x, y: point(("e", min(x, y), max(x, y)), lambda: 0.5 * (points[x] + points[y]))
            f = lambda x, y, z: point(("f",) + tuple(sorted((x, y, z))),
                                      lambda: (points[x] + points[y] + points[z]) / 3.0)
            cells.append((a, m(a, b), m(a, c), f(a, b, c), m(a, d), f(a, b, d), f(a, c, d), g))
    return np.array(coords), np.array(cells, dtype=np.int64)


def boundary_vertices(dim: int, nv: int, cells: np.ndarray) -> np.ndarray:
    """Vertices on a facet (edge in 2D, face in 3D) that belongs to one cell only."""
    count = {}
    for cv in cells:
        for a in range(dim):
            for side in (0, 1):
                f = tuple(sorted(int(cv[c]) for c in range(2 ** dim) if ((c >> a) & 1) == side))
                count[f] = count.get(f, 0) + 1
    out = np.zeros(nv, dtype=bool)
    for f, k in count.items():
        if k == 1:
            out[list(f)] = True
    return out


def corner_dets(coords: np.ndarray, cells: np.ndarray) -> np.ndarray:
    """[n_cells][2^d] determinant of the edge vectors at every corner, each edge
    oriented along its reference axis (positive for a cell that is not inverted
    at that corner)."""
    dim = coords.shape[1]
    X = coords[cells]                                   # [nc][2^d][d]
    out = np.zeros(cells.shape)
    for c in range(2 ** dim):
        J = np.stack([(X[:, c ^ (1 << k)] - X[:, c]) * (1.0 if ((c >> k) & 1) == 0 else -1.0)
                      for k in range(dim)], axis=-1)
        out[:, c] = np.linalg.det(J)
    return out


def jacobian_dets(coords: np.ndarray, cells: np.ndarray, xi=(0.0, 0.02, 0.5, 0.98, 1.0)) -> np.ndarray:
    """[n_cells] smallest determinant of the multilinear map's Jacobian over the
    tensor grid xi^d of reference points (corners included)."""
    dim = coords.shape[1]
    pts = np.array(np.meshgrid(*([np.asarray(xi)] * dim), indexing="ij")).reshape(dim, -1).T     # [np][d]
    dN = np.ones((len(pts), 2 ** dim, dim))                                          # d N_c / d xi_a at pts
    for c in range(2 ** dim):
        for a in range(dim):
            for b in range(dim):
                bit = (c >> b) & 1
                dN[:, c, a] *= (1.0 if bit else -1.0) if b == a else (pts[:, b] if bit else 1.0 - pts[:, b])
    out = np.empty(len(cells))
    for s0 in range(0, len(cells), 4096):
        X = coords[cells[s0:s0 + 4096]]                                             # [n][2^d][d]
        J = np.einsum("pca,ncd->npda", dN, X)
        out[s0:s0 + 4096] = np.linalg.det(J).min(axis=1)
    return out


def perturb_unstructured(coords: np.ndarray, cells: np.ndarray, frac: float, rng: np.random.Generator,
                         first_movable: int = 0):
    """Interior vertices moved by frac * h_v in a direction uniform on the
    sphere, h_v the shortest edge at the vertex.  Vertices of a cell whose
    Jacobian determinant comes out non-positive at a corner or at a point of a
    5^d reference grid go back to their place, repeated until none does.
    Vertices with ids below first_movable are not moved."""
    dim = coords.shape[1]
    nv = len(coords)
    bnd = boundary_vertices(dim, nv, cells)
    h = np.full(nv, np.inf)
    for c in range(2 ** dim):
        for k in range(dim):
            if (c >> k) & 1:
                continue
            a, b = cells[:, c], cells[:, c | (1 << k)]
            L = np.linalg.norm(coords[a] - coords[b], axis=1)
            np.minimum.at(h, a, L)
            np.minimum.at(h, b, L)
    g = rng.normal(size=(nv, dim))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    move = frac * h[:, None] * g
    move[bnd] = 0.0
    move[:first_movable] = 0.0                          # vertices below first_movable stay
    out = coords + move
    for _ in range(64):
        bad = (corner_dets(out, cells) <= 0).any(axis=1) | (jacobian_dets(out, cells) <= 0)
        if not bad.any():
            return out, bnd
        vs = np.unique(cells[bad])
        out[vs] = coords[vs]
    raise ValueError("could not perturb the mesh without inverting a cell")


def unstructured_mesh(kind: str, size: int, seed: int, perturb: float = 0.2):
    """Seeded unstructured meshes of the unit square / cube.

    kind "trisplit2d": a size x size triangulated square, each triangle split
    into 3 quadrilaterals (interior valences 3 to 8); "extruded": that mesh
    (size x size) extruded into size // 2 layers (hexahedra, valences 6 to
    16); "tetsplit": a size^3 cube of tetrahedra (6 per cube), each split into
    4 hexahedra (valences 4, 6, 8, 12 and 24).  Interior vertices are then
    moved by ``perturb`` times their shortest edge in a random direction.
    Returns (coords, cells, vertex_on_boundary)."""
    rng = np.random.default_rng(seed)
    if kind in ("trisplit2d", "extruded"):
        P, T = triangulated_square(size, int(rng.integers(1 << 31)))
        X, C = triangles_to_quads(P, T)
        if kind == "extruded":
            X, C = extrude(X, C, max(1, size // 2))
    elif kind == "tetsplit":
        P, T = cube_tetrahedra(size, int(rng.integers(1 << 31)))
        X, C = tetrahedra_to_hexes(P, T)
    else:
        raise ValueError(kind)
    X, bnd = perturb_unstructured(X, C, perturb, rng)
    return X, C, bnd


@dataclasses.dataclass(frozen=True)
class UProblem:
    """One problem of the batched unstructured workload."""
    name: str
    kind: str
    size: int
    p: int
    seed: int


C4_KINDS = (("extruded", 12), ("tetsplit", 6), ("trisplit2d", 30))


def c4_problems(n: int = 64):
    """The batched unstructured workload: n independent problems, degree
    2, 4, 6, 8 in turn, the mesh kind changing every four problems (extruded
    triangulations, split tetrahedralisations, 2D split triangulations, each
    about 5,000 cells), kappa 10^U(-2, 2) per cell and a U[-1, 1] right-hand
    side on the free DoFs from seed 1004 * 64 + i."""
    out = []
    for i in range(n):
        kind, size = C4_KINDS[(i // 4) % len(C4_KINDS)]
        out.append(UProblem(f"c4_{i}_{kind}_q{(2, 4, 6, 8)[i % 4]}", kind, size, (2, 4, 6, 8)[i % 4], 1004 * 64 + i))
    return out


def make_unstructured_problem(u: UProblem):
    """(coords, cells, vertex_on_boundary, kappa) of one batched problem: the
    mesh from the kind's own seed (shared by every problem of that kind), the
    coefficient from the problem's seed."""
    X, C, bnd = unstructured_mesh(u.kind, u.size, 4004 + [k for k, _ in C4_KINDS].index(u.kind))
    rng = np.random.default_rng(u.seed)
    kappa = 10.0 ** rng.uniform(-2.0, 2.0, len(C))
    return X, C, bnd, kappa


def refine_unstructured(coords: np.ndarray, cells: np.ndarray):
    """Uniform refinement of a quadrilateral / hexahedral mesh: every cell is cut
    into 2^d children at the midpoints of its reference axes.  New vertices:
    the old ones (same ids), then one per edge (sorted vertex pairs), one per
    face in 3D (sorted vertex quadruples), one per cell, each at the average
    of the entity's corners (the multilinear map's value there).  Child k of
    cell P (bit a of k = upper half along axis a) has its corner c at the
    reference point (bits(k) + bits(c)) / 2 of P, so its lexicographic frame is
    P's.  Returns (coords, cells, parent, child_index) of the fine mesh, fine
    cell 2^d P + k being child k of P."""
    dim = coords.shape[1]
    nv, nc, ncorner = len(coords), len(cells), 2 ** dim
    edges, faces = {}, {}
    for cv in cells:
        for c in range(ncorner):
            for a in range(dim):
                if not (c >> a) & 1:
                    edges.setdefault(tuple(sorted((int(cv[c]), int(cv[c | (1 << a)])))), None)
        if dim == 3:
            for a in range(3):
                for side in (0, 1):
                    faces.setdefault(tuple(sorted(int(cv[c]) for c in range(8) if ((c >> a) & 1) == side)), None)
    ekeys, fkeys = sorted(edges), sorted(faces)
    eid = {k: nv + i for i, k in enumerate(ekeys)}
    fid = {k: nv + len(ekeys) + i for i, k in enumerate(fkeys)}
    c0 = nv + len(ekeys) + len(fkeys)
    out = [coords[i] for i in range(nv)]
    out += [coords[list(k)].mean(axis=0) for k in ekeys]
    out += [coords[list(k)].mean(axis=0) for k in fkeys]
    out += [coords[cv].mean(axis=0) for cv in cells]

    def point(P, t):
        # the fine vertex at ternary reference position t (entries 0, 1, 2) of cell P
        cv = cells[P]
        mid = [a for a in range(dim) if t[a] == 1]
        base = sum((t[a] // 2) << a for a in range(dim) if t[a] != 1)
        corners = [int(cv[base | sum(((s >> i) & 1) << mid[i] for i in range(len(mid)))]) for s in range(2 ** len(mid))]
        if not mid:
            return corners[0]
        if len(mid) == 1:
            return eid[tuple(sorted(corners))]
        if len(mid) == 2 and dim == 3:
            return fid[tuple(sorted(corners))]
        return c0 + P

    fcells, parent, child = [], [], []
    for P in range(nc):
        for k in range(ncorner):
            fcells.append([point(P, [((k >> a) & 1) + ((c >> a) & 1) for a in range(dim)]) for c in range(ncorner)])
            parent.append(P)
            child.append(k)
    return np.array(out), np.array(fcells, dtype=np.int64), np.array(parent, dtype=np.int64), \
        np.array(child, dtype=np.uint8)


def make_refined_problem(u: UProblem):
    """Two mesh levels of one batched problem: the problem's mesh (level 0) and
    its uniform refinement (level 1) whose new vertices move by 0.2 x their
    shortest edge in a random direction; kappa 10^U(-2, 2) per coarse cell,
    inherited by its children.  Returns (coarse coords, coarse cells, fine
    coords, fine cells, parent, child, fine vertex_on_boundary, fine kappa)."""
    X, C, Xf, Cf, par, ch, bndf = _refined_mesh(u.kind, u.size)
    kappa = (10.0 ** np.random.default_rng(u.seed).uniform(-2.0, 2.0, len(C)))[par]
    return X, C, Xf, Cf, par, ch, bndf, kappa


_REFINED = {}


def _refined_mesh(kind: str, size: int):
    """The two mesh levels of a mesh kind (seeded by the kind; shared by every
    problem of that kind, built once per process)."""
    if (kind, size) not in _REFINED:
        ki = [k for k, _ in C4_KINDS].index(kind)
        X, C, _ = unstructured_mesh(kind, size, 4004 + ki)
        Xf, Cf, par, ch = refine_unstructured(X, C)
        Xf, bndf = perturb_unstructured(Xf, Cf, 0.2, np.random.default_rng(4011 + ki), first_movable=len(X))
        _REFINED[(kind, size)] = (X, C, Xf, Cf, par, ch, bndf)
    return _REFINED[(kind, size)]
