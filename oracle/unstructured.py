"""Vertex patches on unstructured quadrilateral / hexahedral meshes (oracle).

Test infrastructure only.  Everything is assembled explicitly in FP64 with
dense patch matrices, from the same definitions as the structured oracle
(fem.element_matrix, patch.vcycle): only the mesh topology differs.

Mesh.  d = 2: quadrilaterals; d = 3: hexahedra.  A cell is given by its 2^d
vertex ids in lexicographic corner order: corner c sits at the reference
point whose k-th coordinate is bit k of c.  Each cell is the multilinear image
of [0,1]^d (Q1 geometry), kappa is constant per cell.  The boundary of the
domain is the union of the facets (edges in 2D, faces in 3D) that belong to
one cell only; its DoFs carry homogeneous Dirichlet values.

Global DoF numbering of the degree-q space (a reading: the paper works with
deal.II's numbering and does not state one):
  1. vertices, by vertex id;
  2. edges sorted by (smaller vertex id, larger vertex id), q - 1 interior
     nodes each, numbered from the end with the smaller vertex id;
  3. (3D) faces sorted by their sorted vertex ids, (q - 1)^2 interior nodes,
     numbered in the frame of the face's smallest-id corner: the first axis
     runs toward the smaller-id of its two neighbours on the face, the second
     toward the other, the first axis fastest;
  4. cells by id, (q - 1)^d interior nodes in the cell's own reference frame,
     x fastest.
Nodes sit at the Gauss-Lobatto points of the reference cell, so two cells
sharing an entity agree on its nodes after the orientation above.

Patch j of an interior vertex (one not on the boundary): the cells containing
it (their number is the vertex's valence).  Closure DoFs: every node of those
cells; interior DoFs: the nodes whose every containing cell is a patch cell
and that are not on the domain boundary (the open interior of the union).
p-levels, transfers, smoothers and the V-cycle are those of patch.py
(Section 3.1, Algorithm 2); the p-prolongation entry (k, i) is coarse basis
function i at fine node k, evaluated in a patch cell containing node k.

Colours (the paper does not colour; this greedy rule is a reading): two
patches conflict when they share a cell; vertices are visited in decreasing
priority (splitmix64(vertex id XOR seed), vertex id) and each takes the
smallest colour no conflicting, already coloured patch has.  Within a colour
patches share no cell, so their interiors are disjoint and the sweep (Algorithm
1, colour-major, increasing vertex id within a colour) is independent of the
order inside a colour.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from . import fem, lanczos as lz, patch as pt, rules


def _lex(dim, n):
    return fem._lex(dim, n)


class Mesh:
    def __init__(self, dim: int, coords, cells, kappa):
        self.dim = dim
        self.coords = np.asarray(coords, dtype=np.float64).reshape(-1, dim)
        self.cells = np.asarray(cells, dtype=np.int64).reshape(-1, 2 ** dim)
        self.kappa = np.asarray(kappa, dtype=np.float64).reshape(-1)
        self.nv, self.nc = len(self.coords), len(self.cells)
        assert len(self.kappa) == self.nc
        self._topology()
        self._dofmaps = {}
        self._elem = {}

    # ------------------------------------------------------------- topology
    def _entity_corners(self):
        """Corner lists of the cell's edges (and faces in 3D) in reference terms:
        [(fixed axes and values, running axes, corner ids in lexicographic order of the running axes)]."""
        d = self.dim
        ents = {1: [], 2: []}
        for run in (1, 2):
            if run > d - 1 and not (run == 1):
                continue
            if run == 2 and d < 3:
                continue
            for axes in itertools.combinations(range(d), run):
                fixed = [a for a in range(d) if a not in axes]
                for vals in itertools.product((0, 1), repeat=len(fixed)):
                    corners = []
                    for bits in _lex(run, 2):
                        c = 0
                        for a, v in zip(fixed, vals):
                            c |= v << a
                        for a, bt in zip(axes, bits):
                            c |= bt << a
                        corners.append(c)
                    ents[run].append((tuple(zip(fixed, vals)), axes, corners))
        return ents

    def _topology(self):
        d = self.dim
        self.ref_entities = self._entity_corners()
        edges, faces = {}, {}
        self.cell_edges = []
        self.cell_faces = []
        for ci, cv in enumerate(self.cells):
            ce = []
            for fixed, axes, corners in self.ref_entities[1]:
                key = tuple(sorted(int(cv[c]) for c in corners))
                edges.setdefault(key, []).append(ci)
                ce.append(key)
            self.cell_edges.append(ce)
            cf = []
            for fixed, axes, corners in self.ref_entities[2] if d == 3 else []:
                key = tuple(sorted(int(cv[c]) for c in corners))
                faces.setdefault(key, []).append(ci)
                cf.append(key)
            self.cell_faces.append(cf)
        self.edge_keys = sorted(edges)
        self.edge_id = {k: i for i, k in enumerate(self.edge_keys)}
        self.edge_cells = edges
        self.face_keys = sorted(faces)
        self.face_id = {k: i for i, k in enumerate(self.face_keys)}
        self.face_cells = faces
        self.vertex_cells = [[] for _ in range(self.nv)]
        for ci, cv in enumerate(self.cells):
            for v in cv:
                self.vertex_cells[int(v)].append(ci)
        # boundary facets: one cell only
        facets = faces if d == 3 else edges
        bverts = set()
        self.boundary_edges, self.boundary_faces = set(), set()
        for key, cs in facets.items():
            if len(cs) == 1:
                bverts.update(key)
                if d == 3:
                    self.boundary_faces.add(key)
                else:
                    self.boundary_edges.add(key)
        if d == 3:
            for key in self.boundary_faces:
                # the four edges of a boundary face
                ci = self.face_cells[key][0]
                for fixed, axes, corners in self.ref_entities[2]:
                    cv = self.cells[ci]
                    if tuple(sorted(int(cv[c]) for c in corners)) != key:
                        continue
                    for a in range(2):
                        for val in (0, 1):
                            pair = [corners[i] for i in range(4) if ((i >> (1 - a)) & 1) == val]
                            self.boundary_edges.add(tuple(sorted(int(cv[c]) for c in pair)))
        self.vertex_on_boundary = np.zeros(self.nv, dtype=bool)
        self.vertex_on_boundary[list(bverts)] = True

    def valence(self, v: int) -> int:
        return len(self.vertex_cells[v])

    def interior_vertices(self):
        return [v for v in range(self.nv) if not self.vertex_on_boundary[v]]

    # ---------------------------------------------------------- DoF numbering
    def n_dofs(self, q: int) -> int:
        return self.nv + len(self.edge_keys) * (q - 1) + len(self.face_keys) * (q - 1) ** 2 + self.nc * (q - 1) ** self.dim

    def cell_dofs(self, q: int) -> np.ndarray:
        """[cell][(q+1)^d] global DoF ids of each cell's nodes (local order lexicographic, x fastest)."""
        if q in self._dofmaps:
            return self._dofmaps[q]
        d = self.dim
        ne, nf = len(self.edge_keys), len(self.face_keys)
        e0 = self.nv
        f0 = e0 + ne * (q - 1)
        c0 = f0 + nf * (q - 1) ** 2
        out = np.zeros((self.nc, (q + 1) ** d), dtype=np.int64)
        for ci, cv in enumerate(self.cells):
            for li, m in enumerate(_lex(d, q + 1)):
                onb = [k for k in range(d) if m[k] in (0, q)]
                if len(onb) == d:                                    # a vertex
                    c = sum((m[k] // q) << k for k in range(d))
                    out[ci, li] = cv[c]
                elif len(onb) == d - 1:                              # an edge: one running axis
                    a = [k for k in range(d) if k not in onb][0]
                    base = sum((m[k] // q) << k for k in onb)
                    v0, v1 = int(cv[base]), int(cv[base | (1 << a)])
                    t = m[a] if v0 < v1 else q - m[a]
                    out[ci, li] = e0 + self.edge_id[(min(v0, v1), max(v0, v1))] * (q - 1) + (t - 1)
                elif d == 3 and len(onb) == 1:                       # a face: two running axes
                    fa = onb[0]
                    r1, r2 = [k for k in range(3) if k != fa]
                    fbit = (m[fa] // q) << fa
                    corner = {(b1, b2): fbit | (b1 << r1) | (b2 << r2) for b1 in (0, 1) for b2 in (0, 1)}
                    ids = {bb: int(cv[c]) for bb, c in corner.items()}
                    anchor = min(ids, key=lambda bb: ids[bb])
                    n1 = (1 - anchor[0], anchor[1])                  # neighbour along r1
                    n2 = (anchor[0], 1 - anchor[1])                  # neighbour along r2
                    s1 = m[r1] if anchor[0] == 0 else q - m[r1]      # distances from the anchor
                    s2 = m[r2] if anchor[1] == 0 else q - m[r2]
                    u, w = (s1, s2) if ids[n1] < ids[n2] else (s2, s1)
                    key = tuple(sorted(ids.values()))
                    out[ci, li] = f0 + self.face_id[key] * (q - 1) ** 2 + (u - 1) + (q - 1) * (w - 1)
                else:                                                # cell interior
                    loc = sum((m[k] - 1) * (q - 1) ** k for k in range(d))
                    out[ci, li] = c0 + ci * (q - 1) ** d + loc
        self._dofmaps[q] = out
        return out

    def boundary_dofs(self, q: int) -> np.ndarray:
        """True on the DoFs of the boundary facets (with their edges and vertices)."""
        out = np.zeros(self.n_dofs(q), dtype=bool)
        out[np.nonzero(self.vertex_on_boundary)[0]] = True
        e0 = self.nv
        for key in self.boundary_edges:
            i = self.edge_id[key]
            out[e0 + i * (q - 1): e0 + (i + 1) * (q - 1)] = True
        if self.dim == 3:
            f0 = e0 + len(self.edge_keys) * (q - 1)
            for key in self.boundary_faces:
                i = self.face_id[key]
                out[f0 + i * (q - 1) ** 2: f0 + (i + 1) * (q - 1) ** 2] = True
        return out

    def dof_cells(self, q: int):
        """For every DoF, the cells whose closure holds it."""
        cd = self.cell_dofs(q)
        out = [[] for _ in range(self.n_dofs(q))]
        for ci in range(self.nc):
            for g in cd[ci]:
                out[int(g)].append(ci)
        return out

    def node_coords(self, q: int) -> np.ndarray:
        """Physical position of every DoF (from the first cell holding it)."""
        gl = rules.gauss_lobatto_nodes(q)
        X = np.full((self.n_dofs(q), self.dim), np.nan)
        cd = self.cell_dofs(q)
        for ci in range(self.nc):
            xi = np.array([[gl[m[k]] for k in range(self.dim)] for m in _lex(self.dim, q + 1)])
            Nq, _ = fem.q1_shape(self.dim, xi)
            pts = Nq @ self.coords[self.cells[ci]]
            X[cd[ci]] = pts
        return X

    # ----------------------------------------------------------- assembly
    def cell_vertices(self, ci: int) -> np.ndarray:
        return self.coords[self.cells[ci]]

    def element_matrix(self, ci: int, q: int) -> np.ndarray:
        key = (ci, q)
        if key not in self._elem:
            self._elem[key] = fem.element_matrix(self.cell_vertices(ci), self.kappa[ci], q)
        return self._elem[key]

    def assemble(self, q: int) -> sp.csr_matrix:
        cd = self.cell_dofs(q)
        rows, cols, vals = [], [], []
        for ci in range(self.nc):
            idx = cd[ci]
            rows.append(np.repeat(idx, len(idx)))
            cols.append(np.tile(idx, len(idx)))
            vals.append(self.element_matrix(ci, q).reshape(-1))
        n = self.n_dofs(q)
        return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(n, n)).tocsr()

    def load_vector(self, f, q: int, n_quad: int) -> np.ndarray:
        b = np.zeros(self.n_dofs(q))
        cd = self.cell_dofs(q)
        for ci in range(self.nc):
            b[cd[ci]] += fem.element_load(self.cell_vertices(ci), f, q, n_quad)
        return b


# ---------------------------------------------------------------- patches
class Patch:
    """Patch of interior vertex v of an unstructured mesh, with the interface of
    patch.Patch (levels, lv[q], P[(qc, qf)], residual) used by patch.vcycle."""

    def __init__(self, mesh: Mesh, v: int, levels):
        assert not mesh.vertex_on_boundary[v]
        self.mesh, self.v, self.levels = mesh, v, list(levels)
        self.cells = sorted(mesh.vertex_cells[v])
        self.lv = {q: self._build(q) for q in self.levels}
        self.P = {}
        for a, b in zip(self.levels[:-1], self.levels[1:]):
            self.P[(b, a)] = self._prolongation(b, a)

    def _build(self, q):
        m = self.mesh
        cd = m.cell_dofs(q)
        cellset = set(self.cells)
        closure = sorted({int(g) for c in self.cells for g in cd[c]})
        bnd = m.boundary_dofs(q)
        owners = m.dof_cells(q)
        interior = [g for g in closure if not bnd[g] and all(c in cellset for c in owners[g])]
        pos = {g: i for i, g in enumerate(closure)}
        Acl = np.zeros((len(closure), len(closure)))
        for c in self.cells:
            idx = [pos[int(g)] for g in cd[c]]
            Acl[np.ix_(idx, idx)] += m.element_matrix(c, q)
        ii = [pos[g] for g in interior]
        A_ic = Acl[ii, :]
        A = A_ic[:, ii]
        return pt.PatchLevel(q, np.array(closure), np.array(interior), A_ic, A, np.diag(A).copy(), m.dim)

    def _prolongation(self, qc, qf):
        m, d = self.mesh, self.mesh.dim
        fine, coarse = self.lv[qf], self.lv[qc]
        cdf, cdc = m.cell_dofs(qf), m.cell_dofs(qc)
        glf, glc = rules.gauss_lobatto_nodes(qf), rules.gauss_lobatto_nodes(qc)
        L = rules.lagrange(glc, glf)                                  # L[a, b] = l^qc_b(xi^qf_a)
        cpos = {int(g): i for i, g in enumerate(coarse.interior)}
        fpos = {int(g): i for i, g in enumerate(fine.interior)}
        P = np.zeros((len(fine.interior), len(coarse.interior)))
        done = set()
        for c in self.cells:
            floc = list(_lex(d, qf + 1))
            cloc = list(_lex(d, qc + 1))
            for li, mf in enumerate(floc):
                g = int(cdf[c, li])
                if g not in fpos or g in done:
                    continue
                done.add(g)
                for lj, mc in enumerate(cloc):
                    gc = int(cdc[c, lj])
                    if gc not in cpos:
                        continue
                    val = 1.0
                    for a in range(d):
                        val *= L[mf[a], mc[a]]
                    P[fpos[g], cpos[gc]] = val
        return P

    def residual(self, u, b):
        top = self.lv[self.levels[0]]
        return b[top.interior] - top.A_ic @ u[top.closure]


def colours(mesh: Mesh, seed: int = 0):
    """{vertex: colour} for the interior vertices: greedy in decreasing
    priority (splitmix64(v ^ seed), v), smallest colour free among the
    already coloured patches that share a cell."""
    verts = mesh.interior_vertices()
    key = {v: (lz.splitmix64(v ^ seed), v) for v in verts}
    order = sorted(verts, key=lambda v: key[v], reverse=True)
    col = {}
    for v in order:
        used = set()
        for c in mesh.vertex_cells[v]:
            for w in mesh.cells[c]:
                w = int(w)
                if w in col:
                    used.add(col[w])
        k = 0
        while k in used:
            k += 1
        col[v] = k
    return col


class PatchSmoother:
    """Multiplicative vertex-patch sweep on an unstructured mesh (Algorithm 1,
    colour-major, increasing vertex id within a colour)."""

    def __init__(self, mesh: Mesh, p: int, levels=None, sm=None, bounds_fn=None, seed: int = 0):
        self.mesh, self.p = mesh, p
        self.levels = pt.levels_halving(p) if levels is None else levels
        self.sm = pt.Smoother() if sm is None else sm
        self.bounds_fn = bounds_fn
        self.col = colours(mesh, seed)
        self.n_colours = 1 + max(self.col.values()) if self.col else 0
        self._patches, self._bounds = {}, {}

    def patch(self, v) -> Patch:
        if v not in self._patches:
            self._patches[v] = Patch(self.mesh, v, self.levels)
        return self._patches[v]

    def bounds(self, v):
        if self.sm.kind == "jacobi":
            return {}
        if v not in self._bounds:
            self._bounds[v] = self.bounds_fn(self.patch(v), v)
        return self._bounds[v]

    def sweep(self, u, b, reverse=False):
        u = u.copy()
        order = list(range(self.n_colours))
        if reverse:
            order = order[::-1]
        for c in order:
            for v in sorted(self.col):
                if self.col[v] != c:
                    continue
                P = self.patch(v)
                d = pt.local_solve(P, P.residual(u, b), self.sm, self.bounds(v), 1)
                u[P.lv[self.levels[0]].interior] += d
        return u


# ------------------------------------------------------------ global solver
def q1_prolongation(mesh: Mesh, q: int) -> sp.csr_matrix:
    """Embedding of the Q1 space into the degree-q space of the same mesh:
    entry (k, v) is vertex function v at DoF k, evaluated in a cell holding k."""
    d = mesh.dim
    gl = rules.gauss_lobatto_nodes(q)
    cd = mesh.cell_dofs(q)
    rows, cols, vals = [], [], []
    done = set()
    for c in range(mesh.nc):
        for li, m in enumerate(_lex(d, q + 1)):
            g = int(cd[c, li])
            if g in done:
                continue
            done.add(g)
            for v in range(2 ** d):
                val = 1.0
                for k in range(d):
                    val *= gl[m[k]] if (v >> k) & 1 else 1.0 - gl[m[k]]
                if val != 0.0:
                    rows.append(g)
                    cols.append(int(mesh.cells[c, v]))
                    vals.append(val)
    return sp.coo_matrix((vals, (rows, cols)), shape=(mesh.n_dofs(q), mesh.nv)).tocsr()


class TwoLevel:
    """Two-level preconditioner on an unstructured mesh: one multiplicative
    patch sweep (colours increasing), the residual restricted to the Q1 space
    of the same mesh (re-discretised with its own 2-point Gauss rule, the
    reading of Section 3.1 "Level operators" carried to the global coarse
    level), solved by a dense Cholesky factorisation, prolongated by the
    embedding, then one sweep with the colours reversed: a symmetric
    preconditioner for CG."""

    def __init__(self, mesh: Mesh, p: int, smoother: PatchSmoother):
        import scipy.linalg as sla
        self.mesh, self.p, self.S = mesh, p, smoother
        self.free = ~mesh.boundary_dofs(p)
        self.A = fem.operator_with_dirichlet(mesh.assemble(p), self.free)
        free1 = ~mesh.boundary_dofs(1)
        self.free1 = free1
        A1 = mesh.assemble(1).toarray()[np.ix_(free1, free1)]
        self.chol = sla.cho_factor(A1, lower=True)
        Df = sp.diags(self.free.astype(float))
        D1 = sp.diags(free1.astype(float))
        self.P = (Df @ q1_prolongation(mesh, p) @ D1).tocsr()

    def vcycle(self, b):
        import scipy.linalg as sla
        x = self.S.sweep(np.zeros_like(b), b, reverse=False)
        r = b - self.A @ x
        r1 = self.P.T @ r
        e1 = np.zeros(self.mesh.nv)
        e1[self.free1] = sla.cho_solve(self.chol, r1[self.free1])
        x = x + self.P @ e1
        return self.S.sweep(x, b, reverse=True)


# ------------------------------------------------------ two mesh levels
def h_prolongation(coarse: Mesh, fine: Mesh, parent, child, q: int) -> sp.csr_matrix:
    """Embedding of the degree-q space of `coarse` into that of its uniform
    refinement `fine` (fine cell c is child child[c] of coarse cell parent[c],
    its frame the parent's): entry (g, G) is coarse basis function G at fine
    DoF g, evaluated in the parent of a fine cell holding g at the reference
    point (bits(child) + xi) / 2 (Section 2: transfers through the reference
    cells, which makes them independent of the vertex positions)."""
    d = fine.dim
    gl = rules.gauss_lobatto_nodes(q)
    cdf, cdc = fine.cell_dofs(q), coarse.cell_dofs(q)
    rows, cols, vals = [], [], []
    done = set()
    for c in range(fine.nc):
        P, k = int(parent[c]), int(child[c])
        for li, m in enumerate(_lex(d, q + 1)):
            g = int(cdf[c, li])
            if g in done:
                continue
            done.add(g)
            lx = [rules.lagrange(gl, np.array([(((k >> a) & 1) + gl[m[a]]) / 2.0]))[0] for a in range(d)]
            for lj, mc in enumerate(_lex(d, q + 1)):
                val = 1.0
                for a in range(d):
                    val *= lx[a][mc[a]]
                if val != 0.0:
                    rows.append(g)
                    cols.append(int(cdc[P, lj]))
                    vals.append(val)
    return sp.coo_matrix((vals, (rows, cols)), shape=(fine.n_dofs(q), coarse.n_dofs(q))).tocsr()


class TwoMeshLevels:
    """Degree p on a fine mesh and on the coarse mesh it refines: one
    multiplicative sweep on the fine mesh, the residual restricted by the
    transposed h-embedding, the coarse mesh's two-level cycle (TwoLevel: its
    sweep, its Q1 coarse space, its reversed sweep), the correction
    prolongated, one sweep with the colours reversed: a symmetric
    preconditioner for CG."""

    def __init__(self, coarse: Mesh, fine: Mesh, parent, child, p: int, fine_smoother: PatchSmoother,
                 coarse_smoother: PatchSmoother):
        self.coarse, self.fine, self.p = coarse, fine, p
        self.S = fine_smoother
        self.TLc = TwoLevel(coarse, p, coarse_smoother)
        self.free = ~fine.boundary_dofs(p)
        self.A = fem.operator_with_dirichlet(fine.assemble(p), self.free)
        freec = ~coarse.boundary_dofs(p)
        Df = sp.diags(self.free.astype(float))
        Dc = sp.diags(freec.astype(float))
        self.P = (Df @ h_prolongation(coarse, fine, parent, child, p) @ Dc).tocsr()

    def vcycle(self, b):
        x = self.S.sweep(np.zeros_like(b), b, reverse=False)
        r = b - self.A @ x
        x = x + self.P @ self.TLc.vcycle(self.P.T @ r)
        return self.S.sweep(x, b, reverse=True)
