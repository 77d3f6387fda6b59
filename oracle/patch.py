"""Vertex patches, the local p-multigrid V-cycle and the patch smoother (oracle).

Test infrastructure only.  Dense FP64 linear algebra on explicitly assembled
patch matrices.

* Patch j (Section 2.1): the cells around interior vertex x_j.  Its closure
  DoFs are all nodes of those cells, its interior DoFs the nodes in the open
  interior of their union, i.e. those whose every adjacent cell of the
  unbounded grid lies in the patch (homogeneous Dirichlet on the patch
  boundary).  Both are sorted by global id.  A_j (interior x closure) is
  summed from the element matrices of the patch cells.
* Gather / Evaluate / Solve / Scatter: eqs. gather, main:4, main:5, scatter
  and Algorithm 1.
* p-hierarchy V_{j,1} c ... c V_{j,p} (Section 3.1): level operators are the
  patch operators re-evaluated with the degree-q basis; prolongation is the
  natural embedding (nodal interpolation of the coarse function at the fine
  nodes), restriction its transpose; the p = 1 level has one interior node and
  is solved exactly by A_{j,1}^{-1}.
* Smoothers: damped Jacobi d <- d + omega D^-1 (r - A d) (Section 3.1,
  "Smoothers"), or Chebyshev iteration of degree k on D^-1 A over
  [lo, hi] (three-term recurrence, Saad, Iterative Methods for Sparse Linear
  Systems, 2nd ed., Algorithm 12.1).
* V-cycle: Algorithm 2.
* Sweep: patches of colour 0, 1, ..., C-1 (or reversed) one after another,
  each computing its residual from the current u; within a colour in
  increasing vertex order.  Patches of one colour share no cell, so this is
  Algorithm 1 with the patches ordered colour-major.
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np

from . import fem


# ---------------------------------------------------------------------------
# p-level sequences
def levels_halving(p: int):
    """p, floor(p/2), ..., 1."""
    out = [p]
    while out[-1] > 1:
        out.append(out[-1] // 2)
    return out


def levels_paper(p: int):
    """The nested sequence 1, 3, 7, 15, ... (p_{k+1} = 2 p_k + 1) below p, with p
    on top (Section 3.2: p = 8 uses {1, 3, 7, 8})."""
    seq = [1]
    while 2 * seq[-1] + 1 < p:
        seq.append(2 * seq[-1] + 1)
    if seq[-1] != p:
        seq.append(p)
    return list(reversed(seq))


# ---------------------------------------------------------------------------
def interior_vertices(dim: int, N: int):
    """Interior vertex multi-indices in increasing vertex-id order (x fastest)."""
    return [v for v in fem._lex(dim, N + 1) if all(0 < v[k] < N for k in range(dim))]


def patch_id(dim: int, N: int, v) -> int:
    """Patches are numbered lexicographically over the (N-1)^d interior vertices."""
    return sum((v[k] - 1) * (N - 1) ** k for k in range(dim))


def colour_of(v) -> int:
    """Cartesian colouring: bit k of the colour is the parity of v_k.  Two
    vertices of one colour differ by an even, nonzero amount in some
    coordinate, so their patches share no cell."""
    return sum((v[k] % 2) << k for k in range(len(v)))


@dataclasses.dataclass
class PatchLevel:
    q: int
    closure: np.ndarray     # global node ids (sorted)
    interior: np.ndarray    # global node ids (sorted)
    A_ic: np.ndarray        # interior x closure
    A: np.ndarray           # interior x interior
    diag: np.ndarray
    dim: int = 0


class Patch:
    def __init__(self, mesh: fem.StructuredMesh, v, levels, elem_cache=None, element_fn=None):
        self.mesh, self.v, self.levels = mesh, tuple(v), list(levels)
        # element matrices: element_fn(cell vertices, kappa, q), default fem.element_matrix
        self.element_fn = fem.element_matrix if element_fn is None else element_fn
        d = mesh.dim
        self.cells = [tuple(v[k] - 1 + s[k] for k in range(d)) for s in fem._lex(d, 2)]
        cache = {} if elem_cache is None else elem_cache
        self.lv = {q: self._build(q, cache) for q in self.levels}
        self.P = {}
        for a, b in zip(self.levels[:-1], self.levels[1:]):
            self.P[(b, a)] = self._prolongation(b, a)

    def _build(self, q, cache):
        m = self.mesh
        cellset = set(self.cells)
        closure = sorted({int(n) for c in self.cells for n in m.cell_nodes(q, c)})
        interior = [n for n in closure
                    if all(c in cellset for c in m.cells_of_node(q, m.node_multi(q, n), clip=False))]
        pos = {n: i for i, n in enumerate(closure)}
        Acl = np.zeros((len(closure), len(closure)))
        for c in self.cells:
            key = (q, c)
            if key not in cache:
                cache[key] = self.element_fn(m.cell_vertices(c), m.kappa[m.cell_index(c)], q)
            idx = [pos[int(n)] for n in m.cell_nodes(q, c)]
            Acl[np.ix_(idx, idx)] += cache[key]
        ii = [pos[n] for n in interior]
        A_ic = Acl[ii, :]
        A = A_ic[:, ii]
        return PatchLevel(q, np.array(closure), np.array(interior), A_ic, A, np.diag(A).copy(), m.dim)

    def _prolongation(self, qc: int, qf: int) -> np.ndarray:
        """Embedding V_{j,qc} -> V_{j,qf} on interior DoFs: entry (k, i) is the
        coarse basis function i evaluated at fine node k, in a cell of the
        patch holding node k."""
        m, d = self.mesh, self.mesh.dim
        fine, coarse = self.lv[qf], self.lv[qc]
        glf = fem.rules.gauss_lobatto_nodes(qf)
        glc = fem.rules.gauss_lobatto_nodes(qc)
        L = fem.rules.lagrange(glc, glf)        # L[a, b] = l^qc_b(xi^qf_a)
        P = np.zeros((len(fine.interior), len(coarse.interior)))
        cpos = {int(n): i for i, n in enumerate(coarse.interior)}
        for k, nf in enumerate(fine.interior):
            mf = m.node_multi(qf, int(nf))
            cell = next(c for c in self.cells if all(qf * c[a] <= mf[a] <= qf * c[a] + qf for a in range(d)))
            for loc in fem._lex(d, qc + 1):
                nc = m.node_index(qc, [qc * cell[a] + loc[a] for a in range(d)])
                if nc not in cpos:
                    continue            # a patch-boundary node: zero in V_{j,qc}
                val = 1.0
                for a in range(d):
                    val *= L[mf[a] - qf * cell[a], loc[a]]
                P[k, cpos[nc]] = val
        return P

    # -- Evaluate (eq. main:4) ------------------------------------------------
    def residual(self, u: np.ndarray, b: np.ndarray) -> np.ndarray:
        top = self.lv[self.levels[0]]
        return b[top.interior] - top.A_ic @ u[top.closure]


@dataclasses.dataclass
class Smoother:
    kind: str = "chebyshev"      # "chebyshev", "jacobi" or "fdm" (Cartesian-reinforced)
    degree: int = 3              # Chebyshev degree
    omega: float = 0.5           # damping of the Jacobi and Cartesian-reinforced steps
    steps: int = 1               # smoothing steps (pre and post each)


def jacobi(A, diag, r, d, omega, steps):
    for _ in range(steps):
        d = d + omega * (r - A @ d) / diag
    return d


def chebyshev(A, diag, r, d, lo, hi, degree, zero_start=False):
    """Degree-`degree` Chebyshev iteration for D^-1 A d = D^-1 r on [lo, hi],
    starting from d (Saad, Algorithm 12.1 applied to the Jacobi-preconditioned
    system)."""
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    res = (r if zero_start else r - A @ d) / diag
    dirn = res / theta
    for i in range(degree):
        d = d + dirn
        if i == degree - 1:
            break
        res = res - (A @ dirn) / diag
        rho_new = 1.0 / (2.0 * sigma - rho)
        dirn = rho_new * rho * dirn + (2.0 * rho_new / delta) * res
        rho = rho_new
    return d


_REFERENCE = {}


def reference_patch_matrix(dim: int, q: int) -> np.ndarray:
    """A_{b,q}: the interior matrix of the undeformed Cartesian patch (2^d
    square/cube cells, kappa = 1) at degree q (Section 3.1, Cartesian-reinforced
    smoother), assembled like any patch matrix."""
    key = (dim, q)
    if key not in _REFERENCE:
        g = np.linspace(0.0, 1.0, 3)
        axes = np.meshgrid(*([g] * dim), indexing="ij")
        X = np.stack([a.T.reshape(-1) for a in axes], axis=1)    # x fastest
        m = fem.StructuredMesh(dim, 2, X, np.ones(2 ** dim))
        _REFERENCE[key] = Patch(m, (1,) * dim, [q]).lv[q].A
    return _REFERENCE[key]


def cartesian_reinforced(lv: PatchLevel, r, d, omega, steps):
    """Damped Richardson steps d <- d + omega P^-1 (r - A d) with the
    Cartesian-reinforced preconditioner of Section 3.1: the reference patch
    inverse A_b^-1, rescaled by diag(A_b) and the inverse diagonal of the
    actual patch matrix, P^-1 = diag(A_j)^-1 diag(A_b) A_b^-1."""
    Ab = reference_patch_matrix(lv.dim, lv.q)
    scale = np.diag(Ab) / lv.diag
    for _ in range(steps):
        d = d + omega * scale * np.linalg.solve(Ab, r - lv.A @ d)
    return d


def smooth(lv: PatchLevel, r, d, sm: Smoother, bounds, zero_start):
    if sm.kind == "jacobi":
        return jacobi(lv.A, lv.diag, r, d, sm.omega, sm.steps)
    if sm.kind == "fdm":
        return cartesian_reinforced(lv, r, d, sm.omega, sm.steps)
    lo, hi = bounds
    for s in range(sm.steps):
        d = chebyshev(lv.A, lv.diag, r, d, lo, hi, sm.degree, zero_start and s == 0)
    return d


def vcycle(patch: Patch, k: int, d, r, sm: Smoother, bounds, zero_start=False):
    """Algorithm 2 on level index k of patch.levels; bounds[q] = (lo, hi)."""
    q = patch.levels[k]
    lv = patch.lv[q]
    if q == 1:
        return r / lv.A[0, 0]                                     # coarse 1x1 solve
    d = smooth(lv, r, d, sm, bounds.get(q), zero_start)           # pre-smoothing
    res = r - lv.A @ d                                            # residual
    qc = patch.levels[k + 1]
    P = patch.P[(qc, q)]
    e = vcycle(patch, k + 1, np.zeros(P.shape[1]), P.T @ res, sm, bounds, zero_start=True)
    d = d + P @ e                                                 # correction
    d = smooth(lv, r, d, sm, bounds.get(q), False)                # post-smoothing
    return d


def local_solve(patch: Patch, r, sm: Smoother, bounds, n_cycles=1):
    """N_MG V-cycles, the first from d = 0 (eq. main:5)."""
    d = np.zeros_like(r)
    for c in range(n_cycles):
        d = vcycle(patch, 0, d, r, sm, bounds, zero_start=(c == 0))
    return d


def vcycle_matrix(patch: Patch, sm: Smoother, bounds, n_cycles=1) -> np.ndarray:
    """The linear operator r -> d of the local solver, column by column."""
    n = len(patch.lv[patch.levels[0]].interior)
    return np.column_stack([local_solve(patch, e, sm, bounds, n_cycles) for e in np.eye(n)])


# ---------------------------------------------------------------------------
class PatchSmoother:
    """All interior-vertex patches of one mesh, with per-(patch, level) bounds."""

    def __init__(self, mesh: fem.StructuredMesh, p: int, levels=None, sm: Smoother | None = None,
                 bounds_fn=None, n_cycles: int = 1, order: str = "colour", additive: bool = False,
                 theta: float = 1.0, element_fn=None):
        self.mesh, self.p = mesh, p
        self.element_fn = element_fn   # patch element matrices (None: fem.element_matrix)
        self.order = order             # "colour": colour-major; "vertex": plain vertex order
        self.additive, self.theta = additive, theta
        self._mult = None
        self.levels = levels_halving(p) if levels is None else levels
        self.sm = Smoother() if sm is None else sm
        self.n_cycles = n_cycles
        self.vertices = interior_vertices(mesh.dim, mesh.N)
        self._cache = {}
        self._patches = {}
        self.bounds_fn = bounds_fn     # (patch) -> {q: (lo, hi)}
        self._bounds = {}

    def patch(self, v) -> Patch:
        v = tuple(v)
        if v not in self._patches:
            self._patches[v] = Patch(self.mesh, v, self.levels, self._cache, self.element_fn)
        return self._patches[v]

    def bounds(self, v):
        v = tuple(v)
        if self.sm.kind == "jacobi":
            return {}
        if v not in self._bounds:
            self._bounds[v] = self.bounds_fn(self.patch(v), patch_id(self.mesh.dim, self.mesh.N, v))
        return self._bounds[v]

    def update(self, v, u, b):
        """Gather, Evaluate, Solve; returns (interior ids, d_j)."""
        P = self.patch(v)
        r = P.residual(u, b)
        d = local_solve(P, r, self.sm, self.bounds(v), self.n_cycles)
        return P.lv[self.levels[0]].interior, d

    def multiplicity(self) -> np.ndarray:
        """Number of patches whose interior holds each global DoF (0 off every
        patch), counted patch by patch."""
        if self._mult is None:
            m = np.zeros(self.mesh.n_nodes(self.p))
            for v in self.vertices:
                m[self.patch(v).lv[self.levels[0]].interior] += 1
            self._mult = m
        return self._mult

    def sweep_additive(self, u, b, reverse=False):
        """Weighted additive sweep: every patch solves with the residual of the
        same u, the corrections are summed, u += theta W sum_j Pi_j^T d_j with
        W = diag(1 / multiplicity).  reverse: the transpose, W applied to the
        residual instead (u += theta sum_j Pi_j^T B_j Pi_j W (b - A u)), so that
        a V-cycle with the forward sweep before and the reverse one after the
        coarse correction is symmetric."""
        mult = self.multiplicity()
        w = np.divide(1.0, mult, out=np.zeros_like(mult), where=mult > 0)
        corr = np.zeros_like(u)
        for v in self.vertices:
            P = self.patch(v)
            idx = P.lv[self.levels[0]].interior
            r = P.residual(u, b)
            if reverse:
                r = w[idx] * r
            corr[idx] += local_solve(P, r, self.sm, self.bounds(v), self.n_cycles)
        return u + self.theta * (corr if reverse else w * corr)

    def sweep(self, u, b, reverse=False, colours=None, within="increasing"):
        if self.additive:
            return self.sweep_additive(u, b, reverse)
        """One multiplicative sweep (Algorithm 1, colour-major order).  `within`
        orders the patches of one colour ("increasing" or "decreasing" vertex
        id).  With order "vertex" the patches run in plain vertex order
        (decreasing when reversed), one after the other."""
        u = u.copy()
        if self.order == "vertex":
            for v in (self.vertices[::-1] if reverse else self.vertices):
                idx, d = self.update(v, u, b)
                u[idx] += d
            return u
        n_col = 2 ** self.mesh.dim
        order = list(range(n_col)) if colours is None else list(colours)
        if reverse:
            order = order[::-1]
        verts = self.vertices if within == "increasing" else self.vertices[::-1]
        for c in order:
            for v in verts:
                if colour_of(v) != c:
                    continue
                idx, d = self.update(v, u, b)
                u[idx] += d                                          # Scatter
        return u
