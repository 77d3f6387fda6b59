"""Q_q finite elements on structured-topology meshes with Q1 geometry (oracle).

Test infrastructure only.  Everything is assembled explicitly in FP64.

The bilinear form is a(u, v) = int kappa grad u . grad v (Section 2,
eq. bilinear-form); the discrete operator A_l of eq. matrix collects it on the
basis of V_l.  Each cell is the image of [0,1]^d under the multilinear map of
its 2^d vertices; the element matrix at degree q is

    A^c_ab = sum_g w_g kappa_c det J(xi_g) (J^-T grad phi_a) . (J^-T grad phi_b)

over the (q+1)^d-point Gauss rule.  Nodes and vertices are numbered
lexicographically with x fastest, locally and globally; the global node grid
of a degree-q space on an N^d mesh has (qN+1)^d nodes, those on the boundary
of the unit square/cube carry homogeneous Dirichlet conditions.
"""
from __future__ import annotations

import itertools
from functools import lru_cache

import numpy as np
import scipy.sparse as sp

from . import rules


class DegenerateCell(ValueError):
    pass


def q1_shape(dim: int, xi: np.ndarray):
    """Values N[g, v] and gradients dN[g, v, k] of the 2^d multilinear vertex
    functions at reference points xi (n_g x dim); vertex v has bit k of v = 1
    iff it sits at xi_k = 1."""
    xi = np.atleast_2d(xi)
    ng = xi.shape[0]
    nv = 2 ** dim
    N = np.ones((ng, nv))
    dN = np.ones((ng, nv, dim))
    for v in range(nv):
        for k in range(dim):
            bit = (v >> k) & 1
            f = xi[:, k] if bit else 1.0 - xi[:, k]
            df = 1.0 if bit else -1.0
            N[:, v] *= f
            for j in range(dim):
                dN[:, v, j] *= df if j == k else f
    return N, dN


def jacobians(cell_x: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """J[g, i, j] = d x_i / d xi_j of the multilinear map at points xi."""
    _, dN = q1_shape(cell_x.shape[1], xi)
    return np.einsum("vi,gvj->gij", cell_x, dN)


@lru_cache(maxsize=None)
def tensor_rule(dim: int, n: int):
    """Tensor Gauss rule with n points per direction: points (n^d x d), weights."""
    x, w = rules.gauss(n)
    pts = np.array([[x[i[k]] for k in range(dim)] for i in _lex(dim, n)])
    wts = np.array([np.prod([w[i[k]] for k in range(dim)]) for i in _lex(dim, n)])
    return pts, wts


def _lex(dim: int, n: int):
    """Multi-indices (i_x, i_y[, i_z]) in lexicographic order, x fastest."""
    for t in itertools.product(range(n), repeat=dim):
        yield tuple(reversed(t))


@lru_cache(maxsize=None)
def basis_at(dim: int, q: int, n_quad: int):
    """Reference basis values phi[g, a] and gradients gphi[g, a, k] of the
    degree-q Lagrange basis on Gauss-Lobatto nodes at the tensor Gauss points."""
    nodes = rules.gauss_lobatto_nodes(q)
    xg, _ = rules.gauss(n_quad)
    L = rules.lagrange(nodes, xg)
    D = rules.lagrange_deriv(nodes, xg)
    G = list(_lex(dim, n_quad))
    A = list(_lex(dim, q + 1))
    phi = np.ones((len(G), len(A)))
    gphi = np.ones((len(G), len(A), dim))
    for gi, g in enumerate(G):
        for ai, a in enumerate(A):
            for k in range(dim):
                phi[gi, ai] *= L[g[k], a[k]]
                for j in range(dim):
                    gphi[gi, ai, j] *= D[g[k], a[k]] if j == k else L[g[k], a[k]]
    return phi, gphi


def element_matrix(cell_x: np.ndarray, kappa: float, q: int, n_quad: int | None = None) -> np.ndarray:
    """Element stiffness matrix of degree q on the cell with vertices cell_x."""
    dim = cell_x.shape[1]
    n_quad = q + 1 if n_quad is None else n_quad
    pts, wts = tensor_rule(dim, n_quad)
    _, gphi = basis_at(dim, q, n_quad)
    J = jacobians(cell_x, pts)
    det = np.linalg.det(J)
    if np.any(det <= 0.0):
        raise DegenerateCell("det J <= 0 at a quadrature point")
    Jinv = np.linalg.inv(J)
    grad = np.einsum("gkj,gak->gaj", Jinv, gphi)         # J^-T grad_hat
    return np.einsum("g,gaj,gbj->ab", wts * kappa * det, grad, grad)


def bf16_round(x) -> np.ndarray:
    """x rounded to FP32 and then to the nearest BF16 number (8-bit
    significand, ties to even), returned in FP64: the value that a BF16 copy of
    an FP32 quantity holds (the mixed-precision form's operator data, where
    the error budget allows it).  Finite inputs."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def element_matrix_G(cell_x: np.ndarray, kappa: float, q: int, n_quad: int | None = None,
                     g_round=None) -> np.ndarray:
    """The element matrix of element_matrix written through the per-point
    tensors G_g = w_g kappa det J J^-1 J^-T (A^c_ab = sum_g grad_hat phi_a . G_g
    grad_hat phi_b), each component of G passed through g_round first (None:
    exact).  With g_round = bf16_round it is the operator the patch kernels
    apply when they read BF16 geometry."""
    dim = cell_x.shape[1]
    n_quad = q + 1 if n_quad is None else n_quad
    pts, wts = tensor_rule(dim, n_quad)
    _, gphi = basis_at(dim, q, n_quad)
    J = jacobians(cell_x, pts)
    det = np.linalg.det(J)
    if np.any(det <= 0.0):
        raise DegenerateCell("det J <= 0 at a quadrature point")
    Jinv = np.linalg.inv(J)
    G = np.einsum("g,gkj,glj->gkl", wts * kappa * det, Jinv, Jinv)
    if g_round is not None:
        G = g_round(G)
    return np.einsum("gak,gkl,gbl->ab", gphi, G, gphi)


def element_load(cell_x: np.ndarray, f, q: int, n_quad: int) -> np.ndarray:
    """int f phi_a over the cell with the n_quad-point Gauss rule per direction."""
    dim = cell_x.shape[1]
    pts, wts = tensor_rule(dim, n_quad)
    phi, _ = basis_at(dim, q, n_quad)
    Nq, _ = q1_shape(dim, pts)
    xq = Nq @ cell_x
    det = np.linalg.det(jacobians(cell_x, pts))
    return np.einsum("g,ga->a", wts * det * f(xq), phi)


def corner_dets(cell_x: np.ndarray) -> np.ndarray:
    dim = cell_x.shape[1]
    corners = np.array([[(v >> k) & 1 for k in range(dim)] for v in range(2 ** dim)], dtype=float)
    return np.linalg.det(jacobians(cell_x, corners))


class StructuredMesh:
    """N^d cells on a vertex grid of (N+1)^d points with arbitrary coordinates."""

    def __init__(self, dim: int, N: int, coords: np.ndarray, kappa: np.ndarray):
        self.dim, self.N = dim, N
        self.coords = np.asarray(coords, dtype=np.float64).reshape((N + 1) ** dim, dim)
        self.kappa = np.asarray(kappa, dtype=np.float64).reshape(N ** dim)

    @property
    def n_cells(self) -> int:
        return self.N ** self.dim

    def cell_index(self, c) -> int:
        return sum(c[k] * self.N ** k for k in range(self.dim))

    def cell_multi(self, ci: int):
        return tuple((ci // self.N ** k) % self.N for k in range(self.dim))

    def cell_vertices(self, c) -> np.ndarray:
        ids = [sum((c[k] + ((v >> k) & 1)) * (self.N + 1) ** k for k in range(self.dim))
               for v in range(2 ** self.dim)]
        return self.coords[ids]

    # --- degree-q node grid -------------------------------------------------
    def n_nodes(self, q: int) -> int:
        return (q * self.N + 1) ** self.dim

    def node_index(self, q: int, m) -> int:
        M = q * self.N + 1
        return sum(m[k] * M ** k for k in range(self.dim))

    def node_multi(self, q: int, ni: int):
        M = q * self.N + 1
        return tuple((ni // M ** k) % M for k in range(self.dim))

    def cell_nodes(self, q: int, c) -> np.ndarray:
        return np.array([self.node_index(q, [q * c[k] + a[k] for k in range(self.dim)])
                         for a in _lex(self.dim, q + 1)], dtype=np.int64)

    def cells_of_node(self, q: int, m, clip: bool = True):
        """All cells whose closure contains grid node m.  With clip=False the
        cells of the unbounded grid are listed (indices may be -1 or N), so that
        a node on the boundary of the unit square/cube also sees the cells
        beyond it."""
        per_axis = []
        for k in range(self.dim):
            i = m[k]
            if i % q == 0:
                cand = [i // q - 1, i // q]
            else:
                cand = [i // q]
            per_axis.append([c for c in cand if (0 <= c < self.N) or not clip])
        return [tuple(t) for t in itertools.product(*per_axis)]

    def free_mask(self, q: int) -> np.ndarray:
        M = q * self.N + 1
        out = np.ones(self.n_nodes(q), dtype=bool)
        for ni in range(self.n_nodes(q)):
            m = self.node_multi(q, ni)
            out[ni] = all(0 < m[k] < M - 1 for k in range(self.dim))
        return out

    def element_matrices(self, q: int):
        return [element_matrix(self.cell_vertices(self.cell_multi(ci)), self.kappa[ci], q)
                for ci in range(self.n_cells)]

    def assemble(self, q: int, Ae=None) -> sp.csr_matrix:
        """Global stiffness matrix on all (qN+1)^d nodes (no boundary conditions)."""
        Ae = self.element_matrices(q) if Ae is None else Ae
        rows, cols, vals = [], [], []
        for ci in range(self.n_cells):
            idx = self.cell_nodes(q, self.cell_multi(ci))
            rows.append(np.repeat(idx, len(idx)))
            cols.append(np.tile(idx, len(idx)))
            vals.append(Ae[ci].reshape(-1))
        n = self.n_nodes(q)
        return sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(n, n)).tocsr()

    def load_vector(self, f, q: int, n_quad: int) -> np.ndarray:
        b = np.zeros(self.n_nodes(q))
        for ci in range(self.n_cells):
            c = self.cell_multi(ci)
            b[self.cell_nodes(q, c)] += element_load(self.cell_vertices(c), f, q, n_quad)
        return b

    def node_coords(self, q: int) -> np.ndarray:
        """Physical coordinates of all degree-q nodes (the Q1 map at the
        Gauss-Lobatto reference points of the cell holding each node)."""
        gl = rules.gauss_lobatto_nodes(q)
        X = np.zeros((self.n_nodes(q), self.dim))
        for ni in range(self.n_nodes(q)):
            m = self.node_multi(q, ni)
            c = tuple(min(m[k] // q, self.N - 1) for k in range(self.dim))
            xi = np.array([[gl[m[k] - q * c[k]] for k in range(self.dim)]])
            Nq, _ = q1_shape(self.dim, xi)
            X[ni] = (Nq @ self.cell_vertices(c))[0]
        return X


def operator_with_dirichlet(A: sp.csr_matrix, free: np.ndarray) -> sp.csr_matrix:
    """A on free DoFs, identity-free zero rows on Dirichlet DoFs: (A u)_i = 0 for
    Dirichlet i, and Dirichlet values of u do not enter free rows."""
    D = sp.diags(free.astype(np.float64))
    return (D @ A @ D).tocsr()
