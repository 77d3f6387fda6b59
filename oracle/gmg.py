"""Geometric multigrid with the patch smoother, and preconditioned CG (oracle).

Test infrastructure only.

* Mesh hierarchy M_1 c ... c M_L (Section 2): every level is the unit
  square/cube with N_l = N_c * 2^(l-1) cells per direction.  The vertices of
  a coarser level are the fine-level vertices with even indices (topological
  nestedness; the coarse cells are the multilinear images of those vertices).
  The coefficient of a coarse cell is the arithmetic (default), geometric or
  harmonic mean of its 2^d children.
* Transfers: prolongation is the embedding through the reference cells
  (a fine node's value is the coarse cell's function at the fine node's
  position in the coarse reference cell); restriction is its transpose
  (Section 2).
* V-cycle: one multiplicative patch-smoother sweep before (colours in
  increasing order) and one after (colours reversed, so that the V-cycle is
  symmetric and can precondition CG; or in the same order, the paper's
  choice, Section 4), coarse problem solved by a dense Cholesky factorisation.
* Outer solvers from u = 0, stopping when ||r_k||_2 <= rtol ||r_0||_2:
  preconditioned CG, and restarted GMRES (the paper's, Section 4), right- or
  left-preconditioned, with modified Gram-Schmidt Arnoldi and Givens rotations.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import fem, patch as pt, rules


def coarsen(mesh: fem.StructuredMesh, kappa_rule: str = "arithmetic") -> fem.StructuredMesh:
    d, N = mesh.dim, mesh.N
    assert N % 2 == 0
    Nc = N // 2
    X = mesh.coords.reshape(*([N + 1] * d), d)          # reversed axes: [z][y][x] or [y][x]
    sl = tuple([slice(None, None, 2)] * d)
    Xc = X[sl].reshape(-1, d)
    kap = mesh.kappa.reshape(*([N] * d))
    kc = np.zeros([Nc] * d)
    f, finv = {"arithmetic": (lambda k: k, lambda m: m), "geometric": (np.log, np.exp),
               "harmonic": (lambda k: 1.0 / k, lambda m: 1.0 / m)}[kappa_rule]
    for off in fem._lex(d, 2):
        idx = tuple(slice(off[d - 1 - a], None, 2) for a in range(d))   # array axes are reversed
        kc += f(kap[idx])
    kc = finv(kc / 2 ** d)
    return fem.StructuredMesh(d, Nc, Xc, kc.reshape(-1))


def hierarchy(mesh: fem.StructuredMesh, coarse_N: int, kappa_rule: str = "arithmetic"):
    out = [mesh]
    while out[-1].N > coarse_N:
        out.append(coarsen(out[-1], kappa_rule))
    assert out[-1].N == coarse_N
    return out[::-1]                     # coarsest first


def prolongation(coarse: fem.StructuredMesh, fine: fem.StructuredMesh, q: int) -> sp.csr_matrix:
    """Embedding V_coarse -> V_fine on all nodes (reference-cell embedding)."""
    d = fine.dim
    gl = rules.gauss_lobatto_nodes(q)
    rows, cols, vals = [], [], []
    for nf in range(fine.n_nodes(q)):
        m = fine.node_multi(q, nf)
        fc = [min(m[a] // q, fine.N - 1) for a in range(d)]          # a fine cell holding the node
        cc = [fc[a] // 2 for a in range(d)]                           # its parent
        xi = [(fc[a] % 2 + gl[m[a] - q * fc[a]]) / 2.0 for a in range(d)]
        lx = [rules.lagrange(gl, xi[a])[0] for a in range(d)]     # coarse basis along each axis at the node
        for loc in fem._lex(d, q + 1):
            val = 1.0
            for a in range(d):
                val *= lx[a][loc[a]]
            if abs(val) > 0.0:
                rows.append(nf)
                cols.append(coarse.node_index(q, [q * cc[a] + loc[a] for a in range(d)]))
                vals.append(val)
    return sp.coo_matrix((vals, (rows, cols)), shape=(fine.n_nodes(q), coarse.n_nodes(q))).tocsr()


class GMG:
    def __init__(self, fine: fem.StructuredMesh, p: int, coarse_N: int, smoother_args=None,
                 kappa_rule: str = "arithmetic", post_reverse: bool = True):
        self.p = p
        self.post_reverse = post_reverse
        self.meshes = hierarchy(fine, coarse_N, kappa_rule)
        self.free = [m.free_mask(p) for m in self.meshes]
        self.A = []
        for m, f in zip(self.meshes, self.free):
            self.A.append(fem.operator_with_dirichlet(m.assemble(p), f))
        self.P = []
        for l in range(1, len(self.meshes)):
            Pm = prolongation(self.meshes[l - 1], self.meshes[l], p)
            Df = sp.diags(self.free[l].astype(float))
            Dc = sp.diags(self.free[l - 1].astype(float))
            self.P.append((Df @ Pm @ Dc).tocsr())
        sa = {} if smoother_args is None else smoother_args
        self.smoothers = [None] + [pt.PatchSmoother(m, p, **sa) for m in self.meshes[1:]]
        f0 = self.free[0]
        Ac = self.A[0].toarray()[np.ix_(f0, f0)]
        self.chol = sla.cho_factor(Ac, lower=True)

    def coarse_solve(self, b):
        x = np.zeros_like(b)
        f0 = self.free[0]
        x[f0] = sla.cho_solve(self.chol, b[f0])
        return x

    def vcycle(self, b, l=None):
        l = len(self.meshes) - 1 if l is None else l
        if l == 0:
            return self.coarse_solve(b)
        S = self.smoothers[l]
        x = S.sweep(np.zeros_like(b), b, reverse=False)
        r = b - self.A[l] @ x
        e = self.vcycle(self.P[l - 1].T @ r, l - 1)
        x = x + self.P[l - 1] @ e
        x = S.sweep(x, b, reverse=self.post_reverse)
        return x


def pcg(A, b, M, rtol=1e-8, maxit=200):
    """Preconditioned CG from x = 0; returns (x, iterations, relres history)."""
    x = np.zeros_like(b)
    r = b.copy()
    r0 = np.linalg.norm(r)
    hist = [1.0]
    if r0 == 0.0:
        return x, 0, hist
    z = M(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        Ap = A @ p
        alpha = rz / (p @ Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        rel = np.linalg.norm(r) / r0
        hist.append(rel)
        if rel <= rtol:
            return x, it, hist
        z = M(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, hist


def gmres(A, b, M, rtol=1e-8, maxit=200, restart=50, left=False):
    """Restarted GMRES(restart) from x = 0 with preconditioner M.

    Right (default): x = M y with y from the Krylov space of A M; the residual
    monitored is the true one, b - A x.  Left: the Krylov space of M A, the
    residual monitored is the preconditioned one, M (b - A x).  Returns
    (x, iterations, relres history)."""
    n = len(b)
    x = np.zeros_like(b)
    r = M(b) if left else b.copy()
    r0 = np.linalg.norm(r)
    hist = [1.0]
    if r0 == 0.0:
        return x, 0, hist
    it = 0
    while it < maxit:
        beta = np.linalg.norm(r)
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        V[0] = r / beta
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        k = 0
        for j in range(restart):
            w = M(A @ V[j]) if left else A @ M(V[j])
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                           # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            hist.append(abs(g[j + 1]) / r0)
            if hist[-1] <= rtol or it >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k])
        x = x + (V[:k].T @ y if left else M(V[:k].T @ y))
        r = b - A @ x
        if left:
            r = M(r)
        if hist[-1] <= rtol:
            break
    return x, it, hist
