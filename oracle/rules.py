"""1D quadrature rules and Lagrange bases on [0, 1] (oracle; test infrastructure only).

The finite element space uses tensor-product Lagrange polynomials on
Gauss-Lobatto support points (the Q_p space V_l of Section 2); the integrals of
the bilinear form (eq. bilinear-form) use the (q+1)-point Gauss rule per
direction, which is exact for constant coefficients on affine cells.

Both rules are computed by the Golub-Welsch method: the nodes are eigenvalues
of the symmetric Jacobi matrix of the orthogonal polynomial family, the
weights come from the first components of the eigenvectors.
"""
from __future__ import annotations

import numpy as np


def gauss(n: int):
    """n-point Gauss-Legendre rule on [0,1]: (nodes, weights), weights sum to 1.

    Legendre three-term recurrence: monic beta_k = k^2 / (4k^2 - 1)."""
    if n == 1:
        return np.array([0.5]), np.array([1.0])
    k = np.arange(1, n, dtype=np.float64)
    off = k / np.sqrt(4.0 * k * k - 1.0)
    J = np.diag(off, 1) + np.diag(off, -1)
    lam, V = np.linalg.eigh(J)
    w = V[0, :] ** 2          # mu_0 = 2 on [-1,1]; mapped to [0,1] the weights are v0^2 * 2 / 2
    x = 0.5 * (lam + 1.0)
    order = np.argsort(x)
    return x[order], w[order]


def gauss_lobatto_nodes(q: int) -> np.ndarray:
    """The q+1 Gauss-Lobatto points on [0,1] (q >= 1).

    The interior points are the roots of P'_q, i.e. of the Jacobi polynomial
    P^{(1,1)}_{q-1}; they are the eigenvalues of that family's Jacobi matrix,
    with monic beta_k = k (k + 2) / ((2k + 1)(2k + 3))."""
    if q < 1:
        raise ValueError("degree must be >= 1")
    m = q - 1
    if m == 0:
        inner = np.zeros(0)
    elif m == 1:
        inner = np.array([0.0])
    else:
        k = np.arange(1, m, dtype=np.float64)
        off = np.sqrt(k * (k + 2.0) / ((2.0 * k + 1.0) * (2.0 * k + 3.0)))
        J = np.diag(off, 1) + np.diag(off, -1)
        inner = np.sort(np.linalg.eigvalsh(J))
    t = np.concatenate([[-1.0], inner, [1.0]])
    return 0.5 * (t + 1.0)


def lagrange(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """L[i, j] = l_j(x_i), the Lagrange polynomial of node j evaluated at x_i
    (plain product formula)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    L = np.ones((len(x), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                L[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return L


def lagrange_deriv(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """D[i, j] = l_j'(x_i): derivative of the product formula (sum over the
    factor that is differentiated)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    D = np.zeros((len(x), n))
    for j in range(n):
        for k in range(n):
            if k == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[k]))
            for m in range(n):
                if m != j and m != k:
                    term *= (x - nodes[m]) / (nodes[j] - nodes[m])
            D[:, j] += term
    return D
