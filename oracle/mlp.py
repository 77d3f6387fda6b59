"""Learned Chebyshev intervals: per-patch features and a small MLP (oracle).

Test infrastructure only.  The paper has no learned component: the
Chebyshev smoother needs an interval for the spectrum of D^-1 A_{j,q} on every
patch j and p-level q, which Lanczos provides (oracle/lanczos.py); the MLP
predicts (log theta_max, log theta_min) from cheap per-patch features instead,
and the Lanczos estimate stays the reference it is checked against.

Features (16) of patch j at degree q, from its 2^d cells; for each cell c,
J_c is the Jacobian of its multilinear map at the cell centre, s_c its
singular values, d_c = det J_c, r_c = min over the cell's vertices of
det J(vertex) / d_c, k_c = log kappa_c, t_c = k_c + log d_c - 2 log(mean s_c):
   0  q / 8                         8  min_c r_c
   1  2^d / 8                       9  mean_c r_c
   2  max k - min k                10  max t - min t
   3  mean |k - mean k|            11  mean |t - mean t|
   4  max_c log(s_max / s_min)     12  log(max_c s_max / min_c s_min)
   5  mean_c log(s_max / s_min)    13  (q / 8)^2
   6  min_c log(s_max / s_min)     14  max_c |log d_c - mean log d|
   7  log(max d / min d)           15  (number of p-levels below q) / 4

Network: y = W3 relu(W2 relu(W1 x + b1) + b2) + b3, 16 -> 64 -> 64 -> 2, on
standardised inputs and targets.  Loss per sample: sum_o w_o (y_o - t_o)^2 / 2
with w_0 = asym when the theta_max output underestimates (y_0 < t_0), else 1;
averaged over the batch.  Parameter vector layout: W1 (64x16, row-major), b1,
W2 (64x64), b2, W3 (2x64), b3.
"""
from __future__ import annotations

import numpy as np

from . import fem

NF, H, NO = 16, 64, 2
SIZES = [(H, NF), (H,), (H, H), (H,), (NO, H), (NO,)]
NPARAM = sum(int(np.prod(s)) for s in SIZES)


def unpack(theta):
    out, o = [], 0
    for s in SIZES:
        n = int(np.prod(s))
        out.append(np.asarray(theta[o:o + n]).reshape(s))
        o += n
    return out


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights, zero biases (counter-free numpy stream)."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in SIZES:
        if len(s) == 2:
            lim = np.sqrt(6.0 / s[1])
            parts.append(rng.uniform(-lim, lim, size=s).ravel())
        else:
            parts.append(np.zeros(s))
    return np.concatenate(parts)


def forward(theta, X):
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3.T + b3
    return y, (X, z1, h1, z2, h2)


def forward_rounded(theta, X, rnd):
    """forward with every stored quantity passed through rnd: the weights
    and biases, the inputs and the two hidden activations (after the ReLU);
    the sums themselves in FP64.  With rnd = fem.bf16_round this is the
    BF16-inference form (BF16 operands, wide accumulation)."""
    W1, b1, W2, b2, W3, b3 = (rnd(a) for a in unpack(theta))
    h1 = rnd(np.maximum(rnd(X) @ W1.T + b1, 0.0))
    h2 = rnd(np.maximum(h1 @ W2.T + b2, 0.0))
    return h2 @ W3.T + b3


def loss(theta, X, T, asym: float = 4.0) -> float:
    y, _ = forward(theta, X)
    w = np.ones_like(y)
    w[:, 0] = np.where(y[:, 0] < T[:, 0], asym, 1.0)
    return float(np.sum(w * (y - T) ** 2) / 2.0 / len(X))


def grad(theta, X, T, asym: float = 4.0) -> np.ndarray:
    """Gradient of `loss` by the chain rule (ReLU derivative 1 where z > 0)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    w = np.ones_like(y)
    w[:, 0] = np.where(y[:, 0] < T[:, 0], asym, 1.0)
    gy = w * (y - T) / len(X)
    gW3 = gy.T @ h2
    gb3 = gy.sum(0)
    gh2 = gy @ W3
    gz2 = gh2 * (z2 > 0)
    gW2 = gz2.T @ h1
    gb2 = gz2.sum(0)
    gh1 = gz2 @ W2
    gz1 = gh1 * (z1 > 0)
    gW1 = gz1.T @ X
    gb1 = gz1.sum(0)
    return np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3)])


# ------------------------------------------------------------------ features
def _cell_quantities(X):
    dim = X.shape[1]
    J = fem.jacobians(X, np.full((1, dim), 0.5))[0]
    s = np.linalg.svd(J, compute_uv=False)
    d = np.linalg.det(J)
    r = fem.corner_dets(X).min() / d
    return s, d, r


def patch_features(mesh: fem.StructuredMesh, v, q: int, n_below: int) -> np.ndarray:
    d = mesh.dim
    cells = [tuple(v[k] - 1 + s[k] for k in range(d)) for s in fem._lex(d, 2)]
    S, D, Rr, K = [], [], [], []
    for c in cells:
        s, det, r = _cell_quantities(mesh.cell_vertices(c))
        S.append(s)
        D.append(det)
        Rr.append(r)
        K.append(np.log(mesh.kappa[mesh.cell_index(c)]))
    S, D, Rr, K = np.array(S), np.array(D), np.array(Rr), np.array(K)
    an = np.log(S[:, 0] / S[:, -1])
    t = K + np.log(D) - 2.0 * np.log(S.mean(axis=1))
    ld = np.log(D)
    f = np.array([
        q / 8.0, len(cells) / 8.0, K.max() - K.min(), np.mean(np.abs(K - K.mean())),
        an.max(), an.mean(), an.min(), np.log(D.max() / D.min()),
        Rr.min(), Rr.mean(), t.max() - t.min(), np.mean(np.abs(t - t.mean())),
        np.log(S[:, 0].max() / S[:, -1].min()), (q / 8.0) ** 2, np.max(np.abs(ld - ld.mean())), n_below / 4.0,
    ])
    return f
