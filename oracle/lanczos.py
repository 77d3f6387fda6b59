"""Per-patch eigenvalue estimates of D^-1 A_{j,q} for the Chebyshev smoother (oracle).

Test infrastructure only.  The paper's smoother is damped Jacobi; the
Chebyshev variant needs an interval [lo, hi] containing the upper part of the
spectrum of D^-1 A_{j,q} on every patch j and p-level q.  The estimate is a
k-step Lanczos run with full reorthogonalisation (two classical Gram-Schmidt
passes against all previous vectors) on the similar symmetric
matrix S = D^-1/2 A D^-1/2, followed by Sturm-sequence bisection for the
extreme eigenvalues of the Lanczos tridiagonal matrix.

Start vector: entry i is 1 + (u_i - 1/2), u_i uniform on [0,1) from the
SplitMix64 generator (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) used as a counter-based generator:
    z = seed + (counter + 1) * 0x9E3779B97F4A7C15  (mod 2^64), then the
    SplitMix64 finaliser; u = (z >> 11) * 2^-53,
with counter = (patch << 20) | (q << 16) | i.

Interval: hi = safety * theta_max, lo = max(theta_min, hi / alpha).
"""
from __future__ import annotations

import numpy as np

MASK = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(z: int) -> int:
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def uniform01(seed: int, counter: int) -> float:
    z = splitmix64((seed + (counter + 1) * GOLDEN) & MASK)
    return (z >> 11) * 2.0 ** -53


def start_vector(seed: int, patch: int, q: int, n: int) -> np.ndarray:
    return np.array([1.0 + (uniform01(seed, (patch << 20) | (q << 16) | i) - 0.5) for i in range(n)])


def lanczos(S: np.ndarray, v0: np.ndarray, k: int):
    """k Lanczos steps (or n if n < k) with full reorthogonalisation.
    Returns the tridiagonal (alpha, beta)."""
    n = S.shape[0]
    k = min(k, n)
    V = np.zeros((k, n))
    alpha, beta = [], []
    v = v0 / np.linalg.norm(v0)
    for j in range(k):
        V[j] = v
        w = S @ v
        a = v @ w
        alpha.append(a)
        for _ in range(2):                             # full reorthogonalisation, two
            w = w - V[: j + 1].T @ (V[: j + 1] @ w)    # classical Gram-Schmidt passes
        if j == k - 1:
            break
        b = np.linalg.norm(w)
        if b <= 1e-300:
            break
        beta.append(b)
        v = w / b
    return np.array(alpha), np.array(beta)


def sturm_count(alpha, beta, x) -> int:
    """Number of eigenvalues of the tridiagonal matrix smaller than x (pivots of
    the LDL^T factorisation of T - x I)."""
    cnt = 0
    dval = 1.0
    for i in range(len(alpha)):
        off = beta[i - 1] ** 2 if i > 0 else 0.0
        dval = alpha[i] - x - (off / dval if i > 0 else 0.0)
        if dval == 0.0:
            dval = -1e-300
        if dval < 0.0:
            cnt += 1
    return cnt


def extreme_eigs(alpha, beta, iters: int = 100):
    """Smallest and largest eigenvalue of the tridiagonal matrix by bisection on
    the Gershgorin interval."""
    n = len(alpha)
    b = np.concatenate([[0.0], np.abs(beta), [0.0]]) if n > 1 else np.array([0.0, 0.0])
    lo = min(alpha[i] - b[i] - b[i + 1] for i in range(n))
    hi = max(alpha[i] + b[i] + b[i + 1] for i in range(n))

    def kth(kidx):
        a, c = lo, hi
        for _ in range(iters):
            mid = 0.5 * (a + c)
            if sturm_count(alpha, beta[: n - 1], mid) > kidx:
                c = mid
            else:
                a = mid
        return 0.5 * (a + c)

    return kth(0), kth(n - 1)


def patch_bounds(A: np.ndarray, diag: np.ndarray, seed: int, patch: int, q: int,
                 k: int = 16, safety: float = 1.1, alpha_ratio: float = 10.0):
    s = 1.0 / np.sqrt(diag)
    S = s[:, None] * A * s[None, :]
    al, be = lanczos(S, start_vector(seed, patch, q, A.shape[0]), k)
    tmin, tmax = extreme_eigs(al, be)
    hi = safety * tmax
    lo = max(tmin, hi / alpha_ratio)
    return lo, hi, tmin, tmax


def lanczos_bounds_fn(seed: int = 0, k: int = 16, safety: float = 1.1, alpha_ratio: float = 10.0):
    """bounds_fn for PatchSmoother: {q: (lo, hi)} for every level q > 1."""
    def fn(patch, pid):
        out = {}
        for q in patch.levels:
            if q == 1:
                continue
            lv = patch.lv[q]
            lo, hi, _, _ = patch_bounds(lv.A, lv.diag, seed, pid, q, k, safety, alpha_ratio)
            out[q] = (lo, hi)
        return out
    return fn


def exact_bounds_fn(safety: float = 1.1, alpha_ratio: float = 10.0):
    """Same interval rule with the exact extreme eigenvalues (dense solve)."""
    def fn(patch, pid):
        out = {}
        for q in patch.levels:
            if q == 1:
                continue
            lv = patch.lv[q]
            s = 1.0 / np.sqrt(lv.diag)
            ev = np.linalg.eigvalsh(s[:, None] * lv.A * s[None, :])
            hi = safety * ev[-1]
            out[q] = (max(ev[0], hi / alpha_ratio), hi)
        return out
    return fn


def fixed_bounds_fn(lo: float, hi: float):
    def fn(patch, pid):
        return {q: (lo, hi) for q in patch.levels if q != 1}
    return fn
