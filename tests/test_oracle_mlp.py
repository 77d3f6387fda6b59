"""Pins of the oracle's MLP and patch features (no GPU)."""
import numpy as np
import pytest

from oracle import fem, mlp
from paper_2510_17785_gb300 import inputs


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init_params(1) + 0.01 * rng.standard_normal(mlp.NPARAM)
    X = rng.standard_normal((37, mlp.NF))
    T = rng.standard_normal((37, mlp.NO))
    g = mlp.grad(theta, X, T)
    eps = 1e-6
    fd = np.zeros_like(theta)
    for i in range(mlp.NPARAM):
        e = np.zeros_like(theta)
        e[i] = eps
        fd[i] = (mlp.loss(theta + e, X, T) - mlp.loss(theta - e, X, T)) / (2 * eps)
    assert np.linalg.norm(g - fd) <= 1e-6 * np.linalg.norm(fd)


def test_asymmetric_weight_only_on_underestimated_theta_max():
    theta = mlp.init_params(2)
    X = np.random.default_rng(3).standard_normal((5, mlp.NF))
    y, _ = mlp.forward(theta, X)
    over = y.copy()
    over[:, 0] -= 0.5          # prediction above the target on output 0
    under = y.copy()
    under[:, 0] += 0.5         # prediction below the target on output 0
    assert mlp.loss(theta, X, over, asym=4.0) == pytest.approx(5 * 0.25 / 2 / 5)
    assert mlp.loss(theta, X, under, asym=4.0) == pytest.approx(4 * 5 * 0.25 / 2 / 5)


def test_parameter_layout():
    assert mlp.NPARAM == 16 * 64 + 64 + 64 * 64 + 64 + 2 * 64 + 2
    theta = np.arange(mlp.NPARAM, dtype=float)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(theta)
    assert W1[1, 0] == 16 and b1[0] == 1024 and W3.shape == (2, 64) and b3[-1] == mlp.NPARAM - 1


def _mesh(dim, N, perturb, seed, kappa=("const", 1.0)):
    w = inputs.Workload("t", dim, N, 1, perturb, "uniform", kappa, "uniform", seed)
    pr = inputs.make_problem(w)
    return fem.StructuredMesh(dim, N, pr.coords, pr.kappa)


@pytest.mark.parametrize("dim", [2, 3])
def test_features_of_a_cartesian_patch(dim):
    m = _mesh(dim, 4, 0.0, 0)
    f = mlp.patch_features(m, (2,) * dim, 4, 2)
    expect = np.zeros(16)
    expect[0], expect[1], expect[8], expect[9], expect[13], expect[15] = 0.5, 2 ** dim / 8, 1, 1, 0.25, 0.5
    assert np.allclose(f, expect, atol=1e-14)


def test_features_invariant_under_rigid_motion_and_scaling():
    m = _mesh(3, 3, 0.2, 7, ("loguniform", -2, 2))
    f = mlp.patch_features(m, (1, 2, 1), 3, 1)
    th = 0.9
    R = np.array([[1, 0, 0], [0, np.cos(th), -np.sin(th)], [0, np.sin(th), np.cos(th)]])
    m2 = fem.StructuredMesh(3, 3, 2.5 * m.coords @ R.T + 1.0, m.kappa)
    assert np.allclose(mlp.patch_features(m2, (1, 2, 1), 3, 1), f, atol=1e-12)
    m3 = fem.StructuredMesh(3, 3, m.coords, 10.0 * m.kappa)        # kappa enters through ratios only
    assert np.allclose(mlp.patch_features(m3, (1, 2, 1), 3, 1), f, atol=1e-12)


def test_rounded_forward_reduces_to_forward_and_rounds_what_it_says():
    """forward_rounded with the identity is forward; with BF16 rounding every
    stored quantity (weights, biases, inputs, hidden activations) is a BF16
    number, checked by recomputing it step by step."""
    from oracle import fem
    rng = np.random.default_rng(3)
    theta = mlp.init_params(4)
    theta[mlp.NF * mlp.H:mlp.NF * mlp.H + mlp.H] = rng.uniform(-0.2, 0.2, mlp.H)
    X = rng.standard_normal((40, mlp.NF))
    y, _ = mlp.forward(theta, X)
    assert np.array_equal(mlp.forward_rounded(theta, X, lambda a: np.asarray(a, dtype=float)), y)
    r = fem.bf16_round
    W1, b1, W2, b2, W3, b3 = (r(a) for a in mlp.unpack(theta))
    h1 = r(np.maximum(r(X) @ W1.T + b1, 0.0))
    for a in (W1, b1, W2, b2, W3, b3, h1):
        assert np.array_equal(r(a), a)
    h2 = r(np.maximum(h1 @ W2.T + b2, 0.0))
    assert np.array_equal(mlp.forward_rounded(theta, X, r), h2 @ W3.T + b3)
    d = np.abs(mlp.forward_rounded(theta, X, r) - y).max() / np.abs(y).max()
    assert 1e-4 < d < 5e-2
