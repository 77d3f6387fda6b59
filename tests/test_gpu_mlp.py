"""Learned Chebyshev intervals on the GPU against the CPU oracle (oracle/mlp.py)
and against Lanczos, the method's own estimate."""
import time

import numpy as np
import pytest

from oracle import fem, mlp, patch as pt
from paper_2510_17785_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _levels(N):
    lv, n = 1, N
    while n % 2 == 0 and n // 2 >= 2:
        lv, n = lv + 1, n // 2
    return lv


def _ctx(dim, N, p, seed, perturb=0.25, kappa=("loguniform", -1.0, 1.0), **opt):
    from paper_2510_17785_gb300 import pmg
    w = inputs.Workload(f"m{dim}", dim, N, p, perturb, "uniform", kappa, "uniform", seed)
    prob = inputs.make_problem(w)
    ctx = pmg.Context(0, **opt)
    ctx.mesh_structured(dim, N, p, _levels(N), prob.coords, prob.kappa)
    ctx.setup()
    return ctx, prob


@pytest.mark.parametrize("dim,N,p", [(2, 6, 4), (3, 4, 6), (3, 3, 2)])
def test_features_match_oracle(dim, N, p):
    ctx, prob = _ctx(dim, N, p, 3)
    lf = _levels(N) - 1
    m = fem.StructuredMesh(dim, N, prob.coords, prob.kappa)
    levels = ctx.p_levels()
    npatch, _ = ctx.num_patches(lf)
    for k, q in enumerate(levels):
        X = torch.zeros((npatch, 16), dtype=torch.float32, device="cuda")
        ctx.features(lf, k, X)
        torch.cuda.synchronize()
        X = X.cpu().numpy()
        for v in pt.interior_vertices(dim, N)[:: max(1, npatch // 7)]:
            j = pt.patch_id(dim, N, v)
            ref = mlp.patch_features(m, v, q, len(levels) - 1 - k)
            assert np.allclose(X[j], ref, rtol=1e-5, atol=1e-6), (q, v)
    ctx.close()


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 16)) * 0.7 + 0.2
    T = np.stack([X[:, 2] + 0.3 * X[:, 4] ** 2, -1.0 + 0.5 * X[:, 7]], axis=1)
    return X, T


def _norm(X, T):
    return np.concatenate([X.mean(0), X.std(0) + 1e-6, T.mean(0), T.std(0) + 1e-6])


def _f32(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


def test_gradient_matches_oracle():
    from paper_2510_17785_gb300 import pmg
    X, T = _data(300, 1)
    norm = _norm(X, T)
    theta = mlp.init_params(5)
    loss, g = pmg.mlp_grad(_f32(theta), _f32(norm), _f32(X), _f32(T), asym=4.0)
    Xs = (X - norm[:16]) / norm[16:32]
    Ts = (T - norm[32:34]) / norm[34:36]
    ref_g = mlp.grad(theta, Xs, Ts, 4.0)
    ref_l = mlp.loss(theta, Xs, Ts, 4.0)
    g = g.cpu().numpy().astype(np.float64)
    assert abs(float(loss.item()) - ref_l) <= 1e-5 * ref_l
    assert np.linalg.norm(g - ref_g) <= 1e-4 * np.linalg.norm(ref_g)


@pytest.mark.parametrize("n", [1, 17, 500])
def test_forward_fp32_and_bf16_match_oracle(n):
    """FP32 inference against the oracle's forward; the tensor-core BF16
    inference against the oracle's BF16 form (forward_rounded with
    fem.bf16_round: BF16 operands, wide sums) within 1e-3 of the output scale,
    while the BF16 rounding itself moves the outputs by about 6e-3 (FP32 sums
    flip a BF16 rounding now and then: about 6e-5); ragged tails of the
    16-sample tiles."""
    from paper_2510_17785_gb300 import pmg
    X, T = _data(500, 2)
    X, T = X[:n], T[:n]
    norm = _norm(*_data(500, 2))
    theta = mlp.init_params(6)
    theta[mlp.NF * mlp.H:mlp.NF * mlp.H + mlp.H] = np.random.default_rng(1).uniform(-0.1, 0.1, mlp.H)   # b1 != 0
    theta32 = theta.astype(np.float32).astype(np.float64)
    Xs = (X.astype(np.float32) - norm[:16].astype(np.float32)) / norm[16:32].astype(np.float32)
    y, _ = mlp.forward(theta32, Xs.astype(np.float64))
    yb = mlp.forward_rounded(theta32, Xs.astype(np.float64), fem.bf16_round)
    ref = y * norm[34:36] + norm[32:34]
    ref_bf16 = yb * norm[34:36] + norm[32:34]
    y32 = pmg.mlp_predict(_f32(theta), _f32(norm), _f32(X), bf16=False).cpu().numpy()
    y16 = pmg.mlp_predict(_f32(theta), _f32(norm), _f32(X), bf16=True).cpu().numpy()
    scale = np.abs(ref).max()
    assert y16.shape == (n, 2)
    assert np.abs(y32 - ref).max() <= 1e-5 * scale
    assert np.abs(y16 - ref_bf16).max() <= 1e-3 * scale
    assert np.abs(y16 - ref).max() <= 3e-2 * scale


def test_training_reduces_the_loss():
    from paper_2510_17785_gb300 import pmg
    X, T = _data(4096, 3)
    norm = _norm(X, T)
    params = _f32(mlp.init_params(7))
    hist = pmg.mlp_train(params, _f32(norm), _f32(X), _f32(T), epochs=60, batch=512, lr=3e-3)
    assert hist[-1] < 0.1 * hist[0]


def test_learned_bounds_against_lanczos():
    """Train on Lanczos estimates of several problems, predict the intervals of
    a held-out one: the CG iteration count stays within one of the Lanczos
    intervals' and the intervals cost less to compute."""
    from paper_2510_17785_gb300 import pmg
    train = []
    for seed, (dim, N, p) in enumerate([(3, 8, 4), (3, 8, 2), (3, 6, 3), (3, 4, 6), (3, 8, 4), (3, 6, 5)]):
        ctx, _ = _ctx(dim, N, p, 100 + seed, perturb=0.1 + 0.03 * seed, kappa=("loguniform", -1.5, 1.5))
        train.append(ctx)
    data = [pmg.mlp_training_data(c) for c in train]      # features and log Lanczos estimates, on the device
    for c in train:
        c.close()
    X, T = torch.cat([x for x, _ in data]), torch.cat([t for _, t in data])
    norm = pmg.mlp_norm(X, T)
    params = _f32(pmg.mlp_init(11))
    hist = pmg.mlp_train(params, _f32(norm), X, T, epochs=150, batch=256, lr=2e-3, asym=4.0)
    assert hist[-1] < 0.2 * hist[0]
    # held-out problem, GMG-preconditioned CG with both interval sources
    w = inputs.Workload("held", 3, 8, 4, 0.2, "uniform", ("loguniform", -1.5, 1.5), "uniform", 999)
    prob = inputs.make_problem(w)
    ctxL = pmg.Context(0)
    ctxL.mesh_structured(3, 8, 4, 3, prob.coords, prob.kappa)
    ctxL.setup()
    ctxM = pmg.Context(0, bounds=pmg.BOUNDS_FIXED)
    ctxM.mesh_structured(3, 8, 4, 3, prob.coords, prob.kappa)
    ctxM.setup()
    ctxM.set_mlp(params.cpu().numpy(), norm.astype(np.float32))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctxM.compute_bounds(pmg.BOUNDS_MLP)
    t_mlp = time.perf_counter() - t0
    t0 = time.perf_counter()
    ctxL.compute_bounds(pmg.BOUNDS_LANCZOS)
    t_lan = time.perf_counter() - t0
    b = torch.tensor(prob.rhs, device="cuda")
    xL, xM = torch.zeros_like(b), torch.zeros_like(b)
    itL, relL, _ = ctxL.solve_cg(b, xL, 1e-8, 100)
    itM, relM, _ = ctxM.solve_cg(b, xM, 1e-8, 100)
    assert relL <= 1e-8 and relM <= 1e-8
    assert itM <= itL + 1, (itM, itL)
    # the predicted upper ends cover the Lanczos estimates on most patches
    bl, bm = ctxL.get_bounds(2), ctxM.get_bounds(2)
    covered = np.mean(bm[:, 0, 1] >= bl[:, 0, 1] / 1.1)
    assert covered > 0.9
    assert t_mlp < t_lan
    ctxL.close()
    ctxM.close()


def test_library_training_helpers():
    """pmg_mlp_init: deterministic, weights within +-sqrt(6 / fan_in), zero
    biases; pmg_mlp_targets: (log theta_max, log theta_min) of the context's
    Lanczos estimates; pmg_mlp_norm: column means and population standard
    deviations (+1e-6), checked against numpy."""
    from paper_2510_17785_gb300 import pmg
    a, b = pmg.mlp_init(3), pmg.mlp_init(3)
    assert np.array_equal(a, b) and not np.array_equal(a, pmg.mlp_init(4))
    o = 0
    for rows, cols in ((64, 16), (64, 64), (2, 64)):
        W = a[o:o + rows * cols]
        assert np.abs(W).max() <= np.sqrt(6.0 / cols) and np.abs(W).max() > 0.9 * np.sqrt(6.0 / cols)
        assert abs(W.mean()) < 0.1 * np.sqrt(6.0 / cols)
        o += rows * cols
        assert np.all(a[o:o + rows] == 0)
        o += rows
    assert o == pmg.MLP_NPARAM
    ctx, _ = _ctx(3, 4, 4, 8)
    X, T = pmg.mlp_training_data(ctx)
    ritz = np.concatenate([ctx.get_ritz(lv)[:, k, :] for lv in range(ctx.n_levels)
                           for k, q in enumerate(ctx.p_levels()) if q > 1])
    assert np.allclose(T.cpu().numpy(), np.log(ritz[:, ::-1]), rtol=1e-6, atol=1e-6)
    norm = pmg.mlp_norm(X, T)
    Xn, Tn = X.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64)
    ref = np.concatenate([Xn.mean(0), Xn.std(0) + 1e-6, Tn.mean(0), Tn.std(0) + 1e-6])
    assert np.allclose(norm, ref, rtol=1e-5, atol=1e-6)
    ctx.close()


def test_network_save_and_load_round_trip(tmp_path):
    """A network written by pmg_mlp_save and read by pmg_mlp_load gives the
    same learned intervals; a file of another kind is rejected."""
    from paper_2510_17785_gb300 import pmg
    X, T = _data(256, 9)
    norm = _norm(X, T).astype(np.float32)
    params = pmg.mlp_init(21)
    c1, _ = _ctx(3, 4, 4, 12, bounds=pmg.BOUNDS_FIXED)
    c1.set_mlp(params, norm)
    c1.compute_bounds(pmg.BOUNDS_MLP)
    path = str(tmp_path / "net.bin")
    c1.mlp_save(path)
    c2, _ = _ctx(3, 4, 4, 12, bounds=pmg.BOUNDS_FIXED)
    c2.mlp_load(path)
    c2.compute_bounds(pmg.BOUNDS_MLP)
    for lv in range(c1.n_levels):
        assert np.array_equal(c1.get_bounds(lv), c2.get_bounds(lv))
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"not a network file")
    with pytest.raises(pmg.PMGError):
        c2.mlp_load(str(bad))
    c1.close()
    c2.close()
