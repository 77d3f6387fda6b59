"""BF16 geometry in the patch kernels (options.geometry_bf16 = 1, mixed
precision): the kernels load the geometry tensors G as packed BF16 pairs for
their matrix-free applies (the level operators and Evaluate); the level
diagonals, the dense small levels and the p = 1 scalar are set-up data
computed from exact G.  Checked against the oracle built the same way
(element matrices through G rounded by fem.bf16_round for the matrix-free
levels): one sweep agrees within 5e-5, while the oracle with exact G is 2e-4
or more away (so the rounding is in effect and applied to the right
components); every 3D launch shape gives the same bits (the shapes that stage
G in shared memory read an FP32 copy of the rounded values); GMG-
preconditioned CG within one iteration of FP32 geometry."""
import dataclasses

import numpy as np
import pytest

from oracle import fem, lanczos as lz, patch as pt
from paper_2510_17785_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIX_LO, FIX_HI = 0.25, 2.2


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _wl(dim, N, p, seed=5):
    return inputs.Workload("gb", dim, N, p, 0.2, "uniform", ("loguniform", -1.0, 1.0), "uniform", seed)


def _ctx(w, levels, **opt):
    from paper_2510_17785_gb300 import pmg
    prob = inputs.make_problem(w)
    ctx = pmg.Context(0, precision=pmg.PREC_MIXED, **opt)
    ctx.mesh_structured(w.dim, w.N, w.p, levels, prob.coords, prob.kappa)
    ctx.setup()
    return ctx, prob


def _sweep(ctx, prob, u0, level=0):
    u = torch.tensor(u0, device="cuda")
    ctx.patch_smooth(level, torch.tensor(prob.rhs, device="cuda"), u, 1, False)
    torch.cuda.synchronize()
    return u.cpu().numpy()


def _bf16_element(cx, kappa, q):
    return fem.element_matrix_G(cx, kappa, q, g_round=fem.bf16_round)


def _dense_level(dim, q):
    return q > 1 and (2 * q - 1) ** dim <= 64


def _bf16_smoother(m, p, bfn):
    """The oracle smoother with BF16 geometry where the kernels read it: the
    matrix-free level operators; diagonals, dense levels and the p = 1 scalar
    from exact G."""
    S = pt.PatchSmoother(m, p, bounds_fn=bfn, element_fn=_bf16_element)
    E = pt.PatchSmoother(m, p, bounds_fn=bfn)
    for v in S.vertices:
        Pb, Pe = S.patch(v), E.patch(v)
        for q in Pb.levels:
            if q == 1 or _dense_level(m.dim, q):
                Pb.lv[q] = Pe.lv[q]
            else:
                Pb.lv[q] = dataclasses.replace(Pb.lv[q], diag=Pe.lv[q].diag)
    return S


@pytest.mark.parametrize("dim,N,p", [(3, 4, 4), (3, 4, 3), (2, 6, 5)])
def test_sweep_matches_the_oracle_with_bf16_geometry(dim, N, p):
    from paper_2510_17785_gb300 import pmg
    w = _wl(dim, N, p)
    ctx, prob = _ctx(w, 1, geometry_bf16=1, bounds=pmg.BOUNDS_FIXED, fixed_lo=FIX_LO, fixed_hi=FIX_HI)
    u0 = inputs.random_vector(8, dim, p, N)
    got = _sweep(ctx, prob, u0)
    ctx.close()
    m = fem.StructuredMesh(dim, N, prob.coords, prob.kappa)
    bfn = lz.fixed_bounds_fn(FIX_LO, FIX_HI)
    ref_bf16 = _bf16_smoother(m, p, bfn).sweep(u0, prob.rhs)
    ref_exact = pt.PatchSmoother(m, p, bounds_fn=bfn).sweep(u0, prob.rhs)
    assert relerr(ref_bf16, ref_exact) > 2e-4               # the rounding is visible at this size
    assert relerr(got, ref_bf16) < 5e-5
    assert relerr(got, ref_exact) > 2e-4


@pytest.mark.parametrize("dim,N,p,variants", [(3, 8, 4, (0, 3, 4, 6, 10)), (3, 8, 3, (0, 3, 4, 6, 8))])
def test_every_launch_shape_gives_the_same_bits(dim, N, p, variants):
    from paper_2510_17785_gb300 import pmg
    w = _wl(dim, N, p, seed=7)
    u0 = inputs.random_vector(3, dim, p, N)
    outs = []
    for v in variants:
        ctx, prob = _ctx(w, 2, geometry_bf16=1, autotune=0, variant=v, persistent=0, dense_local=0,
                         bounds=pmg.BOUNDS_FIXED)
        assert ctx.tuning_level(1)[0] == v                  # the finest of the two mesh levels
        outs.append(_sweep(ctx, prob, u0, level=1))
        ctx.close()
    for v, o in zip(variants[1:], outs[1:]):
        assert np.array_equal(o, outs[0]), v


def test_cg_with_bf16_geometry_within_one_iteration():
    w = _wl(3, 16, 4, seed=9)
    ref, prob = _ctx(w, 4)
    bf, _ = _ctx(w, 4, geometry_bf16=1)
    b = torch.tensor(prob.rhs, device="cuda")
    xa, xb = torch.zeros_like(b), torch.zeros_like(b)
    ia, ra, _ = ref.solve_cg(b, xa, 1e-8, 100)
    ib, rb, _ = bf.solve_cg(b, xb, 1e-8, 100)
    assert ra <= 1e-8 and rb <= 1e-8
    assert ib <= ia + 1, (ia, ib)
    assert relerr(xb.cpu().numpy(), xa.cpu().numpy()) < 1e-6
    ref.close()
    bf.close()
