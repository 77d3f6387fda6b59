"""Tabulated local solves: the local solve of a patch (N_MG V-cycles from zero
with fixed Chebyshev intervals) is a fixed linear map; the set-up tabulates it
by applying it to unit vectors, and a sweep then does one dense
matrix-vector product per patch.  Checked against the matrix-free V-cycles
and the oracle: FP64 to 1e-12, FP32 within FP32 rounding, CG iterations and
solutions; the local-solve entry point keeps running the V-cycles."""
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


def _ctx(w, levels, **opt):
    from paper_2510_17785_gb300 import pmg
    prob = inputs.make_problem(w)
    ctx = pmg.Context(0, **opt)
    ctx.mesh_structured(w.dim, w.N, w.p, levels, prob.coords, prob.kappa)
    ctx.setup()
    return ctx, prob


def _wl(dim, N, p, seed=31):
    return inputs.Workload("dl", dim, N, p, 0.2, "uniform", ("loguniform", -1.0, 1.0), "uniform", seed)


@pytest.mark.parametrize("dim,N,p,kind", [(3, 4, 4, "chebyshev"), (3, 4, 3, "jacobi"), (2, 6, 5, "chebyshev"),
                                          (3, 3, 2, "chebyshev"), (2, 5, 8, "jacobi")])
def test_tabulated_sweep_matches_the_oracle_fp64(dim, N, p, kind):
    from paper_2510_17785_gb300 import pmg
    sm = pmg.SMOOTHER_JACOBI if kind == "jacobi" else pmg.SMOOTHER_CHEBYSHEV
    w = _wl(dim, N, p)
    ctx, prob = _ctx(w, 1, precision=pmg.PREC_FP64, autotune=0, dense_local=2, smoother=sm,
                     bounds=pmg.BOUNDS_FIXED, fixed_lo=FIX_LO, fixed_hi=FIX_HI)
    assert ctx.level_dense_local(0)[0]
    u0 = inputs.random_vector(8, dim, p, N)
    u = torch.tensor(u0, device="cuda")
    ctx.patch_smooth(0, torch.tensor(prob.rhs, device="cuda"), u, 1, False)
    torch.cuda.synchronize()
    m = fem.StructuredMesh(dim, N, prob.coords, prob.kappa)
    S = pt.PatchSmoother(m, p, sm=pt.Smoother(kind=kind), bounds_fn=lz.fixed_bounds_fn(FIX_LO, FIX_HI))
    assert relerr(u.cpu().numpy(), S.sweep(u0, prob.rhs)) < 1e-12
    ctx.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_tabulated_levels_in_cg(prec):
    from paper_2510_17785_gb300 import pmg
    pr = pmg.PREC_MIXED if prec == "mixed" else pmg.PREC_FP64
    w = _wl(3, 16, 4)
    ref, prob = _ctx(w, 4, precision=pr, autotune=0, dense_local=0)
    tab, _ = _ctx(w, 4, precision=pr, autotune=0, dense_local=2)
    # a level is tabulated when its table fits 2 GiB: the 16^3 level's is 1.6 GB in FP32, 3.2 GB in FP64
    assert tab.level_dense_local(1)[0] and tab.level_dense_local(2)[0]
    assert tab.level_dense_local(3)[0] == (prec == "mixed")
    b = torch.tensor(prob.rhs, device="cuda")
    u0 = torch.tensor(inputs.random_vector(3, 3, 4, 16), device="cuda")
    ua, ub = u0.clone(), u0.clone()
    ref.patch_smooth(3, b, ua, 1, True)
    tab.patch_smooth(3, b, ub, 1, True)
    torch.cuda.synchronize()
    assert relerr(ub.cpu().numpy(), ua.cpu().numpy()) < (2e-5 if prec == "mixed" else 1e-12)
    xa, xb = torch.zeros_like(b), torch.zeros_like(b)
    ia, ra, _ = ref.solve_cg(b, xa, 1e-8, 100)
    ib, rb, _ = tab.solve_cg(b, xb, 1e-8, 100)
    assert rb <= 1e-8 and abs(ia - ib) <= (1 if prec == "mixed" else 0)
    assert relerr(xb.cpu().numpy(), xa.cpu().numpy()) < 1e-7
    # the local-solve entry point still runs the V-cycles: identical bits in both contexts
    ni = 7 ** 3
    ids = torch.tensor(inputs.sample_patches(5, 15 ** 3, 6), device="cuda")
    r = torch.tensor(np.random.default_rng(2).uniform(-1, 1, 6 * ni), device="cuda")
    da, db = torch.zeros_like(r), torch.zeros_like(r)
    ref.local_vcycle(3, ids, r, da)
    tab.local_vcycle(3, ids, r, db)
    torch.cuda.synchronize()
    assert torch.equal(da, db)
    ref.close()
    tab.close()


def test_setup_times_both_forms():
    from paper_2510_17785_gb300 import pmg
    w = _wl(3, 16, 4)
    ctx, _ = _ctx(w, 4, precision=pmg.PREC_MIXED)                # dense_local = 1 (default)
    for level in range(1, 4):
        on, ms_mf, ms_tab = ctx.level_dense_local(level)
        assert ms_mf > 0 and ms_tab > 0
        assert on == (ms_tab < ms_mf)
    ctx.close()
