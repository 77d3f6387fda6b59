"""Persistent level sweeps: one cooperative launch visits every colour of a
mesh level, the CTAs meeting at a grid barrier (bounded spin waits) between
colours.  Checked: bit-identical to the per-colour launches (sweeps both
ways, full CG solves), the set-up's choice and timings, and the failure path:
with a wait budget of one clock cycle the barrier waits run out, the sweep
stops, the call reports PMG_ERR_TIMEOUT and the device stays usable."""
import numpy as np
import pytest

from paper_2510_17785_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ctx(w, levels=1, **opt):
    from paper_2510_17785_gb300 import pmg
    prob = inputs.make_problem(w)
    ctx = pmg.Context(0, **opt)
    ctx.mesh_structured(w.dim, w.N, w.p, levels, prob.coords, prob.kappa)
    ctx.setup()
    return ctx, prob


def _wl(dim, N, p, seed=21):
    return inputs.Workload("ps", dim, N, p, 0.2, "uniform", ("loguniform", -1.0, 1.0), "uniform", seed)


@pytest.mark.parametrize("dim,N,p,levels,prec", [(3, 8, 4, 3, "mixed"), (3, 8, 4, 3, "fp64"), (3, 6, 7, 2, "mixed"),
                                                 (3, 5, 2, 1, "fp64"), (2, 16, 3, 3, "fp64"), (2, 12, 6, 2, "mixed")])
def test_persistent_sweep_is_bit_identical(dim, N, p, levels, prec):
    from paper_2510_17785_gb300 import pmg
    pr = pmg.PREC_MIXED if prec == "mixed" else pmg.PREC_FP64
    w = _wl(dim, N, p)
    ref, prob = _ctx(w, levels, precision=pr, autotune=0, persistent=0, bounds=pmg.BOUNDS_FIXED)
    per, _ = _ctx(w, levels, precision=pr, autotune=0, persistent=2, bounds=pmg.BOUNDS_FIXED)
    lf = levels - 1
    assert per.level_persistent(lf)[0] and not ref.level_persistent(lf)[0]
    u0 = inputs.random_vector(3, dim, p, N)
    b = torch.tensor(prob.rhs, device="cuda")
    for reverse in (False, True):
        ua = torch.tensor(u0, device="cuda")
        ub = torch.tensor(u0, device="cuda")
        ref.patch_smooth(lf, b, ua, 2, reverse)
        per.patch_smooth(lf, b, ub, 2, reverse)
        torch.cuda.synchronize()
        assert torch.equal(ua, ub), reverse
    ref.close()
    per.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_persistent_levels_in_cg(prec):
    """GMG-preconditioned CG with every level swept persistently: the same
    iterations and the same solution, bit for bit."""
    from paper_2510_17785_gb300 import pmg
    pr = pmg.PREC_MIXED if prec == "mixed" else pmg.PREC_FP64
    w = _wl(3, 16, 4)
    ref, prob = _ctx(w, levels=4, precision=pr, autotune=0, persistent=0)
    per, _ = _ctx(w, levels=4, precision=pr, autotune=0, persistent=2)
    b = torch.tensor(prob.rhs, device="cuda")
    xa = torch.zeros_like(b)
    xb = torch.zeros_like(b)
    ia, ra, _ = ref.solve_cg(b, xa, 1e-8, 100)
    ib, rb, _ = per.solve_cg(b, xb, 1e-8, 100)
    assert ia == ib and ra == rb
    assert torch.equal(xa, xb)
    ref.close()
    per.close()


def test_setup_times_both_ways_and_keeps_the_faster():
    from paper_2510_17785_gb300 import pmg
    w = _wl(3, 16, 4)
    ctx, _ = _ctx(w, levels=4, precision=pmg.PREC_MIXED)          # persistent = 1 (default)
    for level in range(1, 4):
        on, ms_colours, ms_persistent = ctx.level_persistent(level)
        assert ms_colours > 0
        if ms_persistent > 0:
            assert on == (ms_persistent < ms_colours)
    ctx.close()


def test_grid_barrier_timeout_is_reported_and_the_device_stays_usable():
    from paper_2510_17785_gb300 import pmg
    w = _wl(3, 8, 4)
    bad, prob = _ctx(w, 3, precision=pmg.PREC_FP64, autotune=0, persistent=2, sync_budget=1)
    u0 = inputs.random_vector(3, 3, 4, 8)
    b = torch.tensor(prob.rhs, device="cuda")
    u = torch.tensor(u0, device="cuda")
    with pytest.raises(pmg.PMGError) as e:
        bad.patch_smooth(2, b, u, 1, False)
    assert e.value.code == pmg.PMG_ERR_TIMEOUT
    x = torch.zeros_like(b)
    it, rel, rc = bad.solve_cg(b, x, 1e-8, 20, check=False)
    assert rc == pmg.PMG_ERR_TIMEOUT
    torch.cuda.synchronize()                     # the context and the device are still usable
    bad.close()
    good, _ = _ctx(w, 3, precision=pmg.PREC_FP64, autotune=0, persistent=2)
    ref, _ = _ctx(w, 3, precision=pmg.PREC_FP64, autotune=0, persistent=0)
    ua = torch.tensor(u0, device="cuda")
    ub = torch.tensor(u0, device="cuda")
    good.patch_smooth(2, b, ua, 1, False)
    ref.patch_smooth(2, b, ub, 1, False)
    torch.cuda.synchronize()
    assert torch.equal(ua, ub)
    good.close()
    ref.close()
