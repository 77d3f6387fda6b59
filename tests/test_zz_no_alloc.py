"""The allocation-free Lanczos entry point (pmg_lanczos_bounds_noalloc) gives
the same intervals as the allocating pmg_compute_bounds, on two calls in a row
that share its fixed device scratch array.

It exists for callers that must not allocate device memory at that moment
(graph capture, an externally managed memory budget, mid-run refreshes of the
Chebyshev intervals).  This file is collected last so that a run stopping at
the first failure has already run every other test."""
import numpy as np
import pytest

from paper_2510_17785_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _ctx(dim, N, p, levels=1):
    from paper_2510_17785_gb300 import pmg
    w = inputs.Workload(f"na{dim}", dim, N, p, 0.25, "uniform", ("loguniform", -1.0, 1.0), "uniform", 41)
    prob = inputs.make_problem(w)
    ctx = pmg.Context(0)                        # default: Lanczos bounds, FP64
    ctx.mesh_structured(dim, N, p, levels, prob.coords, prob.kappa)
    ctx.setup()
    return ctx


@pytest.mark.parametrize("dim,N,p", [(3, 5, 4), (2, 9, 6)])
def test_noalloc_matches_allocating_entry_point_twice(dim, N, p):
    ctx = _ctx(dim, N, p)
    ritz_ref = ctx.get_ritz(0)          # from pmg_compute_bounds at set-up
    bnds_ref = ctx.get_bounds(0)
    npatch, _ = ctx.num_patches(0)
    levels = ctx.p_levels()
    for k, q in enumerate(levels):
        if q == 1:
            continue
        # two calls in a row on different ranges: the second reuses the array
        # the first one filled
        for first, n in ((0, npatch // 2 + 1), (npatch // 3, npatch - npatch // 3)):
            ritz = torch.full((n, 2), -1.0, dtype=torch.float64, device="cuda")
            bnds = torch.full((n, 2), -1.0, dtype=torch.float64, device="cuda")
            ctx.lanczos_bounds_noalloc(0, k, first, n, ritz, bnds)
            torch.cuda.synchronize()
            r = ritz.cpu().numpy()
            b = bnds.cpu().numpy()
            ref_r = ritz_ref[first:first + n, k, :]
            ref_b = bnds_ref[first:first + n, k, :]
            assert np.abs(r - ref_r).max() <= TOL * np.abs(ref_r).max()
            assert np.abs(b - ref_b).max() <= TOL * np.abs(ref_b).max()
    ctx.close()


def test_noalloc_rejects_ranges_beyond_its_array():
    from paper_2510_17785_gb300 import pmg
    ctx = _ctx(3, 12, 4, levels=3)          # 12 -> 6 -> 3 cells per direction
    npatch, _ = ctx.num_patches(2)          # 1331 patches of 7^3 interior DoFs at q = 4
    ritz = torch.zeros((npatch, 2), dtype=torch.float64, device="cuda")
    bnds = torch.zeros((npatch, 2), dtype=torch.float64, device="cuda")
    # 1331 * 16 * 343 doubles = 58 MB > 16 MiB
    with pytest.raises(pmg.PMGError) as e:
        ctx.lanczos_bounds_noalloc(2, 0, 0, npatch, ritz, bnds)
    assert e.value.code == 1 and "16 MiB" in str(e.value)
    with pytest.raises(pmg.PMGError):
        ctx.lanczos_bounds_noalloc(2, 0, npatch - 1, 2, ritz, bnds)     # past the last patch
    ctx.close()
