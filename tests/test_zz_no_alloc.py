"""The allocation-free Lanczos entry point (pmg_lanczos_bounds_noalloc) gives
the same intervals as the allocating pmg_compute_bounds, on two calls in a row
that share its fixed device scratch array.

It exists for callers that must not allocate device memory at that moment:
code inside a framework that owns the device memory through its own
allocator, or a solver that refreshes its Chebyshev intervals mid-run and must
not stall on cudaMalloc/cudaFree.  This file is collected last so that a run
stopping at the first failure has already run every other test."""
import numpy as np
import pytest

from paper_2510_17785_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def _ctx(dim, N, p, levels=1, **kw):
    from paper_2510_17785_gb300 import pmg
    w = inputs.Workload(f"na{dim}", dim, N, p, 0.25, "uniform", ("loguniform", -1.0, 1.0), "uniform", 41)
    prob = inputs.make_problem(w)
    ctx = pmg.Context(0, **kw)                  # default: Lanczos bounds, FP64
    ctx.mesh_structured(dim, N, p, levels, prob.coords, prob.kappa)
    ctx.setup()
    return ctx


def _check_twice(ctx, level=0):
    ritz_ref = ctx.get_ritz(level)          # from pmg_compute_bounds at set-up
    bnds_ref = ctx.get_bounds(level)
    npatch, _ = ctx.num_patches(level)
    for k, q in enumerate(ctx.p_levels()):
        if q == 1:
            continue
        # two calls in a row on different ranges: the second reuses the array
        # the first one filled
        for first, n in ((0, npatch // 2 + 1), (npatch // 3, npatch - npatch // 3)):
            ritz = torch.full((n, 2), -1.0, dtype=torch.float64, device="cuda")
            bnds = torch.full((n, 2), -1.0, dtype=torch.float64, device="cuda")
            ctx.lanczos_bounds_noalloc(level, k, first, n, ritz, bnds)
            torch.cuda.synchronize()
            r = ritz.cpu().numpy()
            b = bnds.cpu().numpy()
            ref_r = ritz_ref[first:first + n, k, :]
            ref_b = bnds_ref[first:first + n, k, :]
            assert np.abs(r - ref_r).max() <= TOL * np.abs(ref_r).max()
            assert np.abs(b - ref_b).max() <= TOL * np.abs(ref_b).max()


@pytest.mark.parametrize("dim,N,p", [(3, 5, 4), (2, 9, 6)])
def test_noalloc_matches_allocating_entry_point_twice(dim, N, p):
    ctx = _ctx(dim, N, p)
    _check_twice(ctx)
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_degree7_uses_the_fp32_operator_like_the_allocating_path(precision):
    """3D degree 7: the FP64 Lanczos working set exceeds shared memory, so both
    entry points apply the operator in FP32 with FP64 Lanczos vectors."""
    from paper_2510_17785_gb300 import pmg
    prec = pmg.PREC_FP64 if precision == "fp64" else pmg.PREC_MIXED
    ctx = _ctx(3, 3, 7, precision=prec)
    _check_twice(ctx)
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


def test_noalloc_wrapper_rejects_outputs_it_cannot_fill():
    """The C side receives bare pointers; the binding checks type, size and
    device of the output tensors before calling it."""
    ctx = _ctx(2, 5, 4)
    n = 4
    good = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(TypeError):
        ctx.lanczos_bounds_noalloc(0, 0, 0, n, torch.zeros((n, 2), dtype=torch.float32, device="cuda"), good)
    with pytest.raises(ValueError):
        ctx.lanczos_bounds_noalloc(0, 0, 0, n, good, torch.zeros((n, 1), dtype=torch.float64, device="cuda"))
    with pytest.raises(TypeError):
        ctx.lanczos_bounds_noalloc(0, 0, 0, n, torch.zeros((n, 2), dtype=torch.float64), good)
    ctx.lanczos_bounds_noalloc(0, 0, 0, n, good, torch.zeros((n, 2), dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert torch.cuda.current_device() == 0
    ctx.close()
