"""GPU (CUDA path through the C ABI) against the CPU oracle, element by element.

FP64 results must agree to 1e-12 relative (max-norm error over max-norm of the
oracle result); integer structures bit-exactly.  Inputs are seeded synthetic
meshes of the paper's kind (unit square/cube, perturbed interior vertices,
per-cell coefficients).
"""
import numpy as np
import pytest

from oracle import fem, gmg, lanczos as lz, patch as pt
from paper_2510_17785_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
FIX_LO, FIX_HI = 0.25, 2.2


def relerr(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def wl(dim, N, p, perturb=0.25, kappa=("loguniform", -1.0, 1.0), seed=5):
    return inputs.Workload(f"t{dim}d_n{N}_q{p}", dim, N, p, perturb, "uniform", kappa, "uniform", seed)


def gpu_ctx(w, n_levels=1, **opt):
    from paper_2510_17785_gb300 import pmg
    prob = inputs.make_problem(w)
    ctx = pmg.Context(0, **opt)
    ctx.mesh_structured(w.dim, w.N, w.p, n_levels, prob.coords, prob.kappa)
    ctx.setup()
    return ctx, prob


def omesh(prob):
    w = prob.workload
    return fem.StructuredMesh(w.dim, w.N, prob.coords, prob.kappa)


def dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def fixed(**kw):
    from paper_2510_17785_gb300 import pmg
    return dict(bounds=pmg.BOUNDS_FIXED, fixed_lo=FIX_LO, fixed_hi=FIX_HI, **kw)


# ------------------------------------------------------------------ set-up
@pytest.mark.parametrize("dim,N,p", [(2, 6, 4), (2, 4, 7), (3, 3, 4), (3, 2, 6)])
def test_inverse_level_diagonals(dim, N, p):
    w = wl(dim, N, p)
    ctx, prob = gpu_ctx(w, **fixed())
    m = omesh(prob)
    for k, q in enumerate(ctx.p_levels()):
        A = m.assemble(q)
        free = m.free_mask(q)
        ref = np.where(free, 1.0 / A.diagonal(), 0.0)
        out = torch.zeros(m.n_nodes(q), dtype=torch.float64, device="cuda")
        ctx.get_inv_diag(0, k, out)
        torch.cuda.synchronize()
        assert relerr(out.cpu().numpy(), ref) < TOL, (q,)
    ctx.close()


def test_colours_and_patch_map_bit_exact():
    for dim, N in ((2, 7), (3, 5)):
        w = wl(dim, N, 2)
        ctx, prob = gpu_ctx(w, **fixed())
        m = omesh(prob)
        verts = pt.interior_vertices(dim, N)
        col = ctx.get_colours(0)
        pmap = ctx.get_patch_map(0)
        assert len(col) == len(verts) == (N - 1) ** dim
        for v in verts:
            j = pt.patch_id(dim, N, v)
            assert col[j] == pt.colour_of(v)
            cells = [m.cell_index(tuple(v[k] - 1 + s[k] for k in range(dim))) for s in fem._lex(dim, 2)]
            assert list(pmap[j, :-1]) == cells
            assert pmap[j, -1] == m.node_index(2, [2 * (v[k] - 1) for k in range(dim)])
        ctx.close()


# ------------------------------------------------------------------ operator
@pytest.mark.parametrize("dim,N,p", [(2, 5, 1), (2, 6, 4), (2, 3, 8), (3, 3, 2), (3, 3, 4), (3, 2, 6)])
def test_global_apply(dim, N, p):
    w = wl(dim, N, p)
    ctx, prob = gpu_ctx(w, **fixed())
    m = omesh(prob)
    A = fem.operator_with_dirichlet(m.assemble(p), m.free_mask(p))
    u = inputs.random_vector(3, dim, p, N, free_only=False)
    out = torch.zeros(len(u), dtype=torch.float64, device="cuda")
    ctx.apply(0, dev(u), out)
    torch.cuda.synchronize()
    ref = A @ (u * m.free_mask(p))
    assert relerr(out.cpu().numpy(), ref) < TOL
    ctx.close()


@pytest.mark.parametrize("dim,N,p", [(2, 6, 3), (3, 3, 2)])
def test_manufactured_load_vector(dim, N, p):
    w = wl(dim, N, p)
    ctx, prob = gpu_ctx(w, **fixed())
    m = omesh(prob)
    f = lambda X: dim * np.pi ** 2 * np.prod(np.sin(np.pi * X), axis=1)
    ref = m.load_vector(f, p, p + 2) * m.free_mask(p)
    out = torch.zeros(m.n_nodes(p), dtype=torch.float64, device="cuda")
    ctx.rhs_manufactured(out)
    torch.cuda.synchronize()
    assert relerr(out.cpu().numpy(), ref) < TOL
    ctx.close()


# ------------------------------------------------------------- local solver
@pytest.mark.parametrize("dim,N,p,kind,ncyc", [
    (2, 6, 4, "chebyshev", 1), (2, 6, 4, "jacobi", 1), (2, 5, 7, "chebyshev", 2), (2, 4, 2, "chebyshev", 1),
    (2, 4, 1, "chebyshev", 1), (3, 4, 4, "chebyshev", 1), (3, 3, 3, "jacobi", 2), (3, 3, 2, "chebyshev", 3),
    (3, 2, 6, "chebyshev", 1), (3, 2, 5, "jacobi", 1),
    (2, 6, 4, "fdm", 1), (2, 4, 7, "fdm", 2), (3, 3, 4, "fdm", 1), (3, 2, 2, "fdm", 2), (3, 2, 6, "fdm", 1),
    (3, 2, 7, "chebyshev", 1), (3, 2, 7, "fdm", 1)])
def test_local_vcycle(dim, N, p, kind, ncyc):
    from paper_2510_17785_gb300 import pmg
    sm = {"jacobi": pmg.SMOOTHER_JACOBI, "fdm": pmg.SMOOTHER_CARTESIAN}.get(kind, pmg.SMOOTHER_CHEBYSHEV)
    w = wl(dim, N, p)
    ctx, prob = gpu_ctx(w, **fixed(smoother=sm))
    m = omesh(prob)
    npatch = (N - 1) ** dim
    ids = inputs.sample_patches(17, npatch, 5)
    ni = (2 * p - 1) ** dim
    r = np.random.default_rng(4).uniform(-1, 1, (len(ids), ni))
    d = torch.zeros(len(ids) * ni, dtype=torch.float64, device="cuda")
    ctx.local_vcycle(0, torch.tensor(ids, device="cuda"), dev(r.reshape(-1)), d, ncyc)
    torch.cuda.synchronize()
    d = d.cpu().numpy().reshape(len(ids), ni)
    osm = pt.Smoother(kind=kind)
    verts = pt.interior_vertices(dim, N)
    byid = {pt.patch_id(dim, N, v): v for v in verts}
    for i, j in enumerate(ids):
        P = pt.Patch(m, byid[int(j)], pt.levels_halving(p))
        bounds = lz.fixed_bounds_fn(FIX_LO, FIX_HI)(P, int(j))
        ref = pt.local_solve(P, r[i], osm, bounds, ncyc)
        assert relerr(d[i], ref) < TOL, (j,)
    ctx.close()


def test_local_vcycle_ids_out_of_range_give_zero_rows():
    dim, N, p = 2, 5, 3
    ctx, prob = gpu_ctx(wl(dim, N, p), **fixed())
    npatch = (N - 1) ** dim
    ni = (2 * p - 1) ** dim
    ids = np.array([0, npatch, -1, npatch - 1, -(2 ** 40)], dtype=np.int64)
    r = np.random.default_rng(5).uniform(-1, 1, (len(ids), ni))
    d = torch.full((len(ids) * ni,), 7.0, dtype=torch.float64, device="cuda")
    ctx.local_vcycle(0, torch.tensor(ids, device="cuda"), dev(r.reshape(-1)), d, 1)
    torch.cuda.synchronize()
    d = d.cpu().numpy().reshape(len(ids), ni)
    assert np.all(d[[1, 2, 4]] == 0.0)
    assert np.abs(d[0]).max() > 0 and np.abs(d[3]).max() > 0
    ctx.close()


@pytest.mark.parametrize("dim,N,p", [(2, 5, 4), (2, 3, 8), (3, 3, 4), (3, 2, 6)])
def test_lanczos_bounds(dim, N, p):
    w = wl(dim, N, p)
    ctx, prob = gpu_ctx(w)          # default: 16-step Lanczos bounds
    m = omesh(prob)
    ritz = ctx.get_ritz(0)
    bnds = ctx.get_bounds(0)
    levels = ctx.p_levels()
    verts = pt.interior_vertices(dim, N)
    for v in verts[:: max(1, len(verts) // 6)]:
        j = pt.patch_id(dim, N, v)
        P = pt.Patch(m, v, levels)
        for k, q in enumerate(levels):
            if q == 1:
                continue
            lv = P.lv[q]
            lo, hi, tmin, tmax = lz.patch_bounds(lv.A, lv.diag, 0, j, q)
            assert abs(ritz[j, k, 1] - tmax) < 1e-10 * tmax and abs(ritz[j, k, 0] - tmin) < 1e-10 * tmax
            assert abs(bnds[j, k, 1] - hi) < 1e-10 * hi and abs(bnds[j, k, 0] - lo) < 1e-10 * hi
    ctx.close()


# ------------------------------------------------------------------ sweeps
@pytest.mark.parametrize("dim,N,p,kind,reverse", [
    (2, 16, 4, "chebyshev", False),      # the 2D Q4 16x16 workload
    (2, 7, 3, "jacobi", True), (2, 5, 6, "chebyshev", True), (2, 2, 2, "chebyshev", False),
    (2, 3, 1, "chebyshev", False), (3, 4, 4, "chebyshev", False), (3, 3, 2, "jacobi", True),
    (3, 2, 3, "chebyshev", False), (2, 6, 5, "fdm", False), (3, 3, 4, "fdm", True)])
def test_sweep_matches_sequential_oracle(dim, N, p, kind, reverse):
    from paper_2510_17785_gb300 import pmg
    sm = {"jacobi": pmg.SMOOTHER_JACOBI, "fdm": pmg.SMOOTHER_CARTESIAN}.get(kind, pmg.SMOOTHER_CHEBYSHEV)
    w = wl(dim, N, p, perturb=0.25 if N > 2 else 0.0)
    ctx, prob = gpu_ctx(w, **fixed(smoother=sm))
    m = omesh(prob)
    u0 = inputs.random_vector(8, dim, p, N)
    b = prob.rhs
    u = dev(u0)
    ctx.patch_smooth(0, dev(b), u, 1, reverse)
    torch.cuda.synchronize()
    S = pt.PatchSmoother(m, p, sm=pt.Smoother(kind=kind), bounds_fn=lz.fixed_bounds_fn(FIX_LO, FIX_HI))
    ref = S.sweep(u0, b, reverse=reverse)
    assert relerr(u.cpu().numpy(), ref) < TOL
    ctx.close()


def test_sweep_with_lanczos_bounds_both_sides():
    dim, N, p = 2, 8, 4
    w = wl(dim, N, p)
    ctx, prob = gpu_ctx(w)
    m = omesh(prob)
    u0 = inputs.random_vector(9, dim, p, N)
    u = dev(u0)
    ctx.patch_smooth(0, dev(prob.rhs), u, 2, False)
    torch.cuda.synchronize()
    S = pt.PatchSmoother(m, p, bounds_fn=lz.lanczos_bounds_fn(seed=0))
    ref = S.sweep(S.sweep(u0, prob.rhs), prob.rhs)
    assert relerr(u.cpu().numpy(), ref) < 1e-11
    ctx.close()


# -------------------------------------------------------------- GMG and CG
@pytest.mark.parametrize("dim,N,p,levels", [(2, 8, 3, 3), (2, 8, 4, 2), (3, 4, 2, 2)])
def test_gmg_vcycle(dim, N, p, levels):
    w = wl(dim, N, p)
    ctx, prob = gpu_ctx(w, n_levels=levels, **fixed())
    G = gmg.GMG(omesh(prob), p, N >> (levels - 1),
                smoother_args=dict(bounds_fn=lz.fixed_bounds_fn(FIX_LO, FIX_HI)))
    b = prob.rhs
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    ctx.gmg_vcycle(dev(b), x)
    torch.cuda.synchronize()
    assert relerr(x.cpu().numpy(), G.vcycle(b)) < 1e-11
    ctx.close()


@pytest.mark.parametrize("kind", ["chebyshev", "jacobi"])
def test_cg_iterations_match_oracle(kind):
    from paper_2510_17785_gb300 import pmg
    sm = pmg.SMOOTHER_JACOBI if kind == "jacobi" else pmg.SMOOTHER_CHEBYSHEV
    dim, N, p, levels = 2, 8, 3, 3
    w = wl(dim, N, p)
    ctx, prob = gpu_ctx(w, n_levels=levels, smoother=sm)
    G = gmg.GMG(omesh(prob), p, N >> (levels - 1),
                smoother_args=dict(sm=pt.Smoother(kind=kind), bounds_fn=lz.lanczos_bounds_fn(seed=0)))
    b = prob.rhs
    xr, it_ref, hist = gmg.pcg(G.A[-1], b, G.vcycle, 1e-8, 100)
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    it, rel, _ = ctx.solve_cg(dev(b), x, 1e-8, 100)
    assert rel <= 1e-8
    assert abs(it - it_ref) <= 1, (it, it_ref)
    assert relerr(x.cpu().numpy(), xr) < 1e-9
    ctx.close()


def test_cg_host_vectors_match_device_path():
    dim, N, p = 3, 4, 2
    w = wl(dim, N, p)
    ctx, prob = gpu_ctx(w, n_levels=2)
    b = prob.rhs
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    it, rel, _ = ctx.solve_cg(dev(b), x, 1e-8, 100)
    xh = np.zeros_like(b)
    it2, rel2, _ = ctx.solve_cg_host(np.ascontiguousarray(b), xh, 1e-8, 100)
    assert it == it2 and rel2 <= 1e-8
    assert np.array_equal(xh, x.cpu().numpy())
    ctx.close()


def test_mixed_precision_cg_within_one_iteration():
    from paper_2510_17785_gb300 import pmg
    dim, N, p, levels = 3, 8, 4, 3
    w = wl(dim, N, p, kappa=("loguniform", -2.0, 2.0))
    ctx64, prob = gpu_ctx(w, n_levels=levels)
    ctx32, _ = gpu_ctx(w, n_levels=levels, precision=pmg.PREC_MIXED)
    b = dev(prob.rhs)
    x64 = torch.zeros_like(b)
    x32 = torch.zeros_like(b)
    it64, rel64, _ = ctx64.solve_cg(b, x64, 1e-8, 100)
    it32, rel32, _ = ctx32.solve_cg(b, x32, 1e-8, 100)
    assert rel32 <= 1e-8 and rel64 <= 1e-8
    assert it32 <= it64 + 1, (it32, it64)
    assert relerr(x32.cpu().numpy(), x64.cpu().numpy()) < 1e-6
    ctx64.close()
    ctx32.close()


# ------------------------------------------------------------- error paths
def test_degenerate_mesh_is_rejected():
    from paper_2510_17785_gb300 import pmg
    X = inputs.single_patch_vertices(2, 0.36, np.ones(2)) / 2.0      # beyond sqrt(2)/4
    ctx = pmg.Context(0, **fixed())
    ctx.mesh_structured(2, 2, 2, 1, X, np.ones(4))
    with pytest.raises(pmg.PMGError) as e:
        ctx.setup()
    assert e.value.code == 3
    ctx.close()


def test_unsupported_degree_is_rejected():
    from paper_2510_17785_gb300 import pmg
    ctx = pmg.Context(0)
    X = inputs.grid_vertices(3, 2)
    with pytest.raises(pmg.PMGError) as e:
        ctx.mesh_structured(3, 2, 9, 1, X, np.ones(8))
    assert e.value.code == 7
    with pytest.raises(pmg.PMGError) as e:
        ctx.mesh_structured(3, 2, 8, 1, X, np.ones(8))      # FP64 working set of Q8 does not fit
    assert e.value.code == 7
    ctx.close()


def test_empty_local_batch_is_a_no_op():
    w = wl(2, 4, 2)
    ctx, _ = gpu_ctx(w, **fixed())
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.local_vcycle(0, torch.zeros(0, dtype=torch.int64, device="cuda"), d, d, 1)
    ctx.close()


def test_recomputing_bounds_reuses_scratch_and_is_reproducible():
    from paper_2510_17785_gb300 import pmg
    w = wl(3, 4, 4)
    ctx, _ = gpu_ctx(w)
    a = ctx.get_ritz(0)
    for _ in range(3):
        ctx.compute_bounds(pmg.BOUNDS_LANCZOS)
    assert np.array_equal(ctx.get_ritz(0), a)
    ctx.compute_bounds(pmg.BOUNDS_FIXED)
    b = ctx.get_bounds(0)
    assert np.all(b[:, 0, 0] == ctx.options.fixed_lo) and np.all(b[:, 0, 1] == ctx.options.fixed_hi)
    ctx.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("p", [4, 6])
def test_launch_shape_variants_are_bit_identical(precision, p):
    """Every launch-shape variant of the sweep kernel computes the same bits
    (one owner thread per output, fixed summation order), so the set-up
    autotuner may pick any of them."""
    from paper_2510_17785_gb300 import pmg
    prec = pmg.PREC_MIXED if precision == "mixed" else pmg.PREC_FP64
    w = wl(3, 6, p)
    prob = inputs.make_problem(w)
    u0 = inputs.random_vector(31, 3, p, 6)
    outs = []
    for v in range(pmg.NUM_VARIANTS):
        ctx = pmg.Context(0, precision=prec, autotune=0, variant=v, **fixed())
        ctx.mesh_structured(3, 6, p, 2, prob.coords, prob.kappa)
        try:
            ctx.setup()
        except pmg.PMGError as e:
            assert e.code == 7            # variant does not exist for this configuration
            ctx.close()
            continue
        assert all(ctx.tuning_level(lv)[0] == v for lv in range(2))   # without autotuning: the chosen variant
        u = dev(u0)
        ctx.patch_smooth(1, dev(prob.rhs), u, 2, False)
        torch.cuda.synchronize()
        outs.append(u.cpu().numpy())
        ctx.close()
    assert len(outs) >= 2
    for o in outs[1:]:
        assert np.array_equal(o, outs[0]), relerr(o, outs[0])


# ------------------------------------------------ weighted additive sweep
@pytest.mark.parametrize("dim,N,p,reverse,theta", [(2, 6, 3, False, 1.0), (2, 6, 3, True, 0.7), (3, 4, 2, False, 0.5),
                                                   (3, 3, 4, True, 1.0)])
def test_additive_sweep_matches_oracle(dim, N, p, reverse, theta):
    w = wl(dim, N, p)
    ctx, prob = gpu_ctx(w, **fixed(additive=1, additive_theta=theta))
    m = omesh(prob)
    u0 = inputs.random_vector(9, dim, p, N)
    b = prob.rhs
    u = dev(u0)
    ctx.patch_smooth(0, dev(b), u, 1, reverse)
    torch.cuda.synchronize()
    S = pt.PatchSmoother(m, p, bounds_fn=lz.fixed_bounds_fn(FIX_LO, FIX_HI), additive=True, theta=theta)
    ref = S.sweep(u0, b, reverse=reverse)
    assert relerr(u.cpu().numpy(), ref) < TOL
    ctx.close()


def test_additive_gmg_cg_matches_oracle():
    dim, N, p, levels = 2, 8, 3, 3
    w = wl(dim, N, p)
    ctx, prob = gpu_ctx(w, n_levels=levels, **fixed(additive=1, additive_theta=0.6))
    G = gmg.GMG(omesh(prob), p, N >> (levels - 1),
                smoother_args=dict(bounds_fn=lz.fixed_bounds_fn(FIX_LO, FIX_HI), additive=True, theta=0.6))
    b = prob.rhs
    xr, it_ref, hist = gmg.pcg(G.A[-1], b, G.vcycle, 1e-8, 200)
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    it, rel, _ = ctx.solve_cg(dev(b), x, 1e-8, 200)
    assert rel <= 1e-8 and hist[-1] <= 1e-8
    assert abs(it - it_ref) <= 1, (it, it_ref)
    assert relerr(x.cpu().numpy(), xr) < 1e-9
    ctx.close()


def test_autotuner_picks_a_variant_per_level():
    """With autotuning every mesh level gets an existing variant, timed."""
    w = wl(3, 8, 4)
    ctx, prob = gpu_ctx(w, n_levels=3, **fixed())
    for lv in range(1, 3):
        v, ms = ctx.tuning_level(lv)
        assert 0 <= v < 8 and ms[v] > 0 and all(m < 0 or m >= ms[v] for m in ms)
    ctx.close()


def test_coefficient_upload_per_level():
    """pmg_coeff_upload replaces a level's coefficients: uploading the harmonic
    mean of the children on the coarse level gives the operator of the
    harmonic coarse rule, uploading 2 kappa on the finest level doubles its
    operator, and an upload after set-up is rejected."""
    from paper_2510_17785_gb300 import pmg
    w = wl(3, 4, 2, kappa=("loguniform", -1, 1))
    prob = inputs.make_problem(w)
    kap = prob.kappa.reshape(4, 4, 4)
    harm = np.zeros((2, 2, 2))
    for c in range(8):
        off = [(c >> k) & 1 for k in range(3)]
        harm += 1.0 / kap[off[2]::2, off[1]::2, off[0]::2]
    harm = 8.0 / harm

    def apply(ctx, level):
        n, _ = ctx.num_dofs(level)
        u = dev(inputs.random_vector(41 + level, 3, 2, 4 >> (1 - level)))
        out = torch.zeros_like(u)
        ctx.apply(level, u, out)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    ref = pmg.Context(0, coarse_kappa=pmg.KAPPA_HARMONIC, **fixed())
    ref.mesh_structured(3, 4, 2, 2, prob.coords, prob.kappa)
    ref.setup()
    up = pmg.Context(0, **fixed())
    up.mesh_structured(3, 4, 2, 2, prob.coords, prob.kappa)
    up.coeff_upload(0, harm.reshape(-1))
    up.setup()
    a, b = apply(ref, 0), apply(up, 0)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    two = pmg.Context(0, **fixed())
    two.mesh_structured(3, 4, 2, 2, prob.coords, prob.kappa)
    two.coeff_upload(1, 2.0 * prob.kappa)
    two.setup()
    a, b = apply(ref, 1), apply(two, 1)
    assert np.abs(2.0 * a - b).max() <= 1e-12 * np.abs(b).max()
    with pytest.raises(pmg.PMGError):
        two.coeff_upload(0, harm.reshape(-1))
    for c in (ref, up, two):
        c.close()
