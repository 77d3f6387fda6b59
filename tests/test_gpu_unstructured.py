"""Unstructured quadrilateral / hexahedral meshes: the CUDA path through the C
ABI against the unstructured oracle (oracle/unstructured.py).

Integer structures (global DoF maps of every p-level, patch lists, colours)
bit-exactly; FP64 operators, local V-cycles and sweeps to 1e-12 relative
(max-norm error over the max-norm of the oracle result); the two-level CG
within one iteration of the oracle's.  Meshes: seeded triangulations split
into quadrilaterals (interior valences 3 to 8), their extrusions (6 to 16)
and split tetrahedralisations of the cube (4, 6, and up to 24 at the cube's
vertices)."""
import numpy as np
import pytest

from oracle import fem, gmg, lanczos as lz, patch as pt, unstructured as us
from paper_2510_17785_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
FIX_LO, FIX_HI = 0.25, 2.2


def relerr(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def mesh(name, kappa_seed=1):
    if name.startswith("2d"):
        P, T = inputs.triangulated_square(4, 11)
        X, C = inputs.triangles_to_quads(P, T)
    elif name == "3d_extruded":
        P, T = inputs.triangulated_square(2, 12)
        X, C = inputs.triangles_to_quads(P, T)
        X, C = inputs.extrude(X, C, 2)
    else:
        P, T = inputs.cube_tetrahedra(2 if name == "3d_tetsplit" else 1, 13)
        X, C = inputs.tetrahedra_to_hexes(P, T)
    kappa = 10.0 ** np.random.default_rng(kappa_seed).uniform(-1, 1, len(C))
    return X, C, kappa


def ctx_for(name, p, setup=True, **opt):
    from paper_2510_17785_gb300 import pmg
    X, C, kappa = mesh(name)
    dim = X.shape[1]
    o = dict(bounds=pmg.BOUNDS_FIXED, fixed_lo=FIX_LO, fixed_hi=FIX_HI)
    o.update(opt)
    ctx = pmg.Context(0, **o)
    ctx.mesh_upload(dim, X, C, p, kappa=kappa)
    if setup:
        ctx.setup()
    return ctx, us.Mesh(dim, X, C, kappa)


MESHES = ["2d_trisplit", "3d_extruded", "3d_tetsplit_small"]


@pytest.mark.parametrize("name,p", [("2d_trisplit", 4), ("2d_trisplit", 7), ("3d_extruded", 3),
                                    ("3d_tetsplit_small", 4), ("3d_tetsplit", 2)])
def test_dof_maps_patches_and_colours_bit_exact(name, p):
    from paper_2510_17785_gb300 import pmg
    ctx, m = ctx_for(name, p, seed=7)
    assert ctx.p_levels() == pt.levels_halving(p)
    for k, q in enumerate(ctx.p_levels()):
        assert np.array_equal(ctx.get_dof_map(k), m.cell_dofs(q)), q
    total, free = ctx.num_dofs(0)
    assert total == m.n_dofs(p) and free == int((~m.boundary_dofs(p)).sum())
    verts = m.interior_vertices()
    npatch, ncol = ctx.num_patches(0)
    assert npatch == len(verts)
    pm = ctx.get_patch_map(0)
    assert pm.shape == (npatch, 1 + pmg.UMAXC)
    for i, v in enumerate(verts):
        cells = sorted(m.vertex_cells[v])
        assert pm[i, 0] == v
        assert list(pm[i, 1: 1 + len(cells)]) == cells and np.all(pm[i, 1 + len(cells):] == -1)
    col = us.colours(m, seed=7)
    assert np.array_equal(ctx.get_colours(0), np.array([col[v] for v in verts], dtype=np.uint8))
    assert ncol == 1 + max(col.values())
    ni = max(len(us.Patch(m, v, [p]).lv[p].interior) for v in verts)
    assert ctx.local_size(0) == ni
    ctx.close()


@pytest.mark.parametrize("name,p", [("2d_trisplit", 1), ("2d_trisplit", 5), ("2d_trisplit", 8),
                                    ("3d_extruded", 2), ("3d_extruded", 4), ("3d_tetsplit", 3),
                                    ("3d_tetsplit_small", 6)])
def test_global_apply(name, p):
    ctx, m = ctx_for(name, p)
    free = ~m.boundary_dofs(p)
    A = fem.operator_with_dirichlet(m.assemble(p), free)
    u = np.random.default_rng(3).uniform(-1, 1, m.n_dofs(p))
    out = torch.zeros(len(u), dtype=torch.float64, device="cuda")
    ctx.apply(0, dev(u), out)
    torch.cuda.synchronize()
    assert relerr(out.cpu().numpy(), A @ (u * free)) < TOL
    ctx.close()


@pytest.mark.parametrize("name,p,kind,ncyc", [
    ("2d_trisplit", 4, "chebyshev", 1), ("2d_trisplit", 7, "chebyshev", 2), ("2d_trisplit", 3, "jacobi", 1),
    ("3d_extruded", 2, "chebyshev", 1), ("3d_extruded", 4, "jacobi", 2), ("3d_tetsplit", 2, "chebyshev", 1),
    ("3d_tetsplit_small", 4, "chebyshev", 1), ("3d_tetsplit_small", 5, "chebyshev", 1)])
def test_local_vcycle(name, p, kind, ncyc):
    from paper_2510_17785_gb300 import pmg
    sm = pmg.SMOOTHER_JACOBI if kind == "jacobi" else pmg.SMOOTHER_CHEBYSHEV
    ctx, m = ctx_for(name, p, smoother=sm)
    verts = m.interior_vertices()
    ids = inputs.sample_patches(17, len(verts), min(6, len(verts)))
    ni = ctx.local_size(0)
    r = np.random.default_rng(4).uniform(-1, 1, (len(ids), ni))
    d = torch.full((len(ids) * ni,), 7.0, dtype=torch.float64, device="cuda")
    ctx.local_vcycle(0, torch.tensor(ids, device="cuda"), dev(r.reshape(-1)), d, ncyc)
    torch.cuda.synchronize()
    d = d.cpu().numpy().reshape(len(ids), ni)
    osm = pt.Smoother(kind=kind)
    levels = pt.levels_halving(p)
    for i, j in enumerate(ids):
        P = us.Patch(m, verts[int(j)], levels)
        n = len(P.lv[p].interior)
        ref = pt.local_solve(P, r[i, :n], osm, lz.fixed_bounds_fn(FIX_LO, FIX_HI)(P, int(j)), ncyc)
        assert relerr(d[i, :n], ref) < TOL, (j, verts[int(j)])
        assert np.all(d[i, n:] == 0.0)
    ctx.close()


@pytest.mark.parametrize("name,p,kind,reverse", [
    ("2d_trisplit", 4, "chebyshev", False), ("2d_trisplit", 6, "chebyshev", True), ("2d_trisplit", 2, "jacobi", False),
    ("3d_extruded", 3, "chebyshev", True), ("3d_tetsplit", 2, "chebyshev", False),
    ("3d_tetsplit_small", 4, "jacobi", True)])
def test_sweep_matches_sequential_oracle(name, p, kind, reverse):
    from paper_2510_17785_gb300 import pmg
    sm = pmg.SMOOTHER_JACOBI if kind == "jacobi" else pmg.SMOOTHER_CHEBYSHEV
    ctx, m = ctx_for(name, p, smoother=sm)
    rng = np.random.default_rng(8)
    free = ~m.boundary_dofs(p)
    u0 = rng.uniform(-1, 1, m.n_dofs(p)) * free
    b = rng.uniform(-1, 1, m.n_dofs(p)) * free
    u = dev(u0)
    ctx.patch_smooth(0, dev(b), u, 1, reverse)
    torch.cuda.synchronize()
    S = us.PatchSmoother(m, p, sm=pt.Smoother(kind=kind), bounds_fn=lz.fixed_bounds_fn(FIX_LO, FIX_HI))
    assert relerr(u.cpu().numpy(), S.sweep(u0, b, reverse=reverse)) < TOL
    # colour by colour gives the same result
    u2 = dev(u0)
    order = range(ctx.num_patches(0)[1])
    for c in (reversed(order) if reverse else order):
        ctx.patch_smooth_colour(0, c, dev(b), u2)
    torch.cuda.synchronize()
    assert torch.equal(u, u2)
    ctx.close()


@pytest.mark.parametrize("name,p", [("2d_trisplit", 4), ("3d_extruded", 2), ("3d_tetsplit_small", 3)])
def test_user_bounds_per_patch(name, p):
    """PMG_BOUNDS_USER: one interval per patch and p-level, as uploaded."""
    from paper_2510_17785_gb300 import pmg
    ctx, m = ctx_for(name, p, setup=False, bounds=pmg.BOUNDS_USER)
    ctx.setup()
    npatch = ctx.num_patches(0)[0]
    nl = len(ctx.p_levels())
    rng = np.random.default_rng(21)
    lohi = np.zeros((npatch, nl, 2))
    lohi[:, :, 0] = rng.uniform(0.1, 0.4, (npatch, nl))
    lohi[:, :, 1] = rng.uniform(1.6, 2.4, (npatch, nl))
    lohi[:, [i for i, q in enumerate(ctx.p_levels()) if q == 1], :] = 0.0
    ctx.set_bounds(0, lohi)
    assert np.array_equal(ctx.get_bounds(0), lohi)
    free = ~m.boundary_dofs(p)
    u0 = rng.uniform(-1, 1, m.n_dofs(p)) * free
    b = rng.uniform(-1, 1, m.n_dofs(p)) * free
    u = dev(u0)
    ctx.patch_smooth(0, dev(b), u, 1, False)
    torch.cuda.synchronize()
    verts = m.interior_vertices()
    pos = {v: i for i, v in enumerate(verts)}
    levels = pt.levels_halving(p)

    def bfn(P, v):
        return {q: tuple(lohi[pos[v], k]) for k, q in enumerate(levels) if q != 1}

    S = us.PatchSmoother(m, p, bounds_fn=bfn)
    assert relerr(u.cpu().numpy(), S.sweep(u0, b)) < TOL
    ctx.close()


@pytest.mark.parametrize("name,p", [("2d_trisplit", 4), ("3d_extruded", 2), ("3d_tetsplit_small", 4)])
def test_two_level_vcycle_and_cg(name, p):
    """The two-level preconditioner (sweep, Q1 coarse correction, reversed
    sweep) to 1e-11 and the CG iteration count within one of the oracle's."""
    ctx, m = ctx_for(name, p)
    S = us.PatchSmoother(m, p, bounds_fn=lz.fixed_bounds_fn(FIX_LO, FIX_HI))
    TL = us.TwoLevel(m, p, S)
    free = ~m.boundary_dofs(p)
    b = np.random.default_rng(9).uniform(-1, 1, m.n_dofs(p)) * free
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    ctx.gmg_vcycle(dev(b), x)
    torch.cuda.synchronize()
    assert relerr(x.cpu().numpy(), TL.vcycle(b)) < 1e-11
    xr, it_ref, _ = gmg.pcg(TL.A, b, TL.vcycle, 1e-8, 100)
    x.zero_()
    it, rel, _ = ctx.solve_cg(dev(b), x, 1e-8, 100)
    assert rel <= 1e-8
    assert abs(it - it_ref) <= 1, (it, it_ref)
    assert relerr(x.cpu().numpy(), xr) < 1e-8
    ctx.close()


@pytest.mark.parametrize("name,p", [("2d_trisplit", 6), ("3d_tetsplit", 3)])
def test_mixed_precision(name, p):
    """FP32 patch solves (Lanczos intervals, computed with the FP64 operator
    in both modes): a sweep within FP32 rounding of the FP64 one, CG (FP64
    outer iteration) within one iteration of the FP64 preconditioner."""
    from paper_2510_17785_gb300 import pmg
    c64, m = ctx_for(name, p, bounds=pmg.BOUNDS_LANCZOS)
    c32, _ = ctx_for(name, p, bounds=pmg.BOUNDS_LANCZOS, precision=pmg.PREC_MIXED)
    free = ~m.boundary_dofs(p)
    rng = np.random.default_rng(10)
    u0 = rng.uniform(-1, 1, m.n_dofs(p)) * free
    b = rng.uniform(-1, 1, m.n_dofs(p)) * free
    u64, u32 = dev(u0), dev(u0)
    c64.patch_smooth(0, dev(b), u64, 1, False)
    c32.patch_smooth(0, dev(b), u32, 1, False)
    torch.cuda.synchronize()
    assert relerr(u32.cpu().numpy(), u64.cpu().numpy()) < 2e-5
    x64 = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    x32 = torch.zeros_like(x64)
    it64, rel64, _ = c64.solve_cg(dev(b), x64, 1e-8, 100)
    it32, rel32, _ = c32.solve_cg(dev(b), x32, 1e-8, 100)
    assert rel64 <= 1e-8 and rel32 <= 1e-8
    assert abs(it32 - it64) <= 1
    c64.close()
    c32.close()


def test_host_vectors_and_launch_count():
    ctx, m = ctx_for("2d_trisplit", 3)
    b = np.random.default_rng(2).uniform(-1, 1, m.n_dofs(3)) * ~m.boundary_dofs(3)
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    n0 = ctx.launch_count()
    it, rel, _ = ctx.solve_cg(dev(b), x, 1e-8, 100)
    assert ctx.launch_count() > n0
    xh = np.zeros_like(b)
    it2, rel2, _ = ctx.solve_cg_host(np.ascontiguousarray(b), xh, 1e-8, 100)
    assert it == it2 and rel2 <= 1e-8
    assert np.array_equal(xh, x.cpu().numpy())
    ctx.close()


def test_rejections():
    from paper_2510_17785_gb300 import pmg
    X, C, kappa = mesh("2d_trisplit")
    ctx = pmg.Context(0, bounds=pmg.BOUNDS_MLP)
    ctx.mesh_upload(2, X, C, 3)
    with pytest.raises(pmg.PMGError):                 # learned intervals are structured-only
        ctx.setup()
    ctx.close()
    ctx = pmg.Context(0, bounds=pmg.BOUNDS_FIXED)
    with pytest.raises(pmg.PMGError):
        ctx.mesh_upload(2, X, C, 9)                   # degree above 8
    ctx.close()
    ctx = pmg.Context(0, bounds=pmg.BOUNDS_FIXED)
    bad = C.copy()
    bad[0, [2, 3]] = bad[0, [3, 2]]                    # a self-intersecting (bow-tie) cell
    ctx.mesh_upload(2, X, bad, 2)
    with pytest.raises(pmg.PMGError) as e:
        ctx.setup()
    assert e.value.code == pmg.PMG_ERR_DEGENERATE
    ctx.close()
    ctx = pmg.Context(0, bounds=pmg.BOUNDS_FIXED)
    rep = C.copy()
    rep[0, 1] = rep[0, 0]
    with pytest.raises(pmg.PMGError):                 # a cell repeating a vertex
        ctx.mesh_upload(2, X, rep, 2)
    ctx.close()
    ctx, _ = ctx_for("2d_trisplit", 3)
    for call in (lambda: ctx.get_inv_diag(0, 0, torch.zeros(1, device="cuda")),
                 lambda: ctx.rhs_manufactured(torch.zeros(1, device="cuda"))):
        with pytest.raises(pmg.PMGError) as e:
            call()
        assert e.value.code == pmg.PMG_ERR_UNSUPPORTED
    ctx.close()


def test_local_vcycle_ids_out_of_range_give_zero_rows():
    ctx, m = ctx_for("2d_trisplit", 3)
    npatch = ctx.num_patches(0)[0]
    ni = ctx.local_size(0)
    ids = np.array([0, npatch, -1, npatch - 1], dtype=np.int64)
    r = np.random.default_rng(5).uniform(-1, 1, (len(ids), ni))
    d = torch.full((len(ids) * ni,), 7.0, dtype=torch.float64, device="cuda")
    ctx.local_vcycle(0, torch.tensor(ids, device="cuda"), dev(r.reshape(-1)), d, 1)
    torch.cuda.synchronize()
    d = d.cpu().numpy().reshape(len(ids), ni)
    assert np.all(d[1] == 0.0) and np.all(d[2] == 0.0)
    assert np.abs(d[0]).max() > 0 and np.abs(d[3]).max() > 0
    ctx.close()


@pytest.mark.parametrize("name,p", [("2d_trisplit", 4), ("2d_trisplit", 8), ("3d_extruded", 3),
                                    ("3d_tetsplit", 2), ("3d_tetsplit_small", 6)])
def test_lanczos_intervals(name, p):
    """PMG_BOUNDS_LANCZOS on unstructured patches: Ritz values and intervals
    of every patch and p-level q > 1 against the oracle's Lanczos (start
    vector counter from the patch's vertex id), and a sweep with those
    intervals on both sides."""
    from paper_2510_17785_gb300 import pmg
    ctx, m = ctx_for(name, p, bounds=pmg.BOUNDS_LANCZOS, seed=3)
    verts = m.interior_vertices()
    levels = pt.levels_halving(p)
    ritz, bd = ctx.get_ritz(0), ctx.get_bounds(0)
    for j, v in enumerate(verts):
        P = us.Patch(m, v, levels)
        for k, q in enumerate(levels):
            if q == 1:
                continue
            lv = P.lv[q]
            lo, hi, tmin, tmax = lz.patch_bounds(lv.A, lv.diag, 3, v, q)
            assert abs(ritz[j, k, 0] - tmin) <= 1e-9 * tmax and abs(ritz[j, k, 1] - tmax) <= 1e-9 * tmax, (v, q)
            assert abs(bd[j, k, 0] - lo) <= 1e-9 * hi and abs(bd[j, k, 1] - hi) <= 1e-9 * hi, (v, q)
    free = ~m.boundary_dofs(p)
    rng = np.random.default_rng(12)
    u0 = rng.uniform(-1, 1, m.n_dofs(p)) * free
    b = rng.uniform(-1, 1, m.n_dofs(p)) * free
    u = dev(u0)
    ctx.patch_smooth(0, dev(b), u, 1, False)
    torch.cuda.synchronize()
    S = us.PatchSmoother(m, p, bounds_fn=lz.lanczos_bounds_fn(seed=3), seed=3)   # the seed also colours
    assert relerr(u.cpu().numpy(), S.sweep(u0, b)) < 1e-10
    ctx.close()


def test_lanczos_two_level_cg_high_degree():
    """2D degree 8: with Lanczos intervals the two-level CG converges and
    matches the oracle's iteration count within one."""
    from paper_2510_17785_gb300 import pmg
    p = 8
    ctx, m = ctx_for("2d_trisplit", p, bounds=pmg.BOUNDS_LANCZOS)
    S = us.PatchSmoother(m, p, bounds_fn=lz.lanczos_bounds_fn(seed=0))
    TL = us.TwoLevel(m, p, S)
    b = np.random.default_rng(9).uniform(-1, 1, m.n_dofs(p)) * ~m.boundary_dofs(p)
    _, it_ref, _ = gmg.pcg(TL.A, b, TL.vcycle, 1e-8, 100)
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    it, rel, _ = ctx.solve_cg(dev(b), x, 1e-8, 100)
    assert rel <= 1e-8 and it_ref < 100
    assert abs(it - it_ref) <= 1, (it, it_ref)
    ctx.close()
