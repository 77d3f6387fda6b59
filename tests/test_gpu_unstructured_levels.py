"""Unstructured mesh hierarchies: a coarse mesh and its uniform refinement
(pmg_mesh_upload levels 0 and 1 with parent cells and child indices).  The
CUDA path's V-cycle (fine sweep, h-restriction, the coarse mesh's two-level
cycle, h-prolongation, reverse sweep) against the oracle's TwoMeshLevels to
1e-11, per-level operators and sweeps to 1e-12, the CG iteration count within
one; coefficients of the coarse level derived from the children; rejections."""
import numpy as np
import pytest

from oracle import fem, gmg, lanczos as lz, patch as pt, unstructured as us
from paper_2510_17785_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIX_LO, FIX_HI = 0.25, 2.2


def relerr(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def dev(x):
    return torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda")


def hierarchy(kind, perturb_fine):
    if kind == "2d":
        X, C = inputs.triangles_to_quads(*inputs.triangulated_square(3, 21))
    else:
        X, C = inputs.triangles_to_quads(*inputs.triangulated_square(2, 22))
        X, C = inputs.extrude(X, C, 1)
    Xf, Cf, par, ch = inputs.refine_unstructured(X, C)
    if perturb_fine:
        # move the fine vertices; the coarse mesh keeps the fine positions of its own vertices
        Xf, _ = inputs.perturb_unstructured(Xf, Cf, 0.15, np.random.default_rng(3))
        X = Xf[: len(X)].copy()
    kf = 10.0 ** np.random.default_rng(5).uniform(-1, 1, len(Cf))
    return X, C, Xf, Cf, par, ch, kf


def contexts(kind, p, perturb_fine=True, coarse_kappa=False, **opt):
    from paper_2510_17785_gb300 import pmg
    X, C, Xf, Cf, par, ch, kf = hierarchy(kind, perturb_fine)
    dim = X.shape[1]
    kc = kf.reshape(len(C), 2 ** dim).mean(axis=1)       # the mean of the children
    o = dict(bounds=pmg.BOUNDS_FIXED, fixed_lo=FIX_LO, fixed_hi=FIX_HI)
    o.update(opt)
    ctx = pmg.Context(0, **o)
    ctx.mesh_upload(dim, X, C, p, kappa=(kc * 1.3 if coarse_kappa else None))
    ctx.mesh_upload(dim, Xf, Cf, level=1, parent=par, child=ch, kappa=kf)
    ctx.setup()
    mc = us.Mesh(dim, X, C, kc * 1.3 if coarse_kappa else kc)
    mf = us.Mesh(dim, Xf, Cf, kf)
    return ctx, mc, mf, par, ch


@pytest.mark.parametrize("kind,p,coarse_kappa", [("2d", 3, False), ("2d", 4, True), ("3d", 2, False)])
def test_levels_apply_and_sweep(kind, p, coarse_kappa):
    ctx, mc, mf, _, _ = contexts(kind, p, coarse_kappa=coarse_kappa)
    for level, m in ((0, mc), (1, mf)):
        free = ~m.boundary_dofs(p)
        assert ctx.num_dofs(level) == (m.n_dofs(p), int(free.sum()))
        A = fem.operator_with_dirichlet(m.assemble(p), free)
        rng = np.random.default_rng(level)
        u = rng.uniform(-1, 1, m.n_dofs(p))
        out = torch.zeros(len(u), dtype=torch.float64, device="cuda")
        ctx.apply(level, dev(u), out)
        b = rng.uniform(-1, 1, m.n_dofs(p)) * free
        u0 = u * free
        us_ = dev(u0)
        ctx.patch_smooth(level, dev(b), us_, 1, False)
        torch.cuda.synchronize()
        assert relerr(out.cpu().numpy(), A @ (u * free)) < 1e-12, level
        S = us.PatchSmoother(m, p, bounds_fn=lz.fixed_bounds_fn(FIX_LO, FIX_HI))
        assert relerr(us_.cpu().numpy(), S.sweep(u0, b)) < 1e-12, level
    ctx.close()


@pytest.mark.parametrize("kind,p", [("2d", 3), ("2d", 5), ("3d", 2), ("3d", 3)])
def test_hierarchy_vcycle_and_cg_match_the_oracle(kind, p):
    ctx, mc, mf, par, ch = contexts(kind, p)
    bfn = lz.fixed_bounds_fn(FIX_LO, FIX_HI)
    H = us.TwoMeshLevels(mc, mf, par, ch, p, us.PatchSmoother(mf, p, bounds_fn=bfn),
                         us.PatchSmoother(mc, p, bounds_fn=bfn))
    b = np.random.default_rng(9).uniform(-1, 1, mf.n_dofs(p)) * H.free
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    ctx.gmg_vcycle(dev(b), x)
    torch.cuda.synchronize()
    assert relerr(x.cpu().numpy(), H.vcycle(b)) < 1e-11
    xr, it_ref, _ = gmg.pcg(H.A, b, H.vcycle, 1e-8, 100)
    x.zero_()
    it, rel, _ = ctx.solve_cg(dev(b), x, 1e-8, 100)
    assert rel <= 1e-8 and abs(it - it_ref) <= 1, (it, it_ref)
    assert relerr(x.cpu().numpy(), xr) < 1e-8
    ctx.close()


def test_nested_refinement_and_lanczos_intervals():
    """Unperturbed refinement (nested spaces) with Lanczos intervals on both
    levels, mixed precision within one CG iteration of FP64."""
    from paper_2510_17785_gb300 import pmg
    c64, mc, mf, par, ch = contexts("2d", 4, perturb_fine=False, bounds=pmg.BOUNDS_LANCZOS)
    c32, _, _, _, _ = contexts("2d", 4, perturb_fine=False, bounds=pmg.BOUNDS_LANCZOS, precision=pmg.PREC_MIXED)
    H = us.TwoMeshLevels(mc, mf, par, ch, 4, us.PatchSmoother(mf, 4, bounds_fn=lz.lanczos_bounds_fn(seed=0)),
                         us.PatchSmoother(mc, 4, bounds_fn=lz.lanczos_bounds_fn(seed=0)))
    b = np.random.default_rng(2).uniform(-1, 1, mf.n_dofs(4)) * H.free
    _, it_ref, _ = gmg.pcg(H.A, b, H.vcycle, 1e-8, 100)
    x64, x32 = torch.zeros(len(b), dtype=torch.float64, device="cuda"), torch.zeros(len(b), dtype=torch.float64,
                                                                                     device="cuda")
    it64, r64, _ = c64.solve_cg(dev(b), x64, 1e-8, 100)
    it32, r32, _ = c32.solve_cg(dev(b), x32, 1e-8, 100)
    assert r64 <= 1e-8 and r32 <= 1e-8
    assert abs(it64 - it_ref) <= 1 and abs(it32 - it64) <= 1, (it_ref, it64, it32)
    c64.close()
    c32.close()


def test_hierarchy_rejections():
    from paper_2510_17785_gb300 import pmg
    X, C, Xf, Cf, par, ch, kf = hierarchy("2d", False)
    ctx = pmg.Context(0, bounds=pmg.BOUNDS_FIXED)
    with pytest.raises(pmg.PMGError):                    # level 1 before level 0
        ctx.mesh_upload(2, Xf, Cf, level=1, parent=par, child=ch)
    ctx.mesh_upload(2, X, C, 3)
    bad = ch.copy()
    bad[1] = bad[0]                                      # two children of one parent with one index
    with pytest.raises(pmg.PMGError) as e:
        ctx.mesh_upload(2, Xf, Cf, level=1, parent=par, child=bad)
    assert e.value.code == pmg.PMG_ERR_ARG
    Xc = np.ascontiguousarray(Xf)
    Cc = np.ascontiguousarray(Cf, dtype=np.int64)
    rc = ctx.lib.pmg_mesh_upload(ctx.h, 1, 2, len(Xf), Xc.ctypes.data, len(Cf), Cc.ctypes.data, None, None, None)
    assert rc == pmg.PMG_ERR_ARG                         # a refined mesh without its parents
    ctx.close()
