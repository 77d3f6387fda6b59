"""The paper's p-level rule in the kernels (options.level_rule = 1): the local
V-cycle runs on p and the nested degrees 1, 3, 7, ... below it (Section 3.1;
p = 8: 8, 7, 3, 1), with the embeddings between those degrees.  Checked
against the oracle run with the same sequence (oracle.patch.levels_paper):
sweeps and local V-cycles to 1e-12 in FP64, the GMG-preconditioned CG within
one iteration; the reported p-levels; the rejections."""
import numpy as np
import pytest

from oracle import fem, gmg, lanczos as lz, patch as pt
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
    ctx = pmg.Context(0, level_rule=1, **opt)
    ctx.mesh_structured(w.dim, w.N, w.p, levels, prob.coords, prob.kappa)
    ctx.setup()
    return ctx, prob


def _wl(dim, N, p, seed=41):
    return inputs.Workload("lr", dim, N, p, 0.2, "uniform", ("loguniform", -1.0, 1.0), "uniform", seed)


@pytest.mark.parametrize("dim,N,p,kind", [(2, 5, 4, "chebyshev"), (2, 4, 5, "jacobi"), (2, 3, 8, "chebyshev"),
                                          (3, 3, 4, "chebyshev"), (3, 2, 5, "jacobi")])
def test_sweep_and_local_vcycle_match_the_oracle(dim, N, p, kind):
    from paper_2510_17785_gb300 import pmg
    sm = pmg.SMOOTHER_JACOBI if kind == "jacobi" else pmg.SMOOTHER_CHEBYSHEV
    w = _wl(dim, N, p)
    ctx, prob = _ctx(w, 1, precision=pmg.PREC_FP64, smoother=sm, bounds=pmg.BOUNDS_FIXED, fixed_lo=FIX_LO,
                     fixed_hi=FIX_HI)
    levels = pt.levels_paper(p)
    assert ctx.p_levels() == levels
    m = fem.StructuredMesh(dim, N, prob.coords, prob.kappa)
    u0 = inputs.random_vector(8, dim, p, N)
    u = torch.tensor(u0, device="cuda")
    ctx.patch_smooth(0, torch.tensor(prob.rhs, device="cuda"), u, 1, False)
    torch.cuda.synchronize()
    S = pt.PatchSmoother(m, p, levels=levels, sm=pt.Smoother(kind=kind),
                         bounds_fn=lz.fixed_bounds_fn(FIX_LO, FIX_HI))
    assert relerr(u.cpu().numpy(), S.sweep(u0, prob.rhs)) < 1e-12
    # local V-cycles on sampled patches
    npatch = (N - 1) ** dim
    ids = inputs.sample_patches(3, npatch, 4)
    ni = (2 * p - 1) ** dim
    r = np.random.default_rng(4).uniform(-1, 1, (len(ids), ni))
    d = torch.zeros(len(ids) * ni, dtype=torch.float64, device="cuda")
    ctx.local_vcycle(0, torch.tensor(ids, device="cuda"), torch.tensor(r.reshape(-1), device="cuda"), d, 2)
    torch.cuda.synchronize()
    d = d.cpu().numpy().reshape(len(ids), ni)
    verts = pt.interior_vertices(dim, N)
    byid = {pt.patch_id(dim, N, v): v for v in verts}
    for i, j in enumerate(ids):
        P = pt.Patch(m, byid[int(j)], levels)
        ref = pt.local_solve(P, r[i], pt.Smoother(kind=kind), lz.fixed_bounds_fn(FIX_LO, FIX_HI)(P, int(j)), 2)
        assert relerr(d[i], ref) < 1e-12, j
    ctx.close()


@pytest.mark.parametrize("dim,N,p,levels", [(2, 8, 4, 3), (2, 8, 8, 2), (3, 4, 4, 2)])
def test_cg_with_the_paper_levels_matches_the_oracle(dim, N, p, levels):
    from paper_2510_17785_gb300 import pmg
    w = _wl(dim, N, p)
    ctx, prob = _ctx(w, levels, precision=pmg.PREC_FP64)
    G = gmg.GMG(fem.StructuredMesh(dim, N, prob.coords, prob.kappa), p, N >> (levels - 1),
                smoother_args=dict(levels=pt.levels_paper(p), bounds_fn=lz.lanczos_bounds_fn(seed=0)))
    b = prob.rhs
    xr, it_ref, _ = gmg.pcg(G.A[-1], b, G.vcycle, 1e-8, 100)
    x = torch.zeros(len(b), dtype=torch.float64, device="cuda")
    it, rel, _ = ctx.solve_cg(torch.tensor(b, device="cuda"), x, 1e-8, 100)
    assert rel <= 1e-8 and abs(it - it_ref) <= 1, (it, it_ref)
    assert relerr(x.cpu().numpy(), xr) < 1e-8
    ctx.close()


def test_mixed_precision_degree_8_in_3d():
    from paper_2510_17785_gb300 import pmg
    w = _wl(3, 2, 8)
    ref, prob = _ctx(w, 1, precision=pmg.PREC_MIXED, bounds=pmg.BOUNDS_FIXED, fixed_lo=FIX_LO, fixed_hi=FIX_HI)
    assert ref.p_levels() == [8, 7, 3, 1]
    u0 = inputs.random_vector(8, 3, 8, 2)
    u = torch.tensor(u0, device="cuda")
    ref.patch_smooth(0, torch.tensor(prob.rhs, device="cuda"), u, 1, False)
    torch.cuda.synchronize()
    m = fem.StructuredMesh(3, 2, prob.coords, prob.kappa)
    S = pt.PatchSmoother(m, 8, levels=[8, 7, 3, 1], bounds_fn=lz.fixed_bounds_fn(FIX_LO, FIX_HI))
    assert relerr(u.cpu().numpy(), S.sweep(u0, prob.rhs)) < 2e-5
    ref.close()


def test_rule_is_rejected_where_it_is_not_built():
    from paper_2510_17785_gb300 import pmg
    X, C = inputs.triangles_to_quads(*inputs.triangulated_square(2, 1))
    ctx = pmg.Context(0, level_rule=1)
    with pytest.raises(pmg.PMGError) as e:
        ctx.mesh_upload(2, X, C, 4)                  # unstructured meshes: halving only
    assert e.value.code == pmg.PMG_ERR_UNSUPPORTED
    ctx.close()
    w = _wl(3, 2, 8)
    prob = inputs.make_problem(w)
    ctx = pmg.Context(0, level_rule=1, precision=pmg.PREC_FP64)
    with pytest.raises(pmg.PMGError) as e:           # FP64 3D degree 8 does not fit shared memory
        ctx.mesh_structured(3, 2, 8, 1, prob.coords, prob.kappa)
    assert e.value.code == pmg.PMG_ERR_UNSUPPORTED
    ctx.close()
