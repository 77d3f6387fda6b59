"""Full-size checks on the 3D Q4 32^3 perturbed workload, in the launch
configuration the benchmark times: one colour of the patch sweep checked
patch by patch against the oracle on sampled patches (every patch of colour 0
reads the initial u only, so each sampled update is an independent oracle
computation), and the GMG-preconditioned CG solve to 1e-8."""
import numpy as np
import pytest

from oracle import patch as pt
from paper_2510_17785_gb300 import inputs

import oracle_pool

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c2():
    from paper_2510_17785_gb300 import pmg
    w = inputs.C2
    prob = inputs.make_problem(w)
    ctx = pmg.Context(0)
    levels = int(np.log2(w.N // w.coarse_N)) + 1
    ctx.mesh_structured(w.dim, w.N, w.p, levels, prob.coords, prob.kappa)
    ctx.setup()
    yield ctx, prob, levels
    ctx.close()


def test_colour0_sweep_sampled_patches(c2):
    ctx, prob, levels = c2
    w = prob.workload
    lf = levels - 1
    u0 = inputs.random_vector(21, w.dim, w.p, w.N)
    b = inputs.random_vector(22, w.dim, w.p, w.N)
    u = torch.tensor(u0, device="cuda")
    ctx.patch_smooth_colour(lf, 0, torch.tensor(b, device="cuda"), u)
    torch.cuda.synchronize()
    u1 = u.cpu().numpy()
    verts = [v for v in pt.interior_vertices(w.dim, w.N) if pt.colour_of(v) == 0]
    rng = np.random.default_rng(23)
    pick = [verts[i] for i in rng.choice(len(verts), 12, replace=False)]
    pick.append(verts[0])
    pick.append(verts[-1])
    for v, (j, idx, d, _) in zip(pick, oracle_pool.patch_updates(w.name, pick, u0, b)):
        got = u1[idx] - u0[idx]
        assert np.abs(got - d).max() < 1e-12 * np.abs(d).max(), v
    # DoFs outside every colour-0 patch interior are untouched, bit for bit
    outside = ~oracle_pool.interior_union_mask(w.dim, w.p, w.N, 0)
    assert outside.sum() > 0 and np.array_equal(u1[outside], u0[outside])


def test_cg_to_1e8(c2):
    ctx, prob, _ = c2
    w = prob.workload
    n = (w.p * w.N + 1) ** w.dim
    b = torch.zeros(n, dtype=torch.float64, device="cuda")
    ctx.rhs_manufactured(b)
    x = torch.zeros_like(b)
    it, rel, _ = ctx.solve_cg(b, x, 1e-8, 100)
    assert rel <= 1e-8 and it <= 40
    # the discrete solution approximates sin(pi x) sin(pi y) sin(pi z) at the nodes
    assert float(x.abs().max()) == pytest.approx(1.0, abs=0.05)


# ------------------------------------------------ Q7 48^3 and Q8 64^3, mixed precision
# The FP32 local solves of the variable-coefficient workloads against the FP64
# oracle on sampled colour-0 patches.  Both sides use the oracle's Lanczos
# intervals on the sampled patches (uploaded to the library; the others keep
# fixed ones), so the comparison isolates the arithmetic: the FP32 result must
# agree with the FP64 one to MIXED_TOL relative (max norm over the patch):
# about 150 single-precision roundings (unit 6e-8) along a V-cycle's longest
# dependency chain; measured 4e-7 to 7e-7 on these patches.
MIXED_TOL = 1e-5


@pytest.mark.parametrize("name,precision", [("c3_3d_q7_n48_varcoef", "mixed"), ("c5_3d_q8_n64_varcoef", "mixed"),
                                            ("c3_3d_q7_n48_varcoef", "fp64")])
def test_sweep_sampled_patches_large_degree(name, precision):
    """FP32 (mixed) results within MIXED_TOL of the FP64 oracle, FP64 results
    within 1e-12 (3D degree 8 runs in mixed precision only)."""
    from paper_2510_17785_gb300 import pmg
    w = inputs.WORKLOADS[name]
    prob = inputs.make_problem(w)
    levels = int(np.log2(w.N // w.coarse_N)) + 1
    prec = pmg.PREC_MIXED if precision == "mixed" else pmg.PREC_FP64
    tol = MIXED_TOL if precision == "mixed" else 1e-12
    ctx = pmg.Context(0, precision=prec, bounds=pmg.BOUNDS_FIXED, fixed_lo=0.3, fixed_hi=2.5)
    ctx.mesh_structured(w.dim, w.N, w.p, levels, prob.coords, prob.kappa)
    ctx.setup()
    lf = levels - 1
    verts = [v for v in pt.interior_vertices(w.dim, w.N) if pt.colour_of(v) == 0]
    rng = np.random.default_rng(24)
    pick = [verts[i] for i in rng.choice(len(verts), 8, replace=False)]
    u0 = inputs.random_vector(25, w.dim, w.p, w.N)
    b = inputs.random_vector(26, w.dim, w.p, w.N)
    # oracle first (one pool pass): each sampled patch's update and its Lanczos intervals
    upd = oracle_pool.patch_updates(w.name, pick, u0, b)
    qs = ctx.p_levels()
    lohi = ctx.get_bounds(lf)
    for j, _, _, bd in upd:
        for k, q in enumerate(qs):
            if q > 1:
                lohi[j, k] = bd[q]
    ctx.set_bounds(lf, lohi)
    u = torch.tensor(u0, device="cuda")
    ctx.patch_smooth_colour(lf, 0, torch.tensor(b, device="cuda"), u)
    torch.cuda.synchronize()
    u1 = u.cpu().numpy()
    errs = []
    for j, idx, d, _ in upd:
        errs.append(np.abs((u1[idx] - u0[idx]) - d).max() / np.abs(d).max())
    print(name, precision, "relative error of the patch updates:", errs)
    assert max(errs) < tol, errs
    ctx.close()
