"""Several independent problems of different degrees and sizes solved together
(pmg_batch_solve_cg) against the same problems solved one at a time: the same
iteration counts and solutions, bit for bit (each problem runs the same
kernels in the same order on its own stream)."""
import numpy as np
import pytest

from paper_2510_17785_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problem(k, dim, N, p, levels, **opt):
    from paper_2510_17785_gb300 import pmg
    w = inputs.Workload(f"b{k}", dim, N, p, 0.1 + 0.02 * (k % 7), "sphere", ("loguniform", -2.0, 2.0), "uniform",
                        4000 + k)
    prob = inputs.make_problem(w)
    ctx = pmg.Context(0, precision=pmg.PREC_MIXED, **opt)
    ctx.mesh_structured(dim, N, p, levels, prob.coords, prob.kappa)
    ctx.setup()
    return ctx, torch.tensor(prob.rhs, device="cuda")


# mixed degrees and sizes: 3D degrees 2, 4, 6, 8 and 2D problems
SPECS = [(3, 8, 2, 3), (3, 8, 4, 3), (3, 4, 6, 2), (3, 4, 8, 2), (2, 16, 3, 4), (2, 8, 7, 3), (3, 8, 3, 3),
         (2, 32, 4, 5)]


def test_batch_matches_single_solves():
    from paper_2510_17785_gb300 import pmg
    probs = [_problem(k, *sp) for k, sp in enumerate(SPECS)]
    ref = []
    for ctx, b in probs:
        x = torch.zeros_like(b)
        it, rel, _ = ctx.solve_cg(b, x, 1e-8, 200)
        ref.append((it, rel, x.cpu().numpy()))
    us = [torch.full_like(b, 7.0) for _, b in probs]          # overwritten by the solve
    its, rels, sts = pmg.batch_solve_cg([c for c, _ in probs], [b for _, b in probs], us, 1e-8, 200)
    for k, (it, rel, x) in enumerate(ref):
        assert sts[k] == pmg.PMG_OK and its[k] == it and rels[k] == rel, (k, its[k], it)
        assert np.array_equal(us[k].cpu().numpy(), x), k
    for c, _ in probs:
        c.close()


def test_batch_reports_each_problem():
    from paper_2510_17785_gb300 import pmg
    probs = [_problem(k, *sp) for k, sp in enumerate(SPECS[:3])]
    bs = [b for _, b in probs]
    bs[1] = torch.zeros_like(bs[1])                           # zero right-hand side: 0 iterations
    us = [torch.zeros_like(b) for b in bs]
    its, rels, sts = pmg.batch_solve_cg([c for c, _ in probs], bs, us, 1e-30, 3, check=False)
    assert its[1] == 0 and sts[1] == pmg.PMG_OK and not us[1].any()
    assert its[0] == 3 and sts[0] == pmg.PMG_ERR_NOT_CONVERGED
    assert its[2] == 3 and sts[2] == pmg.PMG_ERR_NOT_CONVERGED
    with pytest.raises(pmg.PMGError):
        pmg.batch_solve_cg([probs[0][0], probs[0][0]], bs[:2], us[:2])   # a context twice
    for c, _ in probs:
        c.close()
