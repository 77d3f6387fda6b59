"""The seeded input generator shared by the oracle and the library: the same
seed gives the same mesh, coefficient and right-hand side; every workload's
perturbed mesh has positive corner volumes; the perturbation laws keep their
stated amplitude; boundary vertices stay on the boundary."""
import numpy as np
import pytest

from paper_2510_17785_gb300 import inputs


@pytest.mark.parametrize("name", sorted(inputs.WORKLOADS))
def test_workloads_are_reproducible_and_valid(name):
    w = inputs.WORKLOADS[name]
    a, b = inputs.make_problem(w), inputs.make_problem(w)
    assert np.array_equal(a.coords, b.coords) and np.array_equal(a.kappa, b.kappa)
    assert (a.rhs is None and b.rhs is None) or np.array_equal(a.rhs, b.rhs)
    vol = inputs.corner_volumes(a.coords, w.dim, w.N)
    assert vol.min() > 0.0
    assert a.coords.shape == ((w.N + 1) ** w.dim, w.dim) and a.kappa.shape == (w.N ** w.dim,)
    assert np.all(a.kappa > 0)


@pytest.mark.parametrize("law", ["uniform", "sphere"])
def test_perturbation_amplitude_and_boundary(law):
    rng = np.random.default_rng(5)
    dim, N, frac = 3, 6, 0.3
    disp = inputs.perturbation(rng, dim, N, frac, law)
    inner = inputs.interior_vertex_mask(dim, N)
    assert np.all(disp[~inner] == 0.0)
    h = 1.0 / N
    if law == "uniform":
        assert np.abs(disp[inner]).max() <= frac * h
    else:
        assert np.allclose(np.linalg.norm(disp[inner], axis=1), frac * h)


def test_different_seeds_differ():
    w = inputs.C2
    a = inputs.make_problem(w)
    b = inputs.make_problem(w.with_(seed=w.seed + 1))
    assert not np.array_equal(a.coords, b.coords)


def test_kershaw_type_mesh():
    """The Kershaw-type generator keeps the boundary on itself, is the uniform
    grid at eps = 1, has positive corner volumes at eps = 0.3 (cell sizes in a
    ratio of (2 - eps) / eps along y), and needs N divisible by 3."""
    import numpy as np
    for dim in (2, 3):
        N = 12
        g = inputs.grid_vertices(dim, N)
        assert np.allclose(inputs.kershaw_vertices(dim, N, 1.0), g, atol=1e-15)
        x = inputs.kershaw_vertices(dim, N, 0.3)
        bnd = ~inputs.interior_vertex_mask(dim, N)
        on_bnd = np.any((x[bnd] < 1e-14) | (x[bnd] > 1 - 1e-14), axis=1)
        assert on_bnd.all()
        assert inputs.corner_volumes(x, dim, N).min() > 0
        col = x[:N + 1, :]                                 # the first x-row: y = 0 edge (x varies)
        assert np.allclose(col[:, 0], g[:N + 1, 0])
        ys = np.sort(np.unique(np.round(x[x[:, 0] == 0.0][:, 1], 14)))
        h = np.diff(ys)
        assert abs(h.max() / h.min() - (2 - 0.3) / 0.3) < 1e-9
    try:
        inputs.kershaw_vertices(2, 8, 0.3)
    except ValueError:
        pass
    else:
        raise AssertionError("N = 8 accepted")
