"""Pins of the unstructured-mesh oracle (oracle/unstructured.py) against what
the mathematics fixes: the structured oracle on the same geometry with the
cells' corners listed in arbitrary orientations (numbering and orientation of
shared edges and faces), the patch test (linear functions), principal
submatrices, the Galerkin identity of the p-levels on affine patches, the
colouring's defining properties and a brute-force sweep.  No GPU."""
import itertools

import numpy as np
import pytest

from oracle import fem, lanczos as lz, patch as pt, unstructured as us
from paper_2510_17785_gb300 import inputs


def _symmetries(dim):
    """The orientation-preserving symmetries (rotations) of the reference cell
    as corner permutations: corner c of the image is corner sigma(c) of the
    original."""
    out = []
    for perm in itertools.permutations(range(dim)):
        sign = np.linalg.det(np.eye(dim)[list(perm)])
        for flip in range(2 ** dim):
            if sign * (-1) ** bin(flip).count("1") < 0:
                continue
            m = []
            for c in range(2 ** dim):
                bits = [(c >> perm[k]) & 1 for k in range(dim)]
                bits = [b ^ ((flip >> k) & 1) for k, b in enumerate(bits)]
                m.append(sum(b << k for k, b in enumerate(bits)))
            out.append(m)
    return out


def _structured_as_unstructured(dim, N, seed, kappa=None, perturb=0.2, permute=True):
    w = inputs.Workload("u", dim, N, 1, perturb, "uniform", ("loguniform", -1, 1), "uniform", seed)
    prob = inputs.make_problem(w)
    sm = fem.StructuredMesh(dim, N, prob.coords, prob.kappa if kappa is None else kappa)
    rng = np.random.default_rng(seed + 1)
    syms = _symmetries(dim)
    cells = []
    for ci in range(sm.n_cells):
        c = sm.cell_multi(ci)
        ids = [sum((c[k] + ((v >> k) & 1)) * (N + 1) ** k for k in range(dim)) for v in range(2 ** dim)]
        s = syms[rng.integers(len(syms))] if permute else list(range(2 ** dim))
        cells.append([ids[s[v]] for v in range(2 ** dim)])
    return sm, us.Mesh(dim, prob.coords, cells, sm.kappa)


def _match(Xa, Xb):
    """perm with Xa[perm[i]] == Xb[i] (positions matched to 1e-12)."""
    ka = {tuple(np.round(x, 10)): i for i, x in enumerate(Xa)}
    return np.array([ka[tuple(np.round(x, 10))] for x in Xb])


@pytest.mark.parametrize("dim,N,q", [(2, 3, 1), (2, 3, 3), (2, 2, 4), (3, 2, 1), (3, 2, 2), (3, 2, 3)])
def test_numbering_and_orientation_against_structured_oracle(dim, N, q):
    """Cells given in random orientations (any symmetry of the reference cell)
    assemble the same global matrix as the structured oracle, DoFs matched by
    their physical positions: shared edge and face nodes are identified
    consistently whatever the local orientation."""
    sm, um = _structured_as_unstructured(dim, N, 3 + q)
    As = sm.assemble(q).toarray()
    Au = um.assemble(q).toarray()
    assert um.n_dofs(q) == sm.n_nodes(q)
    perm = _match(um.node_coords(q), sm.node_coords(q))
    assert sorted(perm) == list(range(len(perm)))
    assert np.abs(Au[np.ix_(perm, perm)] - As).max() <= 1e-12 * np.abs(As).max()
    # boundary DoFs are the structured grid's Dirichlet nodes
    assert np.array_equal(um.boundary_dofs(q)[perm], ~sm.free_mask(q))


def _meshes():
    p, t = inputs.triangulated_square(3, 5)
    X, C = inputs.triangles_to_quads(p, t)
    yield "2d_trisplit", us.Mesh(2, X, C, 10.0 ** np.random.default_rng(1).uniform(-1, 1, len(C)))
    X3, C3 = inputs.extrude(X, C, 2)
    yield "3d_extruded", us.Mesh(3, X3, C3, np.ones(len(C3)))
    pt4, tt = inputs.cube_tetrahedra(1, 3)
    X4, C4 = inputs.tetrahedra_to_hexes(pt4, tt)
    yield "3d_tetsplit", us.Mesh(3, X4, C4, 10.0 ** np.random.default_rng(2).uniform(-1, 1, len(C4)))


@pytest.mark.parametrize("name", ["2d_trisplit", "3d_extruded", "3d_tetsplit"])
def test_patch_test_and_symmetry(name):
    """With constant kappa a linear function u = a.x + c (in Q_q under the Q1
    geometry) satisfies (A u)_i = 0 on every interior DoF; A is symmetric,
    positive on the free DoFs and annihilates constants."""
    m = dict(_meshes())[name]
    m = us.Mesh(m.dim, m.coords, m.cells, np.full(m.nc, 2.5))
    for q in (1, 2, 3):
        A = m.assemble(q).toarray()
        X = m.node_coords(q)
        a = np.array([0.3, -1.1, 0.7][: m.dim])
        u = X @ a + 0.4
        free = ~m.boundary_dofs(q)
        assert np.abs((A @ u)[free]).max() <= 1e-12 * np.abs(A).max() * np.abs(u).max()
        assert np.abs(A @ np.ones(len(u))).max() <= 1e-12 * np.abs(A).max()
        assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
        Af = A[np.ix_(free, free)]
        assert np.linalg.eigvalsh(Af).min() > 0


@pytest.mark.parametrize("name", ["2d_trisplit", "3d_extruded", "3d_tetsplit"])
def test_patch_matrices_are_principal_submatrices(name):
    m = dict(_meshes())[name]
    q = 2
    A = m.assemble(q).toarray()
    vs = m.interior_vertices()
    for v in vs[:: max(1, len(vs) // 5)]:
        P = us.Patch(m, v, [q])
        I = P.lv[q].interior
        assert len(I) > 0
        assert np.abs(P.lv[q].A - A[np.ix_(I, I)]).max() <= 1e-13 * np.abs(A).max()
        # Evaluate (eq. main:4) is the global residual restricted to the interior
        rng = np.random.default_rng(v)
        u = rng.uniform(-1, 1, len(A)) * ~m.boundary_dofs(q)
        b = rng.uniform(-1, 1, len(A))
        assert np.allclose(P.residual(u, b), (b - A @ u)[I], atol=1e-12)
        # interior DoFs lie in patch cells only
        owners = m.dof_cells(q)
        assert all(set(owners[g]) <= set(P.cells) for g in I)


def test_valences_of_the_generated_meshes():
    """The generators reach the valences of the unstructured workload: 3 and 5
    in 2D (triangle split), 4 and 6 (tetrahedron split), 8, 10 and 12
    (extrusion)."""
    vals = set()
    for name, m in _meshes():
        vals |= {(m.dim, m.valence(v)) for v in m.interior_vertices()}
    for need in ((2, 3), (2, 5), (3, 4), (3, 6), (3, 8), (3, 10), (3, 12)):
        assert need in vals, need


@pytest.mark.parametrize("p", [2, 4])
def test_galerkin_identity_on_affine_unstructured_patches(p):
    """On patches of parallelogram cells with constant kappa, in arbitrary
    orientations, the re-evaluated coarse operator equals P^T A_p P
    (Section 3.1, level operators); the p-embedding is exact on the coarse
    space."""
    for dim in (2, 3):
        sm, um = _structured_as_unstructured(dim, 3, 7, kappa=np.full(3 ** dim, 1.7), perturb=0.0)
        for v in um.interior_vertices():
            P = us.Patch(um, v, pt.levels_halving(p))
            for (qc, qf), E in P.P.items():
                Af, Ac = P.lv[qf].A, P.lv[qc].A
                assert np.abs(E.T @ Af @ E - Ac).max() <= 1e-12 * np.abs(Ac).max()


def test_colours_are_valid_and_greedy():
    for name, m in _meshes():
        col = us.colours(m, seed=0)
        assert set(col) == set(m.interior_vertices())
        # no two patches of one colour share a cell
        for c in range(m.nc):
            cs = [col[int(v)] for v in m.cells[c] if int(v) in col]
            assert len(cs) == len(set(cs)), name
        # greedy: each colour is the smallest one not taken by a conflicting patch of higher priority
        pri = {v: (lz.splitmix64(v), v) for v in col}
        for v in col:
            nb = {int(w) for c in m.vertex_cells[v] for w in m.cells[c] if int(w) in col and int(w) != v}
            taken = {col[w] for w in nb if pri[w] > pri[v]}
            k = 0
            while k in taken:
                k += 1
            assert col[v] == k


def test_sweep_brute_force_on_an_unstructured_mesh():
    """One colour-major sweep equals u <- u + Pi_j^T B_j (b - A u)_j applied
    patch after patch in that order, with B_j each patch's V-cycle operator and
    A the assembled global matrix."""
    p, t = inputs.triangulated_square(2, 8)
    X, C = inputs.triangles_to_quads(p, t)
    m = us.Mesh(2, X, C, 10.0 ** np.random.default_rng(3).uniform(-1, 1, len(C)))
    q = 2
    S = us.PatchSmoother(m, q, bounds_fn=lz.exact_bounds_fn())
    A = m.assemble(q).toarray()
    free = ~m.boundary_dofs(q)
    rng = np.random.default_rng(4)
    u = rng.uniform(-1, 1, len(A)) * free
    b = rng.uniform(-1, 1, len(A)) * free
    ref = u.copy()
    for c in range(S.n_colours):
        for v in sorted(S.col):
            if S.col[v] != c:
                continue
            P = S.patch(v)
            I = P.lv[q].interior
            B = pt.vcycle_matrix(P, S.sm, S.bounds(v))
            ref[I] += B @ (b - A @ ref)[I]
    assert np.allclose(S.sweep(u, b), ref, atol=1e-12)


def test_q1_embedding_and_two_level_cg():
    """The Q1 embedding reproduces linear functions exactly at every DoF; the
    two-level preconditioner (patch sweeps, Q1 coarse space) is symmetric and
    CG with it reaches 1e-8 and agrees with a sparse direct solve."""
    import scipy.sparse.linalg as spla
    from oracle import gmg
    for name, m in _meshes():
        q = 2
        P = us.q1_prolongation(m, q)
        a = np.array([0.3, -1.1, 0.7][: m.dim])
        lin1 = m.coords @ a + 0.2
        linq = m.node_coords(q) @ a + 0.2
        assert np.abs(P @ lin1 - linq).max() < 1e-13
        S = us.PatchSmoother(m, q, bounds_fn=lz.lanczos_bounds_fn(seed=0))
        T = us.TwoLevel(m, q, S)
        free = T.free
        rng = np.random.default_rng(5)
        b = rng.uniform(-1, 1, len(free)) * free
        y1, y2 = rng.uniform(-1, 1, len(b)) * free, rng.uniform(-1, 1, len(b)) * free
        assert abs(y1 @ T.vcycle(y2) - y2 @ T.vcycle(y1)) < 1e-11 * abs(y1 @ T.vcycle(y1)), name
        x, it, hist = gmg.pcg(T.A, b, T.vcycle, 1e-8, 60)
        assert hist[-1] <= 1e-8 and it <= 30, (name, it)
        ref = np.zeros_like(b)
        ref[free] = spla.spsolve(T.A.tocsr()[free][:, free].tocsc(), b[free])
        assert np.linalg.norm(x - ref) < 1e-6 * np.linalg.norm(ref), name


def _affine_mesh(dim, N, seed):
    """A structured grid under a global affine map (every cell a
    parallelogram / parallelepiped), cells listed in random orientations."""
    sm, um = _structured_as_unstructured(dim, N, seed, perturb=0.0)
    Amap = np.eye(dim) + 0.3 * np.random.default_rng(seed).uniform(-1, 1, (dim, dim))
    return us.Mesh(dim, um.coords @ Amap.T, um.cells, np.full(um.nc, 1.7))


@pytest.mark.parametrize("q", [1, 2, 3])
def test_h_embedding_is_exact_on_linear_functions(q):
    """On the unperturbed refinement of any Q1 mesh the geometry is nested:
    a physically linear function is in both spaces and the embedding maps
    its coarse interpolant to its fine one."""
    for name, m in _meshes():
        Xf, Cf, par, ch = inputs.refine_unstructured(m.coords, m.cells)
        f = us.Mesh(m.dim, Xf, Cf, np.ones(len(Cf)))
        P = us.h_prolongation(m, f, par, ch, q)
        a = np.array([0.7, -0.4, 1.3][: m.dim])
        uc = m.node_coords(q) @ a + 0.25
        uf = f.node_coords(q) @ a + 0.25
        assert np.abs(P @ uc - uf).max() <= 1e-12, name


@pytest.mark.parametrize("dim,q", [(2, 2), (2, 3), (3, 2)])
def test_h_galerkin_identity_on_affine_meshes(dim, q):
    """Parallelogram cells and constant kappa: the coarse matrix equals
    P^T A_fine P (exact quadrature, nested spaces)."""
    m = _affine_mesh(dim, 3 if dim == 2 else 2, 5 + q)
    Xf, Cf, par, ch = inputs.refine_unstructured(m.coords, m.cells)
    f = us.Mesh(dim, Xf, Cf, np.full(len(Cf), 1.7))
    P = us.h_prolongation(m, f, par, ch, q).toarray()
    Ac, Af = m.assemble(q).toarray(), f.assemble(q).toarray()
    assert np.abs(P.T @ Af @ P - Ac).max() <= 1e-11 * np.abs(Ac).max()


def test_two_mesh_level_cycle_is_symmetric_and_preconditions_cg():
    P0, T0 = inputs.triangulated_square(2, 3)
    X, C = inputs.triangles_to_quads(P0, T0)
    Xf, Cf, par, ch = inputs.refine_unstructured(X, C)
    rng = np.random.default_rng(4)
    mc = us.Mesh(2, X, C, 10.0 ** rng.uniform(-1, 1, len(C)))
    mf = us.Mesh(2, Xf, Cf, np.repeat(mc.kappa, 4))
    p = 3
    H = us.TwoMeshLevels(mc, mf, par, ch, p,
                         us.PatchSmoother(mf, p, bounds_fn=lz.lanczos_bounds_fn(seed=0)),
                         us.PatchSmoother(mc, p, bounds_fn=lz.lanczos_bounds_fn(seed=0)))
    free = H.free
    x = rng.uniform(-1, 1, len(free)) * free
    y = rng.uniform(-1, 1, len(free)) * free
    assert abs(x @ H.vcycle(y) - y @ H.vcycle(x)) <= 1e-10 * abs(x @ H.vcycle(x))
    from oracle import gmg
    b = rng.uniform(-1, 1, len(free)) * free
    _, it, hist = gmg.pcg(H.A, b, H.vcycle, 1e-8, 60)
    assert hist[-1] <= 1e-8 and it < 30
