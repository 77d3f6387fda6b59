"""Oracle patch updates computed in a spawned process pool (test
infrastructure).  The GPU tests compare sampled patches of the full-size
workloads with the oracle; building one oracle patch at degree 7 or 8 takes
seconds, so the samples are spread over the host cores.  The pool is started
with the spawn method: a process forked after the parent has used the GPU can
hang.  This module imports only the oracle and the seeded input generators."""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np


def _update(task):
    from oracle import fem, lanczos as lz, patch as pt
    from paper_2510_17785_gb300 import inputs
    name, v, u0, b, bounds = task
    w = inputs.WORKLOADS[name]
    prob = inputs.make_problem(w)
    m = fem.StructuredMesh(w.dim, w.N, prob.coords, prob.kappa)
    P = pt.Patch(m, v, pt.levels_halving(w.p))
    j = pt.patch_id(w.dim, w.N, v)
    bd = lz.lanczos_bounds_fn(seed=0)(P, j) if bounds is None else bounds
    d = pt.local_solve(P, P.residual(u0, b), pt.Smoother(), bd, 1)
    return j, P.lv[w.p].interior, d, bd


def patch_updates(name, vertices, u0, b, bounds=None):
    """[(patch id, interior DoF ids, oracle update d_j, Lanczos bounds)] of one
    Evaluate + V-cycle per vertex from (u0, b), in the order given; with
    bounds=None each patch uses its own oracle Lanczos intervals."""
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}
    os.environ["OMP_NUM_THREADS"] = os.environ["OPENBLAS_NUM_THREADS"] = "1"
    try:
        n = max(1, min(len(vertices), os.cpu_count() or 1))
        with cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(_update, [(name, tuple(v), u0, b, bounds) for v in vertices]))
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def interior_union_mask(dim, p, N, colour):
    """True on every DoF of the (pN+1)^d grid that lies in the interior of a
    patch of the given Cartesian colour (bit k = parity of the vertex's k-th
    index): per axis, the open interval (p(v-1), p(v+1)) of an interior vertex
    index v of the right parity."""
    axes = []
    for k in range(dim):
        m1 = np.zeros(p * N + 1, dtype=bool)
        for v in range(1, N):
            if v % 2 == (colour >> k) & 1:
                m1[p * (v - 1) + 1: p * (v + 1)] = True
        axes.append(m1)
    mask = axes[0]
    for k in range(1, dim):             # x fastest: flat index = g_x + (pN+1) g_y (+ (pN+1)^2 g_z)
        mask = np.logical_and.outer(axes[k], mask).reshape(-1)
    return mask
