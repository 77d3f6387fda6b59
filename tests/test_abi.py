"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/pmg.h declares.  No GPU: only calls that fail before touching CUDA."""
import ctypes as C
import os
import re

import pytest

import __graft_entry__ as entry
from paper_2510_17785_gb300 import pmg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pmg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    entry.build()
    return pmg.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(pmg.SYMBOLS) == names


def test_default_options(lib):
    o = pmg.default_options()
    assert o.smoother == pmg.SMOOTHER_CHEBYSHEV and o.cheb_degree == 3 and o.n_mg == 1
    assert o.lanczos_steps == 16 and o.bound_safety == 1.1 and o.bound_ratio == 10.0
    assert o.jacobi_omega == 0.5 and o.precision == pmg.PREC_FP64
    # the trailing fields: the ctypes layout matches the C struct to its end
    assert o.additive_theta == 1.0 and o.persistent == 1 and o.sync_budget == 0
    assert o.geometry_bf16 == 0 and o.dense_local == 1
    assert pmg.Options.dense_local.offset + 4 <= C.sizeof(pmg.Options)


def test_argument_validation_without_device(lib):
    h = C.c_void_p()
    assert lib.pmg_create(0, None, None) == 1                       # null out pointer
    bad = pmg.default_options(cheb_degree=0)
    assert lib.pmg_create(0, C.byref(bad), C.byref(h)) == 1
    bad = pmg.default_options(n_mg=0)
    assert lib.pmg_create(0, C.byref(bad), C.byref(h)) == 1
    bad = pmg.default_options(lanczos_steps=65)
    assert lib.pmg_create(0, C.byref(bad), C.byref(h)) == 1
    for kw in (dict(persistent=3), dict(sync_budget=-1), dict(geometry_bf16=1), dict(dense_local=3)):
        bad = pmg.default_options(**kw)                              # geometry_bf16 needs mixed precision
        assert lib.pmg_create(0, C.byref(bad), C.byref(h)) == 1, kw
    assert lib.pmg_destroy(None) == 1
    assert lib.pmg_setup(None) == 1
    assert lib.pmg_sweep_flops(None, 0) == 0.0
    assert lib.pmg_batch_solve_cg(None, -1, None, None, 1e-8, 10, None, None, None) == 1   # negative count
    assert lib.pmg_batch_solve_cg(None, 2, None, None, 1e-8, 10, None, None, None) == 1    # null arrays
    assert lib.pmg_batch_solve_cg(None, 0, None, None, 1e-8, 10, None, None, None) == 0    # empty batch
    nul = (C.c_void_p * 1)(None)
    assert lib.pmg_batch_solve_cg(nul, 1, nul, nul, 1e-8, 10, None, None, None) == 1       # null context


def test_binding_fails_loudly_without_library(tmp_path):
    saved = pmg._lib
    pmg._lib = None
    try:
        with pytest.raises(RuntimeError):
            pmg.load(str(tmp_path / "missing.so"))
    finally:
        pmg._lib = saved
