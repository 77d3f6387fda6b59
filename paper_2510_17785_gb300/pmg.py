"""Thin ctypes binding of the C ABI in include/pmg.h.

Argument marshalling only: every numerical step runs in the CUDA kernels of
libpmg.so.  Device vectors are torch CUDA tensors (contiguous float64); the
stream is torch's current stream unless one is given.  There is no CPU
fallback: loading fails loudly if the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpmg.so")

PMG_OK = 0
ERRORS = {1: "PMG_ERR_ARG", 2: "PMG_ERR_CUDA", 3: "PMG_ERR_DEGENERATE", 4: "PMG_ERR_NOT_CONVERGED",
          5: "PMG_ERR_NUMERIC", 6: "PMG_ERR_TIMEOUT", 7: "PMG_ERR_UNSUPPORTED"}
globals().update({name: code for code, name in ERRORS.items()})
SMOOTHER_CHEBYSHEV, SMOOTHER_JACOBI, SMOOTHER_CARTESIAN = 0, 1, 2
BOUNDS_LANCZOS, BOUNDS_FIXED, BOUNDS_USER, BOUNDS_MLP = 0, 1, 2, 3
MLP_NPARAM, MLP_NNORM = 5378, 36
PREC_FP64, PREC_MIXED = 0, 1
NUM_VARIANTS = 16              # PMG_NUM_VARIANTS of include/pmg.h
UMAXC = 32                     # PMG_UMAXC: most cells of an unstructured patch
KAPPA_ARITHMETIC, KAPPA_GEOMETRIC, KAPPA_HARMONIC = 0, 1, 2

# every symbol include/pmg.h declares
SYMBOLS = (
    "pmg_default_options", "pmg_create", "pmg_destroy", "pmg_last_error", "pmg_mesh_structured", "pmg_setup",
    "pmg_num_dofs", "pmg_num_patches", "pmg_p_levels", "pmg_apply", "pmg_patch_smooth", "pmg_patch_smooth_colour",
    "pmg_local_vcycle", "pmg_get_bounds", "pmg_set_bounds", "pmg_compute_bounds", "pmg_get_ritz",
    "pmg_gmg_vcycle", "pmg_solve_cg", "pmg_solve_cg_host", "pmg_rhs_manufactured", "pmg_get_colours",
    "pmg_get_patch_map", "pmg_get_inv_diag", "pmg_sweep_flops", "pmg_launch_count", "pmg_fma_peak",
    "pmg_lanczos_bounds_noalloc", "pmg_tuning", "pmg_default_train_options", "pmg_features", "pmg_mlp_grad",
    "pmg_mlp_train", "pmg_mlp_predict", "pmg_set_mlp", "pmg_solve_gmres", "pmg_batch_solve_cg",
    "pmg_tuning_level", "pmg_coeff_upload", "pmg_mlp_init", "pmg_mlp_targets", "pmg_mlp_norm", "pmg_mlp_save",
    "pmg_mlp_load", "pmg_mesh_upload", "pmg_set_degree", "pmg_get_dof_map", "pmg_local_size",
    "pmg_level_persistent", "pmg_level_dense_local",
)


class Options(C.Structure):
    _fields_ = [
        ("smoother", C.c_int), ("cheb_degree", C.c_int), ("jacobi_omega", C.c_double), ("n_mg", C.c_int),
        ("bounds", C.c_int), ("lanczos_steps", C.c_int), ("bound_safety", C.c_double),
        ("bound_ratio", C.c_double), ("fixed_lo", C.c_double), ("fixed_hi", C.c_double),
        ("seed", C.c_uint64), ("precision", C.c_int), ("autotune", C.c_int), ("variant", C.c_int),
        ("mlp_safety", C.c_double), ("coarse_kappa", C.c_int), ("post_reverse", C.c_int),
        ("additive", C.c_int), ("additive_theta", C.c_double), ("persistent", C.c_int),
        ("sync_budget", C.c_longlong), ("geometry_bf16", C.c_int), ("dense_local", C.c_int),
        ("level_rule", C.c_int),
    ]


class TrainOptions(C.Structure):
    _fields_ = [("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("asym", C.c_float), ("seed", C.c_uint64)]


class PMGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libpmg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpmg.so not found at {path}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    vp, i, d, i64 = C.c_void_p, C.c_int, C.c_double, C.c_int64
    P = C.POINTER
    sig = {
        "pmg_default_options": (None, [P(Options)]),
        "pmg_create": (i, [i, P(Options), P(vp)]),
        "pmg_destroy": (i, [vp]),
        "pmg_last_error": (C.c_char_p, [vp]),
        "pmg_mesh_structured": (i, [vp, i, i, i, i, vp, vp]),
        "pmg_setup": (i, [vp]),
        "pmg_num_dofs": (i, [vp, i, P(i64), P(i64)]),
        "pmg_num_patches": (i, [vp, i, P(i64), P(i)]),
        "pmg_p_levels": (i, [vp, P(i), P(i)]),
        "pmg_apply": (i, [vp, i, vp, vp, vp]),
        "pmg_patch_smooth": (i, [vp, i, vp, vp, i, i, vp]),
        "pmg_patch_smooth_colour": (i, [vp, i, i, vp, vp, vp]),
        "pmg_local_vcycle": (i, [vp, i, i64, vp, vp, vp, i, vp]),
        "pmg_get_bounds": (i, [vp, i, vp]),
        "pmg_set_bounds": (i, [vp, i, vp]),
        "pmg_compute_bounds": (i, [vp, i]),
        "pmg_get_ritz": (i, [vp, i, vp]),
        "pmg_gmg_vcycle": (i, [vp, vp, vp, vp]),
        "pmg_solve_cg": (i, [vp, vp, vp, d, i, P(i), P(d), vp]),
        "pmg_solve_cg_host": (i, [vp, vp, vp, d, i, P(i), P(d), vp]),
        "pmg_rhs_manufactured": (i, [vp, vp, vp]),
        "pmg_get_colours": (i, [vp, i, vp]),
        "pmg_get_patch_map": (i, [vp, i, vp]),
        "pmg_get_inv_diag": (i, [vp, i, i, vp, vp]),
        "pmg_sweep_flops": (d, [vp, i]),
        "pmg_launch_count": (i, [vp, P(i64)]),
        "pmg_fma_peak": (i, [vp, i, P(d)]),
        "pmg_lanczos_bounds_noalloc": (i, [vp, i, i, i64, i64, vp, vp, vp]),
        "pmg_tuning": (i, [vp, P(i), P(i), P(i), P(C.c_float)]),
        "pmg_default_train_options": (None, [P(TrainOptions)]),
        "pmg_features": (i, [vp, i, i, vp, vp]),
        "pmg_mlp_grad": (i, [i, vp, vp, vp, vp, i, C.c_float, vp, vp, vp]),
        "pmg_mlp_train": (i, [i, vp, vp, vp, vp, i64, P(TrainOptions), vp]),
        "pmg_mlp_predict": (i, [i, vp, vp, vp, i64, i, vp, vp]),
        "pmg_set_mlp": (i, [vp, vp, vp]),
        "pmg_solve_gmres": (i, [vp, vp, vp, d, i, i, i, P(i), P(d), vp]),
        "pmg_batch_solve_cg": (i, [vp, i, vp, vp, d, i, P(i), P(d), P(i)]),
        "pmg_tuning_level": (i, [vp, i, P(i), P(C.c_float)]),
        "pmg_coeff_upload": (i, [vp, i, vp]),
        "pmg_mlp_init": (None, [C.c_uint64, vp]),
        "pmg_mlp_targets": (i, [vp, i, i, vp, vp]),
        "pmg_mlp_norm": (i, [i, vp, vp, i64, vp]),
        "pmg_mlp_save": (i, [vp, C.c_char_p]),
        "pmg_mlp_load": (i, [vp, C.c_char_p]),
        "pmg_mesh_upload": (i, [vp, i, i, i64, vp, i64, vp, vp, vp, vp]),
        "pmg_set_degree": (i, [vp, i]),
        "pmg_get_dof_map": (i, [vp, i, vp]),
        "pmg_local_size": (i, [vp, i, P(i64)]),
        "pmg_level_persistent": (i, [vp, i, P(i), P(C.c_float), P(C.c_float)]),
        "pmg_level_dense_local": (i, [vp, i, P(i), P(C.c_float), P(C.c_float)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def default_options(**kw) -> Options:
    lib = load()
    o = Options()
    lib.pmg_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def train_options(**kw) -> TrainOptions:
    lib = load()
    o = TrainOptions()
    lib.pmg_default_train_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _check_rc(rc, what):
    if rc != PMG_OK:
        raise PMGError(rc, what)


def batch_solve_cg(ctxs, bs, us, rtol=1e-8, maxit=200, check=True):
    """pmg_batch_solve_cg over Contexts ctxs with device vectors bs[k], us[k];
    returns (iterations, relres, status) lists."""
    K = len(ctxs)
    if len(bs) != K or len(us) != K:
        raise ValueError("one right-hand side and one solution vector per context")
    lib = load()
    hs = (C.c_void_p * K)(*[c.h for c in ctxs])
    bp = (C.c_void_p * K)(*[_ptr(b) for b in bs])
    up = (C.c_void_p * K)(*[_ptr(u) for u in us])
    it, rel, st = (C.c_int * K)(), (C.c_double * K)(), (C.c_int * K)()
    rc = lib.pmg_batch_solve_cg(hs, K, bp, up, rtol, maxit, it, rel, st)
    if check and rc != PMG_OK:
        bad = [k for k in range(K) if st[k] != PMG_OK]
        k = bad[0] if bad else 0
        msg = lib.pmg_last_error(ctxs[k].h) if ctxs else b""
        raise PMGError(rc, f"problem {k}: " + (msg.decode() if msg else ""))
    return list(it), list(rel), list(st)


def mlp_init(seed: int = 0) -> np.ndarray:
    """Initial MLP parameters from the library (pmg_mlp_init): float32 array of
    MLP_NPARAM values in the library's layout."""
    theta = np.zeros(MLP_NPARAM, dtype=np.float32)
    load().pmg_mlp_init(seed, theta.ctypes.data)
    return theta


def mlp_training_data(ctx):
    """(features X [n, 16], targets T [n, 2]) as float32 CUDA tensors: every
    patch, mesh level and p-level q > 1 of a set-up context with Lanczos
    intervals (pmg_features and pmg_mlp_targets), stacked."""
    import torch
    Xs, Ts = [], []
    for lv in range(ctx.n_levels):
        npatch, _ = ctx.num_patches(lv)
        for k, q in enumerate(ctx.p_levels()):
            if q == 1:
                continue
            X = torch.zeros((npatch, 16), dtype=torch.float32, device="cuda")
            T = torch.zeros((npatch, 2), dtype=torch.float32, device="cuda")
            ctx.features(lv, k, X)
            ctx.mlp_targets(lv, k, T)
            Xs.append(X)
            Ts.append(T)
    return torch.cat(Xs), torch.cat(Ts)


def mlp_norm(X, T, device=0) -> np.ndarray:
    """The MLP_NNORM normalisation floats of a training set (pmg_mlp_norm)."""
    norm = np.zeros(MLP_NNORM, dtype=np.float32)
    _check_rc(load().pmg_mlp_norm(device, _ptr(X), _ptr(T), X.shape[0], norm.ctypes.data), "pmg_mlp_norm")
    return norm


def mlp_grad(params, norm, X, T, asym=4.0, device=0):
    """(loss, grad) of the loss on all samples; float32 CUDA tensors."""
    import torch
    lib = load()
    loss = torch.zeros(1, dtype=torch.float32, device=params.device)
    g = torch.zeros_like(params)
    _check_rc(lib.pmg_mlp_grad(device, _ptr(params), _ptr(norm), _ptr(X), _ptr(T), X.shape[0], asym, _ptr(loss),
                               _ptr(g), _stream(None)), "pmg_mlp_grad")
    return loss, g


def mlp_train(params, norm, X, T, device=0, **opts):
    """Train params (float32 CUDA tensor) in place; returns the per-epoch losses."""
    lib = load()
    o = train_options(**opts)
    hist = np.zeros(max(o.epochs, 1), dtype=np.float32)
    import torch
    torch.cuda.synchronize()
    _check_rc(lib.pmg_mlp_train(device, _ptr(params), _ptr(norm), _ptr(X), _ptr(T), X.shape[0], C.byref(o),
                                hist.ctypes.data), "pmg_mlp_train")
    return hist[: o.epochs]


def mlp_predict(params, norm, X, bf16=True, device=0):
    import torch
    lib = load()
    Y = torch.zeros((X.shape[0], 2), dtype=torch.float32, device=X.device)
    _check_rc(lib.pmg_mlp_predict(device, _ptr(params), _ptr(norm), _ptr(X), X.shape[0], int(bf16), _ptr(Y),
                                  _stream(None)), "pmg_mlp_predict")
    return Y


def _ptr(t) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise TypeError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class Context:
    """A pmg_ctx; methods are the C functions without the ``pmg_`` prefix."""

    def __init__(self, device: int = 0, options: Optional[Options] = None, **kw):
        self.lib = load()
        opt = options if options is not None else default_options(**kw)
        h = C.c_void_p()
        rc = self.lib.pmg_create(device, C.byref(opt), C.byref(h))
        if rc != PMG_OK:
            raise PMGError(rc, "pmg_create failed")
        self.h = h
        self.device = int(device)
        self.options = opt
        self.dim = self.N = self.p = self.n_levels = None

    def _check(self, rc):
        if rc != PMG_OK:
            msg = self.lib.pmg_last_error(self.h)
            raise PMGError(rc, msg.decode() if msg else "")
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.pmg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- mesh / set-up
    def mesh_structured(self, dim: int, N: int, p: int, n_levels: int, coords: np.ndarray, kappa: np.ndarray):
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        kappa = np.ascontiguousarray(kappa, dtype=np.float64)
        if coords.size != (N + 1) ** dim * dim or kappa.size != N ** dim:
            raise ValueError("coords / kappa have the wrong size")
        self._check(self.lib.pmg_mesh_structured(self.h, dim, N, p, n_levels, coords.ctypes.data,
                                                 kappa.ctypes.data))
        self.dim, self.N, self.p, self.n_levels = dim, N, p, n_levels

    def mesh_upload(self, dim: int, coords: np.ndarray, cells: np.ndarray, p: Optional[int] = None,
                    vertex_on_boundary: Optional[np.ndarray] = None, kappa: Optional[np.ndarray] = None,
                    level: int = 0, parent: Optional[np.ndarray] = None, child: Optional[np.ndarray] = None):
        """Unstructured quadrilateral / hexahedral mesh level: coords [n_v][dim],
        cells [n_c][2^dim] vertex ids (lexicographic corner order).  Level 0
        takes the degree p; a finer level gives each cell's parent cell and
        child index in the level below."""
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        nv, nc = coords.shape[0], cells.shape[0]
        if coords.shape != (nv, dim) or cells.shape != (nc, 2 ** dim):
            raise ValueError("coords must be [n_v][dim] and cells [n_c][2^dim]")
        vob = None
        if vertex_on_boundary is not None:
            vob = np.ascontiguousarray(vertex_on_boundary, dtype=np.uint8)
            if vob.shape != (nv,):
                raise ValueError("vertex_on_boundary must hold n_v flags")
        par = ch = None
        if parent is not None or child is not None:
            par = np.ascontiguousarray(parent, dtype=np.int64)
            ch = np.ascontiguousarray(child, dtype=np.uint8)
            if par.shape != (nc,) or ch.shape != (nc,):
                raise ValueError("parent and child must hold n_c entries")
        self._check(self.lib.pmg_mesh_upload(self.h, level, dim, nv, coords.ctypes.data, nc, cells.ctypes.data,
                                             None if vob is None else vob.ctypes.data,
                                             None if par is None else par.ctypes.data,
                                             None if ch is None else ch.ctypes.data))
        if level == 0:
            if p is None:
                raise ValueError("level 0 takes the degree p")
            self._check(self.lib.pmg_set_degree(self.h, p))
            self.p = p
            self.n_cells_levels = []
        self.n_cells_levels.append(nc)
        if kappa is not None:
            self.coeff_upload(level, kappa)
        self.dim, self.N, self.n_levels = dim, None, level + 1
        self.n_cells = nc

    def set_degree(self, p: int):
        self._check(self.lib.pmg_set_degree(self.h, p))
        self.p = p

    def get_dof_map(self, k: int = 0):
        q = self.p_levels()[k]
        out = np.zeros((self.n_cells, (q + 1) ** self.dim), dtype=np.int32)
        self._check(self.lib.pmg_get_dof_map(self.h, k, out.ctypes.data))
        return out

    def local_size(self, level: int) -> int:
        n = C.c_int64()
        self._check(self.lib.pmg_local_size(self.h, level, C.byref(n)))
        return n.value

    def setup(self):
        self._check(self.lib.pmg_setup(self.h))

    def num_dofs(self, level: int):
        t, f = C.c_int64(), C.c_int64()
        self._check(self.lib.pmg_num_dofs(self.h, level, C.byref(t), C.byref(f)))
        return t.value, f.value

    def num_patches(self, level: int):
        n, c = C.c_int64(), C.c_int()
        self._check(self.lib.pmg_num_patches(self.h, level, C.byref(n), C.byref(c)))
        return n.value, c.value

    def p_levels(self):
        arr = (C.c_int * 8)()
        n = C.c_int()
        self._check(self.lib.pmg_p_levels(self.h, arr, C.byref(n)))
        return list(arr[: n.value])

    # ---- operators
    def apply(self, level, u, Au, stream=None):
        self._check(self.lib.pmg_apply(self.h, level, _ptr(u), _ptr(Au), _stream(stream)))

    def patch_smooth(self, level, b, u, n_sweeps=1, reverse=False, stream=None):
        self._check(self.lib.pmg_patch_smooth(self.h, level, _ptr(b), _ptr(u), n_sweeps, int(reverse),
                                              _stream(stream)))

    def patch_smooth_colour(self, level, colour, b, u, stream=None):
        self._check(self.lib.pmg_patch_smooth_colour(self.h, level, colour, _ptr(b), _ptr(u), _stream(stream)))

    def local_vcycle(self, level, patch_ids, r, d, n_cycles=1, stream=None):
        n = patch_ids.numel()
        self._check(self.lib.pmg_local_vcycle(self.h, level, n, _ptr(patch_ids), _ptr(r), _ptr(d), n_cycles,
                                              _stream(stream)))

    def gmg_vcycle(self, b, x, stream=None):
        self._check(self.lib.pmg_gmg_vcycle(self.h, _ptr(b), _ptr(x), _stream(stream)))

    def solve_cg(self, b, u, rtol=1e-8, maxit=200, stream=None, check=True):
        it, rel = C.c_int(), C.c_double()
        rc = self.lib.pmg_solve_cg(self.h, _ptr(b), _ptr(u), rtol, maxit, C.byref(it), C.byref(rel),
                                   _stream(stream))
        if check:
            self._check(rc)
        return it.value, rel.value, rc

    def solve_gmres(self, b, u, rtol=1e-8, maxit=200, restart=50, left=False, stream=None, check=True):
        it, rel = C.c_int(), C.c_double()
        rc = self.lib.pmg_solve_gmres(self.h, _ptr(b), _ptr(u), rtol, maxit, restart, int(bool(left)), C.byref(it),
                                      C.byref(rel), _stream(stream))
        if check:
            self._check(rc)
        return it.value, rel.value, rc

    def solve_cg_host(self, b: np.ndarray, u: np.ndarray, rtol=1e-8, maxit=200, check=True):
        """b, u: host float64 arrays (ideally pinned); copies are part of the call."""
        it, rel = C.c_int(), C.c_double()
        rc = self.lib.pmg_solve_cg_host(self.h, C.c_void_p(b.ctypes.data if isinstance(b, np.ndarray) else b),
                                        C.c_void_p(u.ctypes.data if isinstance(u, np.ndarray) else u),
                                        rtol, maxit, C.byref(it), C.byref(rel), None)
        if check:
            self._check(rc)
        return it.value, rel.value, rc

    def rhs_manufactured(self, b, stream=None):
        self._check(self.lib.pmg_rhs_manufactured(self.h, _ptr(b), _stream(stream)))

    # ---- bounds and integer structures
    def get_bounds(self, level):
        n, _ = self.num_patches(level)
        out = np.zeros((n, len(self.p_levels()), 2))
        self._check(self.lib.pmg_get_bounds(self.h, level, out.ctypes.data))
        return out

    def get_ritz(self, level):
        n, _ = self.num_patches(level)
        out = np.zeros((n, len(self.p_levels()), 2))
        self._check(self.lib.pmg_get_ritz(self.h, level, out.ctypes.data))
        return out

    def set_bounds(self, level, lohi: np.ndarray):
        lohi = np.ascontiguousarray(lohi, dtype=np.float64)
        self._check(self.lib.pmg_set_bounds(self.h, level, lohi.ctypes.data))

    def compute_bounds(self, source):
        self._check(self.lib.pmg_compute_bounds(self.h, source))

    def get_colours(self, level):
        n, _ = self.num_patches(level)
        out = np.zeros(n, dtype=np.uint8)
        self._check(self.lib.pmg_get_colours(self.h, level, out.ctypes.data))
        return out

    def get_patch_map(self, level):
        n, _ = self.num_patches(level)
        width = 2 ** self.dim + 1 if self.N is not None else 1 + UMAXC
        out = np.zeros((n, width), dtype=np.int64)
        self._check(self.lib.pmg_get_patch_map(self.h, level, out.ctypes.data))
        return out

    def get_inv_diag(self, level, k, out, stream=None):
        self._check(self.lib.pmg_get_inv_diag(self.h, level, k, _ptr(out), _stream(stream)))

    def sweep_flops(self, level) -> float:
        return self.lib.pmg_sweep_flops(self.h, level)

    def tuning(self):
        """(variant, threads per CTA, patches per CTA, [ms per candidate variant])"""
        v, t, b = C.c_int(), C.c_int(), C.c_int()
        ms = (C.c_float * NUM_VARIANTS)()
        self._check(self.lib.pmg_tuning(self.h, C.byref(v), C.byref(t), C.byref(b), ms))
        return v.value, t.value, b.value, list(ms)

    def level_persistent(self, level):
        """(persistent sweeps on mesh level `level`?, set-up ms per-colour, ms persistent)"""
        on, a, b = C.c_int(), C.c_float(), C.c_float()
        self._check(self.lib.pmg_level_persistent(self.h, level, C.byref(on), C.byref(a), C.byref(b)))
        return bool(on.value), a.value, b.value

    def level_dense_local(self, level):
        """(tabulated local solves on mesh level `level`?, set-up ms matrix-free, ms tabulated)"""
        on, a, b = C.c_int(), C.c_float(), C.c_float()
        self._check(self.lib.pmg_level_dense_local(self.h, level, C.byref(on), C.byref(a), C.byref(b)))
        return bool(on.value), a.value, b.value

    def tuning_level(self, level):
        """(variant used on mesh level `level`, [set-up ms per candidate variant])"""
        v = C.c_int()
        ms = (C.c_float * NUM_VARIANTS)()
        self._check(self.lib.pmg_tuning_level(self.h, level, C.byref(v), ms))
        return v.value, list(ms)

    def features(self, level, k, X, stream=None):
        self._check(self.lib.pmg_features(self.h, level, k, _ptr(X), _stream(stream)))

    def mlp_targets(self, level, k, T, stream=None):
        self._check(self.lib.pmg_mlp_targets(self.h, level, k, _ptr(T), _stream(stream)))

    def mlp_save(self, path: str):
        self._check(self.lib.pmg_mlp_save(self.h, os.fsencode(path)))

    def mlp_load(self, path: str):
        self._check(self.lib.pmg_mlp_load(self.h, os.fsencode(path)))

    def coeff_upload(self, level: int, kappa: np.ndarray):
        kappa = np.ascontiguousarray(kappa, dtype=np.float64)
        self._check(self.lib.pmg_coeff_upload(self.h, level, kappa.ctypes.data))

    def set_mlp(self, params: np.ndarray, norm: np.ndarray):
        params = np.ascontiguousarray(params, dtype=np.float32)
        norm = np.ascontiguousarray(norm, dtype=np.float32)
        self._check(self.lib.pmg_set_mlp(self.h, params.ctypes.data, norm.ctypes.data))

    def launch_count(self) -> int:
        n = C.c_int64()
        self._check(self.lib.pmg_launch_count(self.h, C.byref(n)))
        return n.value

    def lanczos_bounds_noalloc(self, level, k, first_patch, n_patches, ritz, bounds, stream=None):
        """Lanczos intervals for a patch range without any device allocation
        (see include/pmg.h); ritz and bounds are contiguous float64 CUDA
        tensors of at least n_patches x 2 values on the context's device.
        The C side receives bare pointers and cannot check their size or type,
        so this wrapper does, before the call."""
        import torch
        for name, t in (("ritz", ritz), ("bounds", bounds)):
            if not hasattr(t, "is_cuda") or not t.is_cuda:
                raise TypeError(f"{name} must be a CUDA tensor")
            if t.dtype != torch.float64:
                raise TypeError(f"{name} must be float64, got {t.dtype}")
            if t.device.index != self.device:
                raise ValueError(f"{name} is on cuda:{t.device.index}, the context on cuda:{self.device}")
            if t.numel() < 2 * int(n_patches):
                raise ValueError(f"{name} holds {t.numel()} values, needs 2 * n_patches = {2 * int(n_patches)}")
        self._check(self.lib.pmg_lanczos_bounds_noalloc(self.h, level, k, first_patch, n_patches, _ptr(ritz),
                                                        _ptr(bounds), _stream(stream)))

    def fma_peak(self, precision) -> float:
        f = C.c_double()
        self._check(self.lib.pmg_fma_peak(self.h, precision, C.byref(f)))
        return f.value
