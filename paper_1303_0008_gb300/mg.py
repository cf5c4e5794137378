"""Thin ctypes binding of libmg (include/mg.h), same names as the C-ABI.

Only argument marshalling lives here: every step of the solve runs in the CUDA
library.  Arrays may be numpy arrays (host, float64, C-contiguous) or torch
tensors (float64, contiguous; CUDA tensors are passed as device pointers and
ordered on the handle's stream).  A missing library raises: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmg.so")

MG_OK, MG_EINVAL, MG_ENOMEM, MG_ECUDA, MG_ENOCONV, MG_ENAN, MG_ETIMEOUT, MG_ESTATE = range(8)
MG_FP64, MG_MIXED = 0, 1
MG_GUARD_FLOOR, MG_GUARD_ROOT = 0, 1
STATUS_NAMES = {0: "MG_OK", 1: "MG_EINVAL", 2: "MG_ENOMEM", 3: "MG_ECUDA", 4: "MG_ENOCONV",
                5: "MG_ENAN", 6: "MG_ETIMEOUT", 7: "MG_ESTATE"}


class MGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class mg_options(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int),
                ("coarsest", ctypes.c_int), ("max_cycles", ctypes.c_int),
                ("inner_cycles", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("coarse_sweeps", ctypes.c_int), ("coarse_drop", ctypes.c_double),
                ("time_kernels", ctypes.c_int), ("guard", ctypes.c_int),
                ("patch_coarse_sweeps", ctypes.c_int), ("fuse_coarse", ctypes.c_int),
                ("omega", ctypes.c_double), ("omega_patch", ctypes.c_double),
                ("patch_mg_levels", ctypes.c_int), ("patch_cgc", ctypes.c_double),
                ("sweep32", ctypes.c_int), ("pair32", ctypes.c_int),
                ("tau_stop", ctypes.c_double), ("w", ctypes.c_double),
                ("patch_galerkin", ctypes.c_int), ("half32", ctypes.c_int),
                ("barrier_timeout_s", ctypes.c_double), ("slab32", ctypes.c_int),
                ("tile32", ctypes.c_int)]


class mg_solve_stats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("outer", ctypes.c_int), ("status", ctypes.c_int),
                ("levels", ctypes.c_int), ("res0", ctypes.c_double), ("res", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("wall_s", ctypes.c_double),
                ("guard_hits", ctypes.c_longlong), ("hist_len", ctypes.c_int),
                ("res_hist", ctypes.c_double * 128), ("launches", ctypes.c_longlong),
                ("kernel_launches", ctypes.c_longlong), ("kernel_ms", ctypes.c_double),
                ("kernel_cells", ctypes.c_double), ("tau", ctypes.c_double)]

    def as_dict(self):
        return {"cycles": self.cycles, "outer": self.outer, "status": self.status,
                "levels": self.levels, "res0": self.res0, "res": self.res,
                "lambda": self.lambda_, "wall_s": self.wall_s, "guard_hits": self.guard_hits,
                "hist": list(self.res_hist[:self.hist_len]), "launches": self.launches,
                "kernel_launches": self.kernel_launches, "kernel_ms": self.kernel_ms,
                "kernel_cells": self.kernel_cells, "tau": self.tau}


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.c_int
_F = ctypes.c_double

_SIGS = {
    "mg_default_options": (None, [ctypes.POINTER(mg_options)]),
    "mg_create_grid": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(mg_options)]),
    "mg_set_stream": (_I, [_P, _P]),
    "mg_add_patches": (_I, [_P, _I, _I, ctypes.POINTER(ctypes.c_int32)]),
    "mg_set_density": (_I, [_P, _I, _I, _P, _I]),
    "mg_set_field": (_I, [_P, _I, _I, _P, _I]),
    "mg_solve": (_I, [_P, _I, _F, _F, _F, ctypes.POINTER(mg_solve_stats)]),
    "mg_get_field": (_I, [_P, _I, _I, _P, _I]),
    "mg_get_force": (_I, [_P, _I, _I, _P, _I]),
    "mg_get_density": (_I, [_P, _I, _I, _P, _I]),
    "mg_solve_newton": (_I, [_P, _F, _F, ctypes.POINTER(mg_solve_stats)]),
    "mg_assign_density": (_I, [_P, _I, _I, ctypes.c_longlong, _P, _P, _I]),
    "mg_refine_blocks": (_I, [_P, _I, _F, _F, ctypes.POINTER(ctypes.c_int32), _I,
                              ctypes.POINTER(ctypes.c_int)]),
    "mg_get_newton_field": (_I, [_P, _I, _I, _P, _I]),
    "mg_get_total_force": (_I, [_P, _I, _I, _P, _I]),
    "mg_destroy_grid": (None, [_P]),
    "mg_last_error": (ctypes.c_char_p, []),
    "mg_create_batch": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(mg_options)]),
    "mg_solve_batch": (_I, [_P, ctypes.POINTER(ctypes.c_int), _D, _D, _F,
                            ctypes.POINTER(mg_solve_stats)]),
    "mg_op_residual": (_I, [_I, _P, _P, _P, _I, _F, _F, _P, _D, _P]),
    "mg_op_smooth": (_I, [_I, _P, _P, _P, _I, _F, _F, _F, _I, _P]),
    "mg_op_restrict": (_I, [_I, _P, _P, _P]),
    "mg_op_prolong_correct": (_I, [_I, _P, _P, _P, _P]),
    "mg_op_force": (_I, [_I, _P, _P, _P]),
    "mg_op_residual_noalloc": (_I, [_I, _P, _P, _P, _I, _F, _F, _P, _D, _P]),
    "mg_get_options": (_I, [_P, ctypes.POINTER(mg_options)]),
    "mg_get_level_stats": (_I, [_P, _I, ctypes.POINTER(mg_solve_stats)]),
    "mg_set_options": (_I, [_P, ctypes.POINTER(mg_options)]),
    "mg_autotune": (_I, [_P, _I, _F, _F, _F, ctypes.c_char_p, _I, ctypes.POINTER(mg_options), _D]),
    "mg_slab_order": (_I, [_I, _I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                           ctypes.POINTER(ctypes.c_int), _I, ctypes.POINTER(ctypes.c_int)]),
}


def lib():
    """Load libmg.so (built in-tree by paper_1303_0008_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libmg.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def mg_last_error() -> str:
    return lib().mg_last_error().decode()


def _check(st, what):
    if st != MG_OK:
        raise MGError(st, f"{what}: {mg_last_error()}")


def _arr(x, writable=False):
    """(pointer, on_device, size) of a float64 numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise TypeError("numpy arrays must be float64 and C-contiguous")
        if writable and not x.flags["WRITEABLE"]:
            raise TypeError("output array is read-only")
        return x.ctypes.data, 0, x.size
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("tensors must be float64 and contiguous")
        return x.data_ptr(), int(x.is_cuda), x.numel()
    raise TypeError(f"unsupported array type {type(x)}")


def _dev(x):
    """Device pointer of a CUDA tensor (None passes NULL)."""
    if x is None:
        return None
    p, on_dev, _ = _arr(x)
    if not on_dev:
        raise TypeError("this entry point takes device tensors")
    return p


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def options(**kw) -> mg_options:
    o = mg_options()
    lib().mg_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def mg_create_grid(n: int, opt: mg_options | None = None):
    h = _P()
    _check(lib().mg_create_grid(ctypes.byref(h), n, ctypes.byref(opt) if opt else None),
           "mg_create_grid")
    return h


def mg_create_batch(ns, opt: mg_options | None = None):
    h = _P()
    arr = (ctypes.c_int * len(ns))(*ns)
    _check(lib().mg_create_batch(ctypes.byref(h), len(ns), arr, ctypes.byref(opt) if opt else None),
           "mg_create_batch")
    return h


def mg_set_stream(g, stream=None):
    _check(lib().mg_set_stream(g, _stream(stream)), "mg_set_stream")


def mg_add_patches(g, level: int, origins):
    o = np.ascontiguousarray(origins, dtype=np.int32).reshape(-1, 3)
    _check(lib().mg_add_patches(g, level, o.shape[0],
                                o.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
           "mg_add_patches")


def mg_set_density(g, level: int, patch: int, delta):
    p, dev, _ = _arr(delta)
    _check(lib().mg_set_density(g, level, patch, p, dev), "mg_set_density")


def mg_set_field(g, level: int, patch: int, phi):
    """phi = None (refinement levels, patch -1): the next solve starts the level
    from the interpolation of the level below."""
    if phi is None:
        _check(lib().mg_set_field(g, level, patch, None, 0), "mg_set_field")
        return
    p, dev, _ = _arr(phi)
    _check(lib().mg_set_field(g, level, patch, p, dev), "mg_set_field")


def mg_solve(g, branch: int, alpha: float, kappa: float, tol: float, check: bool = True):
    st = mg_solve_stats()
    rc = lib().mg_solve(g, branch, alpha, kappa, tol, ctypes.byref(st))
    if check and rc not in (MG_OK,):
        raise MGError(rc, f"mg_solve: {mg_last_error()}")
    d = st.as_dict()
    d["rc"] = rc
    return d


def mg_solve_batch(g, branch, alpha, kappa, tol: float, check: bool = True):
    n = len(branch)
    b = (ctypes.c_int * n)(*branch)
    a = (ctypes.c_double * n)(*alpha)
    k = (ctypes.c_double * n)(*kappa)
    stats = (mg_solve_stats * n)()
    rc = lib().mg_solve_batch(g, b, a, k, tol, stats)
    if check and rc != MG_OK:
        raise MGError(rc, f"mg_solve_batch: {mg_last_error()}")
    out = [s.as_dict() for s in stats]
    return rc, out


def mg_get_field(g, level: int, patch: int, out):
    p, dev, _ = _arr(out, writable=True)
    _check(lib().mg_get_field(g, level, patch, p, dev), "mg_get_field")
    return out


def mg_get_density(g, level: int, patch: int, out):
    p, dev, _ = _arr(out, writable=True)
    _check(lib().mg_get_density(g, level, patch, p, dev), "mg_get_density")
    return out


def mg_get_force(g, level: int, patch: int, out):
    p, dev, _ = _arr(out, writable=True)
    _check(lib().mg_get_force(g, level, patch, p, dev), "mg_get_force")
    return out


def mg_solve_newton(g, coef: float, tol: float, check: bool = True):
    st = mg_solve_stats()
    rc = lib().mg_solve_newton(g, coef, tol, ctypes.byref(st))
    if check and rc != MG_OK:
        raise MGError(rc, f"mg_solve_newton: {mg_last_error()}")
    d = st.as_dict()
    d["rc"] = rc
    return d


def mg_get_newton_field(g, level: int, patch: int, out):
    p, dev, _ = _arr(out, writable=True)
    _check(lib().mg_get_newton_field(g, level, patch, p, dev), "mg_get_newton_field")
    return out


def mg_get_total_force(g, level: int, patch: int, out):
    p, dev, _ = _arr(out, writable=True)
    _check(lib().mg_get_total_force(g, level, patch, p, dev), "mg_get_total_force")
    return out


MG_CIC, MG_TSC = 1, 2


def mg_assign_density(g, level: int, pos, mass=None, scheme: int = MG_TSC):
    """pos: (3, count) float64 (numpy or CUDA tensor, C-contiguous, box units)."""
    p, dev, keep = _arr(pos)
    count = (pos.shape[1] if len(pos.shape) == 2 else pos.shape[0] // 3)
    mp, mdev, keep2 = (None, dev, None) if mass is None else _arr(mass)
    if mass is not None and mdev != dev:
        raise ValueError("pos and mass must both be host or both be device arrays")
    _check(lib().mg_assign_density(g, level, scheme, count, p, mp, dev), "mg_assign_density")


def mg_refine_blocks(g, level: int, npc: float, particle_mass: float):
    """Origins (k, 3) int32 of the next level's patches (Sec. III.B criterion)."""
    found = ctypes.c_int()
    _check(lib().mg_refine_blocks(g, level, npc, particle_mass, None, 0, ctypes.byref(found)),
           "mg_refine_blocks")
    out = np.zeros((max(found.value, 1), 3), dtype=np.int32)
    _check(lib().mg_refine_blocks(g, level, npc, particle_mass,
                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  found.value, ctypes.byref(found)), "mg_refine_blocks")
    return out[:found.value]


def mg_get_level_stats(g, level):
    st = mg_solve_stats()
    _check(lib().mg_get_level_stats(g, level, ctypes.byref(st)), "mg_get_level_stats")
    return st.as_dict()


def mg_get_options(g) -> mg_options:
    o = mg_options()
    _check(lib().mg_get_options(g, ctypes.byref(o)), "mg_get_options")
    return o


def mg_set_options(g, opt: mg_options):
    _check(lib().mg_set_options(g, ctypes.byref(opt)), "mg_set_options")


def mg_autotune(g, branch, alpha, kappa, tol, cache_path=None, use_cache=True):
    """Tune sweep counts on the handle's problem; returns (options, seconds)."""
    o = mg_options()
    t = ctypes.c_double()
    path = cache_path.encode() if cache_path else None
    _check(lib().mg_autotune(g, branch, alpha, kappa, tol, path, int(bool(use_cache)),
                             ctypes.byref(o), ctypes.byref(t)), "mg_autotune")
    return o, t.value


def mg_slab_order(n, slab):
    """Launch order of one FP32 sweep in slabs: a list of (colour, z0, nz)."""
    cap = 4 * max(n // max(slab, 1), 1)
    arr = [(ctypes.c_int * cap)() for _ in range(3)]
    count = ctypes.c_int()
    _check(lib().mg_slab_order(n, slab, arr[0], arr[1], arr[2], cap, ctypes.byref(count)),
           "mg_slab_order")
    return [(arr[0][m], arr[1][m], arr[2][m]) for m in range(count.value)]


def options_dict(o: mg_options) -> dict:
    return {name: getattr(o, name) for name, _ in mg_options._fields_}


def mg_destroy_grid(g):
    if g:
        lib().mg_destroy_grid(g)


# ---- single-kernel entry points (device tensors) ----
def mg_op_residual(n, phi, delta, f, branch, alpha, kappa, d=None, stream=None):
    norms = (ctypes.c_double * 5)()
    _check(lib().mg_op_residual(n, _dev(phi), _dev(delta), _dev(f), branch, alpha, kappa, _dev(d),
                                norms, _stream(stream)), "mg_op_residual")
    return {"sum": norms[0], "max": norms[1], "min": norms[2], "guards": int(norms[3]),
            "nonfinite": int(norms[4])}


def mg_op_smooth(n, phi, delta, f, branch, alpha, kappa, lam, sweeps, stream=None):
    _check(lib().mg_op_smooth(n, _dev(phi), _dev(delta), _dev(f), branch, alpha, kappa, lam,
                              sweeps, _stream(stream)), "mg_op_smooth")


def mg_op_restrict(n, fine, coarse, stream=None):
    _check(lib().mg_op_restrict(n, _dev(fine), _dev(coarse), _stream(stream)), "mg_op_restrict")


def mg_op_prolong_correct(n, coarse, coarse_ref, fine, stream=None):
    _check(lib().mg_op_prolong_correct(n, _dev(coarse), _dev(coarse_ref), _dev(fine),
                                       _stream(stream)), "mg_op_prolong_correct")


def mg_op_residual_noalloc(n, phi, delta, f, branch, alpha, kappa, d=None, stream=None,
                           want_norms=True):
    """mg_op_residual for callers that cannot allocate device memory (n <= 256).
    With want_norms=False the C call gets a NULL norms pointer and None is returned."""
    norms = (ctypes.c_double * 5)() if want_norms else None
    _check(lib().mg_op_residual_noalloc(n, _dev(phi), _dev(delta), _dev(f), branch, alpha, kappa,
                                        _dev(d), norms, _stream(stream)), "mg_op_residual_noalloc")
    if norms is None:
        return None
    return {"sum": norms[0], "max": norms[1], "min": norms[2], "guards": int(norms[3]),
            "nonfinite": int(norms[4])}


def mg_op_force(n, phi, out, stream=None):
    _check(lib().mg_op_force(n, _dev(phi), _dev(out), _stream(stream)), "mg_op_force")
