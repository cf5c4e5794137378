"""ctypes binding of the CPU oracle (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg may
import this module.  It loads ``oracle/liboracle.so`` (built by
``oracle/build_oracle.py`` from ``mg_oracle.c``) and shares nothing with the CUDA
library.  Every array is a C-contiguous float64 numpy array; grids are indexed
``a[k, j, i]`` so that x (i) is the fastest axis.

Conventions (see the header of ``mg_oracle.c`` for the paper passages):
``alpha`` is the coefficient of the nonlinear term in
``lap(phi) + alpha[(lap phi)^2 - (grad grad phi)^2] = kappa * delta``; the
paper's own alpha is ``1/alpha``.  ``branch`` is the sign in front of the square
root of Eq. two_branch, 0 meaning sgn(alpha) (Eq. one_branch).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build_oracle

_LIB = None
_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)

OK, EINVAL, ENOMEM, ENOCONV, ENAN = 0, 1, 2, 4, 5
W_PAPER = 1.0 / 3.0


def lib():
    global _LIB
    if _LIB is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        L.orc_residual.restype = ctypes.c_long
        L.orc_residual.argtypes = [ctypes.c_int, ctypes.c_double, _D, _D, _D, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int, ctypes.c_double, _D]
        L.orc_assign.restype = ctypes.c_int
        L.orc_assign.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_long, _D, _D, _D, _D, _D]
        L.orc_density_floor.restype = ctypes.c_long
        L.orc_density_floor.argtypes = [ctypes.c_long, _D, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, _D]
        L.orc_restrict.restype = None
        L.orc_restrict.argtypes = [ctypes.c_int, _D, _D]
        L.orc_prolong_add.restype = None
        L.orc_prolong_add.argtypes = [ctypes.c_int, _D, _D]
        L.orc_force.restype = None
        L.orc_force.argtypes = [ctypes.c_int, ctypes.c_double, _D, _D]
        L.orc_num_levels.restype = ctypes.c_int
        L.orc_num_levels.argtypes = [ctypes.c_int, ctypes.c_int]
        L.orc_fas_solve.restype = ctypes.c_int
        L.orc_fas_solve.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
        L.orc_gs_sweeps.restype = None
        L.orc_gs_sweeps.argtypes = [ctypes.c_int, _D, _D, _D, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int]
        L.orc_patch_residual.restype = ctypes.c_long
        L.orc_patch_residual.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _I32, _D, _D, _D,
                                         ctypes.c_int, _I32, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_double, _D]
        L.orc_patch_solve.restype = ctypes.c_int
        L.orc_patch_solve.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _I32, _D, _D, _D,
                                      ctypes.c_int, _I32, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                      _D]
        L.orc_patch_ghosts.restype = ctypes.c_int
        L.orc_patch_ghosts.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _I32, _D,
                                       ctypes.c_int, _I32, _D]
        _LIB = L
    return _LIB


_LIBC = None


def lib_colour():
    """The four-colour OpenMP build of the oracle (liboracle_colour.so)."""
    global _LIBC
    if _LIBC is None:
        L = ctypes.CDLL(build_oracle.build_colour())
        L.orc_fas_solve_colour.restype = ctypes.c_int
        L.orc_fas_solve_colour.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
        L.orc_colour_sweeps.restype = ctypes.c_int
        L.orc_colour_sweeps.argtypes = [ctypes.c_int, _D, _D, _D, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_int, ctypes.c_int]
        _LIBC = L
    return _LIBC


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _p(a):
    return None if a is None else a.ctypes.data_as(_D)


def _pi(a):
    return None if a is None else a.ctypes.data_as(_I32)


def residual(phi, delta, alpha, kappa, branch=0, f=None, w=W_PAPER, h=None):
    """d = L^h phi - f on a periodic grid; returns (d, guarded cells).  h defaults
    to 1/n; passing the spacing of a larger grid evaluates a cell of that grid from
    its 3^3 neighbourhood (the centre of a 3^3 array)."""
    phi, delta = _f64(phi), _f64(delta)
    n = phi.shape[0]
    f = None if f is None else _f64(f)
    d = np.empty_like(phi)
    g = lib().orc_residual(n, 1.0 / n if h is None else h, _p(phi), _p(delta), _p(f), alpha,
                           kappa, branch, w, _p(d))
    return d, int(g)


def density_floor(delta, alpha, kappa, w=W_PAPER):
    """delta held at 1 + 4(1-w) alpha kappa delta >= 0; returns (delta', cells changed)."""
    delta = _f64(delta)
    out = np.empty_like(delta)
    hits = lib().orc_density_floor(delta.size, _p(delta), alpha, kappa, w, _p(out))
    return out, int(hits)


def restrict(fine):
    fine = _f64(fine)
    nc = fine.shape[0] // 2
    out = np.empty((nc, nc, nc))
    lib().orc_restrict(nc, _p(fine), _p(out))
    return out


def prolong_add(corr, fine):
    """Return fine + P(corr) (cell-centred trilinear)."""
    corr = _f64(corr)
    out = _f64(fine).copy()
    lib().orc_prolong_add(corr.shape[0], _p(corr), _p(out))
    return out


def force(phi):
    """-(1/2) grad phi by central differences, shape (3, n, n, n) (x, y, z)."""
    phi = _f64(phi)
    n = phi.shape[0]
    out = np.empty((3, n, n, n))
    lib().orc_force(n, 1.0 / n, _p(phi), _p(out))
    return out


def num_levels(n, coarsest=4):
    return lib().orc_num_levels(n, coarsest)


def gs_sweeps(phi, delta, alpha, kappa, branch=0, f=None, lam=0.0, sweeps=1, w=W_PAPER):
    """Plain lexicographic Newton-Gauss-Seidel sweeps of L^h phi = f + lam."""
    phi = _f64(phi).copy()
    delta = _f64(delta)
    f = None if f is None else _f64(f)
    lib().orc_gs_sweeps(phi.shape[0], _p(phi), _p(delta), _p(f), lam, alpha, kappa, branch, w,
                        sweeps)
    return phi


def fas_solve(delta, alpha, kappa, branch=0, tol=1e-10, phi0=None, max_cycles=100, nu_pre=2,
              nu_post=2, coarsest=4, w=W_PAPER):
    """Periodic FAS solve.  Returns (phi (zero mean), stats dict)."""
    delta = _f64(delta)
    n = delta.shape[0]
    phi = np.zeros_like(delta) if phi0 is None else _f64(phi0).copy()
    stats = np.zeros(6 + max(max_cycles, 1))
    st = lib().orc_fas_solve(n, _p(delta), _p(phi), alpha, kappa, branch, w, tol, max_cycles,
                             nu_pre, nu_post, coarsest, _p(stats))
    cyc = int(stats[0])
    return phi, {"status": int(st), "cycles": cyc, "res": float(stats[1]),
                 "lambda": float(stats[2]), "guard_hits": int(stats[3]),
                 "res0": float(stats[5]), "hist": stats[6:6 + cyc].copy()}


def fas_solve_colour(delta, alpha, kappa, branch=0, tol=1e-10, phi0=None, max_cycles=100,
                     nu_pre=2, nu_post=2, coarsest=4, w=W_PAPER, threads=0):
    """fas_solve with four-colour sweeps on `threads` OpenMP threads (0: all cores).
    Returns (phi (zero mean), stats dict with "threads")."""
    delta = _f64(delta)
    phi = np.zeros_like(delta) if phi0 is None else _f64(phi0).copy()
    stats = np.zeros(7 + max(max_cycles, 1))
    st = lib_colour().orc_fas_solve_colour(delta.shape[0], _p(delta), _p(phi), alpha, kappa,
                                           branch, w, tol, max_cycles, nu_pre, nu_post,
                                           coarsest, threads, _p(stats))
    cyc = int(stats[0])
    return phi, {"status": int(st), "cycles": cyc, "res": float(stats[1]),
                 "lambda": float(stats[2]), "guard_hits": int(stats[3]),
                 "res0": float(stats[5]), "hist": stats[6:6 + cyc].copy(),
                 "threads": int(stats[6 + max_cycles])}


def colour_sweeps(phi, delta, alpha, kappa, branch=0, f=None, lam=0.0, sweeps=1, w=W_PAPER,
                  threads=0):
    """Four-colour Newton-Gauss-Seidel sweeps of L^h phi = f + lam in place on a copy;
    returns (phi, threads used)."""
    phi = _f64(phi).copy()
    delta = _f64(delta)
    f = None if f is None else _f64(f)
    t = lib_colour().orc_colour_sweeps(phi.shape[0], _p(phi), _p(delta), _p(f), lam, alpha,
                                       kappa, branch, w, sweeps, threads)
    return phi, int(t)


def _parent_args(level, parent, parent_org):
    if level == 1:
        return _f64(parent), 0, None
    po = np.ascontiguousarray(parent_org, dtype=np.int32)
    return _f64(parent), po.shape[0], po


def patch_residual(n0, level, org, phi, delta, parent, alpha, kappa, branch=0, parent_org=None,
                   w=W_PAPER):
    """Residual on the union of level-`level` 8^3 patches; phi, delta: (count, 8, 8, 8)."""
    org = np.ascontiguousarray(org, dtype=np.int32)
    phi, delta = _f64(phi), _f64(delta)
    par, pc, po = _parent_args(level, parent, parent_org)
    d = np.empty_like(phi)
    g = lib().orc_patch_residual(n0, level, org.shape[0], _pi(org), _p(phi), _p(delta), _p(par),
                                 pc, _pi(po), alpha, kappa, branch, w, _p(d))
    return d, int(g)


def patch_solve(n0, level, org, delta, parent, alpha, kappa, branch=0, parent_org=None,
                tol=1e-10, max_sweeps=100000, phi0=None, w=W_PAPER):
    org = np.ascontiguousarray(org, dtype=np.int32)
    delta = _f64(delta)
    phi = np.zeros_like(delta) if phi0 is None else _f64(phi0).copy()
    par, pc, po = _parent_args(level, parent, parent_org)
    stats = np.zeros(4)
    st = lib().orc_patch_solve(n0, level, org.shape[0], _pi(org), _p(phi), _p(delta), _p(par), pc,
                               _pi(po), alpha, kappa, branch, w, tol, max_sweeps, _p(stats))
    return phi, {"status": int(st), "sweeps": int(stats[0]), "res": float(stats[1]),
                 "guard_hits": int(stats[2])}


def patch_ghosts(n0, level, org, parent, parent_org=None, fill=np.nan):
    """Coarse-to-fine fill values on each patch's 10^3 ghosted block (k, j, i)."""
    org = np.ascontiguousarray(org, dtype=np.int32)
    par, pc, po = _parent_args(level, parent, parent_org)
    out = np.full((org.shape[0], 10, 10, 10), fill)
    st = lib().orc_patch_ghosts(n0, level, org.shape[0], _pi(org), _p(par), pc, _pi(po), _p(out))
    if st != 0:
        raise ValueError("nesting violated: a ghost needs a parent cell outside the parent level")
    return out


def assign_density(nside, pos, mass=None, scheme=2):
    """Mass assignment (Sec. VI): rho on a periodic nside^3 cell-centred grid from
    particles at pos (3, count) in box units; scheme 1 = CIC, 2 = TSC; masses in
    units of the total mass (None: 1/count each).  Returns delta = rho - 1."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    count = pos.shape[1]
    m = None if mass is None else _f64(mass)
    rho = np.zeros((nside,) * 3)
    rc = lib().orc_assign(nside, scheme, count, _p(pos[0]), _p(pos[1]), _p(pos[2]),
                          None if m is None else _p(m), _p(rho))
    if rc:
        raise ValueError("scheme must be 1 (CIC) or 2 (TSC)")
    return rho - 1.0


def refine_blocks(delta, npc, particle_mass, covered=None):
    """Refinement criterion (Sec. III.B: refine where the effective number of
    particles in a cell exceeds N_pc), on 4^3-aligned blocks of a level of side
    n: a block is refined when any of its cells holds more than npc effective
    particles, (1 + delta) h^3 / particle_mass.  `covered` (bool, n^3) limits the
    blocks to cells that exist on this level.  Returns the origins (x, y, z) of
    the next level's 8^3 patches (twice the block origins), sorted by z, y, x."""
    delta = np.asarray(delta, dtype=np.float64)
    n = delta.shape[0]
    count = (1.0 + delta) / float(n) ** 3 / particle_mass
    hot = count > npc
    if covered is not None:
        hot &= covered
    b = n // 4
    blocks = hot.reshape(b, 4, b, 4, b, 4).any(axis=(1, 3, 5))  # [bz, by, bx]
    bz, by, bx = np.nonzero(blocks)
    org = np.stack([bx, by, bz], axis=1).astype(np.int32) * 8
    order = np.lexsort((org[:, 0], org[:, 1], org[:, 2]))
    return org[order]
