"""ctypes front end of the CPU oracle (TEST INFRASTRUCTURE ONLY).

Every function takes numpy float64 arrays in the SoA layout of the inputs
module ((nvar, ny, nx) in 2D, (nvar, nz, ny, nx) in 3D) and a GridSpec-like
object with dim, n, length and bc.  The arithmetic lives in fv_oracle.hpp.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

GAMMA = 1.4


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("len", C.c_double * 3), ("bc", (C.c_int * 2) * 3)]


LIM_MINMOD, LIM_VANLEER, LIM_NONE = 0, 1, 2


RECON_CONSERVED, RECON_PRIMITIVE = 0, 1


class Scheme(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("eps", C.c_double), ("kappa", C.c_double),
                ("efix", C.c_double), ("limiter", C.c_int), ("recon", C.c_int)]


def scheme(gamma=GAMMA, cfl=0.5, eps=1.0, kappa=-1.0, efix=0.1, limiter=LIM_MINMOD,
           recon=RECON_CONSERVED) -> Scheme:
    return Scheme(gamma, cfl, eps, kappa, efix, limiter, recon)


_lib = None
_D = C.POINTER(C.c_double)
_L = C.POINTER(C.c_long)


def lib():
    global _lib
    if _lib is None:
        _lib = load_library(_build.build())
    return _lib


def load_library(path: str):
    """Load an oracle shared library and declare its C signatures."""
    L = C.CDLL(path)
    if True:
        GP, SP = C.POINTER(Grid), C.POINTER(Scheme)
        L.orc_residual.argtypes = [GP, SP, _D, _D, _D]
        L.orc_time_step.argtypes = [GP, SP, _D]
        L.orc_time_step.restype = C.c_double
        L.orc_rk3_step.argtypes = [GP, SP, _D, C.c_double, _D]
        L.orc_rk3_step.restype = C.c_double
        L.orc_run.argtypes = [GP, SP, _D, C.c_int, C.c_double, C.c_double, _D]
        L.orc_run.restype = C.c_double
        L.orc_residual_ext.argtypes = [GP, SP, _D, _D, _D]
        L.orc_residual_terms.argtypes = [GP, SP, _D, _D, _D]
        L.orc_residual_cells.argtypes = [GP, SP, _D, C.c_long, _L, _D, _D]
        L.orc_residual_cells_ext.argtypes = [GP, SP, _D, C.c_long, _L, _D, _D]
        L.orc_roe_flux.argtypes = [SP, C.c_int, C.c_int, _D, _D, _D]
        L.orc_roe_flux.restype = None
        L.orc_physical_flux.argtypes = [SP, C.c_int, C.c_int, _D, _D]
        L.orc_physical_flux.restype = None
        L.orc_muscl.argtypes = [SP, _D, _D, _D]
        L.orc_muscl.restype = None
        L.orc_residual_jvp.argtypes = [GP, SP, _D, _D, _D, _D]
        L.orc_rk3_jvp.argtypes = [GP, SP, _D, _D, C.c_int, C.c_double]
        L.orc_count_ops.argtypes = [GP, SP, _D, C.c_double, _L]
        L.orc_max_threads.argtypes = []
        L.orc_max_threads.restype = C.c_int
    return L


def grid(g) -> Grid:
    G = Grid()
    G.dim = g.dim
    for a in range(3):
        G.n[a] = g.n[a] if a < g.dim else 1
        G.len[a] = g.length[a]
        G.bc[a][0] = g.bc[a][0]
        G.bc[a][1] = g.bc[a][1]
    return G


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _check(g, U):
    U = np.ascontiguousarray(U, dtype=np.float64)
    assert U.shape == tuple(g.shape), (U.shape, g.shape)
    return U


def residual(g, U, s: Scheme | None = None, S=None) -> np.ndarray:
    """R_h of Eq. (5) with face areas; S: cell-averaged source (None: 0)."""
    U = _check(g, U)
    R = np.empty_like(U)
    S = None if S is None else _check(g, S)
    lib().orc_residual(C.byref(grid(g)), C.byref(s or scheme()), _ptr(U), _ptr(R), None if S is None else _ptr(S))
    return R


def residual_ext(g, U, s: Scheme | None = None, S=None) -> np.ndarray:
    """R_h evaluated in extended precision (long double) and rounded to double."""
    U = _check(g, U)
    R = np.empty_like(U)
    S = None if S is None else _check(g, S)
    lib().orc_residual_ext(C.byref(grid(g)), C.byref(s or scheme()), _ptr(U), _ptr(R),
                           None if S is None else _ptr(S))
    return R


def residual_terms(g, U, s: Scheme | None = None, S=None) -> np.ndarray:
    """Per cell and variable, the sum of the magnitudes of the terms R_h adds
    (face fluxes times face areas, and |Omega| |S|): the scale of its rounding."""
    U = _check(g, U)
    R = np.empty_like(U)
    S = None if S is None else _check(g, S)
    lib().orc_residual_terms(C.byref(grid(g)), C.byref(s or scheme()), _ptr(U), _ptr(R),
                             None if S is None else _ptr(S))
    return R


def residual_cells(g, U, cells, s: Scheme | None = None, extended: bool = False, S=None) -> np.ndarray:
    """R_h of Eq. (5) at the listed cells (flat interior indices), the same
    values as residual() there; shape (len(cells), nvar).  S: the source of the
    whole grid (None: 0).  extended=True evaluates in long double and rounds
    the result to double."""
    U = _check(g, U)
    S = None if S is None else _check(g, S)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    out = np.empty((cells.size, g.nvar), dtype=np.float64)
    fn = lib().orc_residual_cells_ext if extended else lib().orc_residual_cells
    rc = fn(C.byref(grid(g)), C.byref(s or scheme()), _ptr(U), cells.size, cells.ctypes.data_as(_L), _ptr(out),
            None if S is None else _ptr(S))
    if rc != 0:
        raise ValueError("residual_cells: a cell index lies outside the grid")
    return out


def time_step(g, U, s: Scheme | None = None) -> float:
    U = _check(g, U)
    return lib().orc_time_step(C.byref(grid(g)), C.byref(s or scheme()), _ptr(U))


def rk3_step(g, U, dt: float = 0.0, s: Scheme | None = None, S=None):
    """One SSP-RK3 step (source S: None for 0); returns (U_new, dt_used)."""
    U = _check(g, U).copy()
    S = None if S is None else _check(g, S)
    dt_used = lib().orc_rk3_step(C.byref(grid(g)), C.byref(s or scheme()), _ptr(U), dt,
                                 None if S is None else _ptr(S))
    return U, dt_used


def run(g, U, nsteps: int, dt_fixed: float = 0.0, t_end: float = 0.0, s: Scheme | None = None, S=None):
    """nsteps SSP-RK3 steps (CFL dt unless dt_fixed > 0; source S: None for 0);
    returns (U_new, t)."""
    U = _check(g, U).copy()
    S = None if S is None else _check(g, S)
    t = lib().orc_run(C.byref(grid(g)), C.byref(s or scheme()), _ptr(U), nsteps, dt_fixed, t_end,
                      None if S is None else _ptr(S))
    return U, t


def roe_flux(QL, QR, d: int, dim: int | None = None, s: Scheme | None = None) -> np.ndarray:
    QL = np.ascontiguousarray(QL, dtype=np.float64)
    QR = np.ascontiguousarray(QR, dtype=np.float64)
    dim = dim or QL.size - 2
    F = np.empty(dim + 2)
    lib().orc_roe_flux(C.byref(s or scheme()), dim, d, _ptr(QL), _ptr(QR), _ptr(F))
    return F


def physical_flux(Q, d: int, s: Scheme | None = None) -> np.ndarray:
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    F = np.empty(Q.size)
    lib().orc_physical_flux(C.byref(s or scheme()), Q.size - 2, d, _ptr(Q), _ptr(F))
    return F


def muscl(q4, s: Scheme | None = None):
    q4 = np.ascontiguousarray(q4, dtype=np.float64)
    QL, QR = C.c_double(), C.c_double()
    lib().orc_muscl(C.byref(s or scheme()), _ptr(q4), C.byref(QL), C.byref(QR))
    return QL.value, QR.value


def residual_jvp(g, U, dU, s: Scheme | None = None):
    """(R, dR) with dR = (dR/dU) dU, by forward-mode dual numbers."""
    U = _check(g, U)
    dU = _check(g, dU)
    R = np.empty_like(U)
    dR = np.empty_like(U)
    lib().orc_residual_jvp(C.byref(grid(g)), C.byref(s or scheme()), _ptr(U), _ptr(dU), _ptr(R), _ptr(dR))
    return R, dR


def rk3_jvp(g, U, dU, nsteps: int, dt: float, s: Scheme | None = None):
    """State after nsteps fixed-dt SSP-RK3 steps and its directional derivative."""
    U = _check(g, U).copy()
    dU = _check(g, dU).copy()
    lib().orc_rk3_jvp(C.byref(grid(g)), C.byref(s or scheme()), _ptr(U), _ptr(dU), nsteps, dt)
    return U, dU


def max_threads() -> int:
    """Threads the oracle's OpenMP loops use on this host."""
    return lib().orc_max_threads()


def count_ops(g, U, dt: float, s: Scheme | None = None) -> dict:
    """Floating-point operation counts of one residual, one time step and one
    SSP-RK3 step on U: {'residual': (add, mul, div, sqrt), ...}."""
    U = _check(g, U)
    c = np.zeros(12, dtype=np.int64)
    lib().orc_count_ops(C.byref(grid(g)), C.byref(s or scheme()), _ptr(U), dt, c.ctypes.data_as(_L))
    return {"residual": tuple(c[0:4]), "time_step": tuple(c[4:8]), "rk3_step": tuple(c[8:12])}
