"""Python binding of libfv (include/fv.h): argument marshalling only.

Every numerical step runs in the library's CUDA kernels; this module converts
torch tensors / numpy arrays to pointers and status codes to exceptions.  It
never computes anything itself and has no CPU fallback: if libfv cannot be
built or loaded, or there is no CUDA device, calls raise.

Functions mirror the C ABI one to one (fv_init, fv_residual, fv_time_step,
fv_rk_step, fv_run, fv_sync, fv_destroy, ...); `Solver` wraps a context.
State arrays: torch.float64 CUDA tensors (device pointers, stream-ordered) or
numpy float64 arrays (host pointers: the library stages them and waits).
Shapes follow the inputs module: (nvar, ny, nx) in 2D, (nvar, nz, ny, nx) in 3D.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import build as _build

FV_OK, FV_EINVAL, FV_ENOMEM, FV_ECUDA, FV_ENONPHYSICAL, FV_ETIMEOUT, FV_EUNSUPPORTED = range(7)
FV_BC_PERIODIC, FV_BC_TRANSMISSIVE = 0, 1
FV_LOADER_TMA, FV_LOADER_PLAIN = 0, 1


class FvError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} (status {status})")


class fv_grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("len", C.c_double * 3), ("bc", (C.c_int * 2) * 3)]


FV_LIM_MINMOD, FV_LIM_VANLEER, FV_LIM_NONE = 0, 1, 2
FV_RECON_CONSERVED, FV_RECON_PRIMITIVE = 0, 1


class fv_scheme(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("eps", C.c_double), ("kappa", C.c_double),
                ("efix", C.c_double), ("limiter", C.c_int), ("recon", C.c_int)]


class fv_kernel_cfg(C.Structure):
    _fields_ = [("tile", C.c_int * 3), ("threads", C.c_int), ("grid", C.c_int), ("loader", C.c_int),
                ("march", C.c_int)]


FV_FUSED, FV_SPLIT = 0, 1
FV_SK_LIMITER, FV_SK_FLUX, FV_SK_SOURCE, FV_SK_RHS, FV_SK_UPDATE, FV_SK_COUNT = 0, 3, 6, 7, 8, 9


class fv_launch(C.Structure):
    _fields_ = [("stage", fv_kernel_cfg * 3), ("dt", fv_kernel_cfg), ("mode", C.c_int),
                ("split", fv_kernel_cfg * FV_SK_COUNT)]


class fv_mlp_hyper(C.Structure):
    _fields_ = [("alpha", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("lr", C.c_double),
                ("eps", C.c_double), ("tol", C.c_double), ("batch", C.c_int), ("max_epochs", C.c_int),
                ("n_iter_no_change", C.c_int)]


class fv_tune_opts(C.Structure):
    _fields_ = [("samples", C.c_int), ("steps", C.c_int), ("repeats", C.c_int), ("candidates", C.c_int),
                ("top", C.c_int), ("exhaustive", C.c_int), ("final_repeats", C.c_int), ("rounds", C.c_int),
                ("refine", C.c_int), ("seed", C.c_ulonglong),
                ("hidden", C.c_int * 4), ("mlp", fv_mlp_hyper)]


class fv_tune_report(C.Structure):
    _fields_ = [("t_default", C.c_double), ("t_tuned", C.c_double), ("t_search", C.c_double),
                ("t_best_sampled", C.c_double), ("t_exhaustive", C.c_double), ("r2_train", C.c_double),
                ("r2_test", C.c_double), ("space_size", C.c_double), ("n_params", C.c_int), ("n_train", C.c_int),
                ("n_test", C.c_int), ("epochs", C.c_int), ("n_measured", C.c_int), ("n_exhaustive", C.c_int),
                ("rounds", C.c_int), ("n_refined", C.c_int), ("chosen", C.c_int), ("exhaustive_best", fv_launch),
                ("search_best", fv_launch)]


_lib = None
_VP = C.c_void_p


def load() -> C.CDLL:
    """Build (if stale) and load libfv.so from the package's _build folder."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.POINTER
        L.fv_strerror.argtypes = [C.c_int]
        L.fv_strerror.restype = C.c_char_p
        L.fv_default_launch.argtypes = [P(fv_grid), P(fv_launch)]
        L.fv_init.argtypes = [P(_VP), P(fv_grid), C.c_int, P(fv_scheme), P(fv_launch), _VP]
        L.fv_set_launch.argtypes = [_VP, P(fv_launch)]
        L.fv_get_launch.argtypes = [_VP, P(fv_launch)]
        L.fv_residual.argtypes = [_VP, _VP, _VP, _VP]
        L.fv_time_step.argtypes = [_VP, _VP, _VP]
        L.fv_rk_step.argtypes = [_VP, _VP, C.c_double, _VP]
        L.fv_run.argtypes = [_VP, _VP, C.c_int, C.c_double, _VP]
        L.fv_sync.argtypes = [_VP]
        L.fv_destroy.argtypes = [_VP]
        L.fv_destroy.restype = None
        L.fv_debug_math.argtypes = [_VP, _VP, _VP, C.c_long, _VP]
        L.fv_residual_noalloc.argtypes = [P(fv_grid), P(fv_scheme), _VP, _VP, _VP, _VP]
        L.fv_residual_noalloc.restype = C.c_int
        L.fv_mlp_train.argtypes = [C.c_int, P(C.c_int), _VP, _VP, _VP, C.c_long, _VP, C.c_int, P(fv_mlp_hyper),
                                   P(C.c_double), P(C.c_int), _VP]
        L.fv_mlp_train.restype = C.c_int
        L.fv_mlp_predict.argtypes = [C.c_int, P(C.c_int), _VP, _VP, C.c_long, _VP, _VP]
        L.fv_mlp_predict.restype = C.c_int
        L.fv_tune.argtypes = [_VP, _VP, P(fv_tune_opts), P(fv_launch), P(fv_tune_report)]
        L.fv_tune.restype = C.c_int
        L.fv_tune_space.argtypes = [C.c_int, C.c_int, P(C.c_int), P(C.c_double)]
        L.fv_tune_space.restype = C.c_int
        L.fv_set_source.argtypes = [_VP, _VP]
        L.fv_set_source.restype = C.c_int
        L.fv_debug_wait.argtypes = [C.c_int, C.c_double, _VP]
        L.fv_debug_wait.restype = C.c_int
        L.fv_debug_bits.argtypes = [C.c_int, _VP, _VP, _VP, C.c_long, _VP]
        L.fv_debug_fp64_rate.argtypes = [C.c_int, P(C.c_double), _VP]
        L.fv_debug_fp64_rate.restype = C.c_int
        L.fv_debug_bits.restype = C.c_int
        L.fv_layout.argtypes = [_VP, P(C.c_longlong), C.c_int]
        L.fv_layout.restype = C.c_int
        L.fv_adjoint_vjp.argtypes = [_VP, C.c_int, _VP, _VP, C.c_double, _VP]
        L.fv_adjoint_vjp.restype = C.c_int
        L.fv_rk_step_stages.argtypes = [_VP, _VP, C.c_double, _VP, _VP]
        L.fv_rk_step_stages.restype = C.c_int
        L.fv_adjoint_vjp_stages.argtypes = [_VP, _VP, _VP, _VP, _VP, C.c_double, _VP]
        L.fv_adjoint_vjp_stages.restype = C.c_int
        for name in ("fv_default_launch", "fv_init", "fv_set_launch", "fv_get_launch", "fv_residual",
                     "fv_time_step", "fv_rk_step", "fv_run", "fv_sync", "fv_debug_math"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def library_path() -> str:
    return _build.LIB


def strerror(status: int) -> str:
    return load().fv_strerror(status).decode()


def _check(status: int, where: str):
    if status != FV_OK:
        raise FvError(status, where)


# ----------------------------------------------------------------------------- marshalling

def make_grid(g) -> fv_grid:
    G = fv_grid()
    G.dim = g.dim
    for a in range(3):
        G.n[a] = g.n[a] if a < g.dim else 1
        G.len[a] = g.length[a]
        G.bc[a][0], G.bc[a][1] = g.bc[a]
    return G


def make_scheme(gamma=1.4, cfl=0.5, eps=1.0, kappa=-1.0, efix=0.1, limiter=FV_LIM_MINMOD,
                recon=FV_RECON_CONSERVED) -> fv_scheme:
    return fv_scheme(gamma, cfl, eps, kappa, efix, limiter, recon)


def launch_to_dict(l: fv_launch) -> dict:
    st = [dict(tile=tuple(l.stage[s].tile), threads=l.stage[s].threads, loader=l.stage[s].loader,
               march=l.stage[s].march) for s in range(3)]
    sp = [dict(grid=l.split[k].grid, threads=l.split[k].threads) for k in range(FV_SK_COUNT)]
    return dict(stage=st, dt=dict(threads=l.dt.threads, grid=l.dt.grid), mode=l.mode, split=sp)


def launch_from_dict(d: dict) -> fv_launch:
    """The inverse of launch_to_dict; "mode" defaults to FV_FUSED and "split"
    (a list of FV_SK_COUNT dicts with grid and threads) may be omitted in
    FV_FUSED mode."""
    l = fv_launch()
    l.mode = d.get("mode", FV_FUSED)
    for k, e in enumerate(d.get("split", [])):
        l.split[k].grid = e.get("grid", 0)
        l.split[k].threads = e["threads"]
    for s in range(3):
        e = d["stage"][s]
        for a in range(3):
            l.stage[s].tile[a] = e["tile"][a]
        l.stage[s].threads = e["threads"]
        l.stage[s].grid = 0
        l.stage[s].loader = e.get("loader", FV_LOADER_TMA)
        l.stage[s].march = e.get("march", 0)
    l.dt.threads = d["dt"]["threads"]
    l.dt.grid = d["dt"].get("grid", 0)
    return l


def _ptr(x) -> int:
    """Device pointer of a CUDA float64 tensor or host pointer of a numpy array."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags.c_contiguous:
            raise TypeError("numpy arrays must be C-contiguous float64")
        return x.ctypes.data
    import torch
    if isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        if not x.is_cuda:
            return _ptr(x.numpy())
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ----------------------------------------------------------------------------- C ABI mirror

def fv_default_launch(g) -> fv_launch:
    l = fv_launch()
    _check(load().fv_default_launch(C.byref(make_grid(g)), C.byref(l)), "fv_default_launch")
    return l


def fv_init(g, scheme: fv_scheme, launch: Optional[fv_launch] = None, stream=None) -> int:
    """g: a GridSpec, or a list of 2D GridSpecs for a batched context."""
    ctx = _VP()
    grids = list(g) if isinstance(g, (list, tuple)) else [g]
    G = (fv_grid * len(grids))(*[make_grid(x) for x in grids])
    _check(load().fv_init(C.byref(ctx), G, len(grids), C.byref(scheme), C.byref(launch) if launch else None,
                          _stream_handle(stream)), "fv_init")
    return ctx.value


def fv_layout(ctx: int, ngrids: int):
    """Offsets (in doubles) of each grid's block in the packed state, plus the total."""
    off = (C.c_longlong * (ngrids + 1))()
    _check(load().fv_layout(ctx, off, ngrids), "fv_layout")
    return [off[i] for i in range(ngrids + 1)]


def fv_set_launch(ctx: int, launch: fv_launch):
    _check(load().fv_set_launch(ctx, C.byref(launch)), "fv_set_launch")


def fv_get_launch(ctx: int) -> fv_launch:
    l = fv_launch()
    _check(load().fv_get_launch(ctx, C.byref(l)), "fv_get_launch")
    return l


def fv_residual(ctx: int, U, R, rnorm2=None):
    _check(load().fv_residual(ctx, _ptr(U), _ptr(R), None if rnorm2 is None else _ptr(rnorm2)), "fv_residual")


def fv_time_step(ctx: int, U, dt_out=None) -> Optional[float]:
    if dt_out is None:
        d = C.c_double()
        _check(load().fv_time_step(ctx, _ptr(U), C.addressof(d)), "fv_time_step")
        return d.value
    _check(load().fv_time_step(ctx, _ptr(U), _ptr(dt_out)), "fv_time_step")
    return None


def fv_rk_step(ctx: int, U, dt: float = 0.0, want_dt: bool = False) -> Optional[float]:
    d = C.c_double()
    _check(load().fv_rk_step(ctx, _ptr(U), float(dt), C.addressof(d) if want_dt else None), "fv_rk_step")
    return d.value if want_dt else None


def fv_run(ctx: int, U, nsteps: int, dt_fixed: float = 0.0, want_time: bool = False, ngrids: int = 1):
    """Returns the simulated time (a list of ngrids times for a batch) if want_time."""
    t = (C.c_double * ngrids)()
    _check(load().fv_run(ctx, _ptr(U), int(nsteps), float(dt_fixed), C.addressof(t) if want_time else None),
           "fv_run")
    if not want_time:
        return None
    return t[0] if ngrids == 1 else [t[i] for i in range(ngrids)]


def fv_sync(ctx: int):
    _check(load().fv_sync(ctx), "fv_sync")


def fv_destroy(ctx: int):
    load().fv_destroy(ctx)


def fv_residual_noalloc(g, scheme: fv_scheme, U, R, rnorm2=None, stream=None):
    """Residual (and norms) without a context and without allocating: for
    callers that cannot allocate device memory when they call (a fixed
    device-memory budget, a host application that owns the device's memory).
    Equals fv_residual on a context with the same grid and scheme and no
    source.  Device tensors of the current GPU only; grids above the fixed
    scratch limit raise FvError(FV_EINVAL).  Calls sharing the GPU must not
    overlap (they share one scratch array)."""
    _check(load().fv_residual_noalloc(C.byref(make_grid(g)), C.byref(scheme), _ptr(U), _ptr(R),
                                      None if rnorm2 is None else _ptr(rnorm2), _stream_handle(stream)),
           "fv_residual_noalloc")


def mlp_hyper(**kw) -> fv_mlp_hyper:
    """Table "para-setting" values unless overridden."""
    d = dict(alpha=1e-4, beta1=0.95, beta2=0.90, lr=9e-4, eps=1e-9, tol=1e-6, batch=200, max_epochs=200,
             n_iter_no_change=10)
    d.update(kw)
    return fv_mlp_hyper(**d)


def fv_mlp_train(sizes, params, X, y, order, hyper: fv_mlp_hyper, stream=None):
    """Train on the device in place.  sizes: layer widths; params, X, y, order:
    CUDA tensors (float64 params/X/y, int32 order [epochs][n]).  Returns the
    list of per-epoch mean losses actually run."""
    nl = len(sizes) - 1
    S = (C.c_int * len(sizes))(*sizes)
    epochs = order.shape[0]
    losses = (C.c_double * max(1, epochs))()
    ran = C.c_int()
    _check(load().fv_mlp_train(nl, S, _ptr(params), _ptr(X), _ptr(y), X.shape[0], order.data_ptr(), epochs,
                               C.byref(hyper), losses, C.byref(ran), _stream_handle(stream)), "fv_mlp_train")
    return [losses[i] for i in range(ran.value)]


def fv_mlp_predict(sizes, params, X, out, stream=None):
    nl = len(sizes) - 1
    S = (C.c_int * len(sizes))(*sizes)
    _check(load().fv_mlp_predict(nl, S, _ptr(params), _ptr(X), X.shape[0], _ptr(out), _stream_handle(stream)),
           "fv_mlp_predict")


def fv_tune(ctx: int, U, **opts):
    """Autotune the context's launch configuration for state U (not modified).
    opts: fields of fv_tune_opts (samples, steps, repeats, candidates, top,
    exhaustive, final_repeats, seed, hidden=(...)).  Returns (launch dict,
    report dict); the tuned launch is installed in the context."""
    o = fv_tune_opts()
    for k, v in opts.items():
        if k == "hidden":
            for i, w in enumerate(v):
                o.hidden[i] = w
        elif k == "mlp":
            o.mlp = v
        else:
            setattr(o, k, v)
    best = fv_launch()
    rep = fv_tune_report()
    _check(load().fv_tune(ctx, _ptr(U), C.byref(o), C.byref(best), C.byref(rep)), "fv_tune")
    report = {f[0]: getattr(rep, f[0]) for f in fv_tune_report._fields_
              if f[0] not in ("exhaustive_best", "search_best")}
    report["exhaustive_best"] = launch_to_dict(rep.exhaustive_best) if rep.n_exhaustive else None
    report["search_best"] = launch_to_dict(rep.search_best)
    return launch_to_dict(best), report


def fv_tune_space(dim: int, mode: int = FV_FUSED):
    """(number of tuning parameters, points in the search space) for a dim-D
    grid in kernel structure `mode`."""
    n = C.c_int(0)
    size = C.c_double(0.0)
    _check(load().fv_tune_space(dim, mode, C.byref(n), C.byref(size)), "fv_tune_space")
    return n.value, size.value


def fv_set_source(ctx: int, S):
    """Cell-averaged source of Eq. (5): a device array shaped like the state, or
    None for S = 0 (the caller keeps S alive while the context uses it)."""
    _check(load().fv_set_source(ctx, None if S is None else _ptr(S)), "fv_set_source")


def fv_debug_wait(kind: int, limit_seconds: float, stream=None):
    """Run one of the library's bounded device waits on something that never
    completes (kind 0: the tile-load mbarrier wait, 1: the grid-barrier spin);
    raises FvError(FV_ETIMEOUT) when it gives up as designed."""
    _check(load().fv_debug_wait(int(kind), float(limit_seconds), _stream_handle(stream)), "fv_debug_wait")


FV_VJP_RESIDUAL, FV_VJP_RKSTEP = 0, 1


def fv_adjoint_vjp(ctx: int, what: int, U, lam, dt: float, out):
    """out = (dR/dU)^T lam (what = FV_VJP_RESIDUAL) or (dU_{n+1}/dU_n)^T lam for
    one SSP-RK3 step with fixed dt (FV_VJP_RKSTEP).  Device tensors."""
    _check(load().fv_adjoint_vjp(ctx, what, _ptr(U), _ptr(lam), float(dt), _ptr(out)), "fv_adjoint_vjp")


def fv_rk_step_stages(ctx: int, U, dt: float, U1, U2):
    """One fixed-dt SSP-RK3 step in place on U that also writes its stage
    states U1, U2 (device tensors of U's shape)."""
    _check(load().fv_rk_step_stages(ctx, _ptr(U), float(dt), _ptr(U1), _ptr(U2)), "fv_rk_step_stages")


def fv_adjoint_vjp_stages(ctx: int, U, U1, U2, lam, dt: float, out):
    """out = (dU_{n+1}/dU_n)^T lam for one fixed-dt SSP-RK3 step from its
    stage states U1, U2 (as fv_rk_step_stages wrote them).  Device tensors."""
    _check(load().fv_adjoint_vjp_stages(ctx, _ptr(U), _ptr(U1), _ptr(U2), _ptr(lam), float(dt), _ptr(out)),
           "fv_adjoint_vjp_stages")


def fv_debug_bits(op: int, x, out, y=None, stream=None):
    """out = op(x[, y]) with the kernels' integer-pipe helpers (see fv.h)."""
    _check(load().fv_debug_bits(int(op), _ptr(x), None if y is None else _ptr(y), _ptr(out), x.numel(),
                                _stream_handle(stream)), "fv_debug_bits")


def fv_debug_fp64_rate(kind: int = 0, stream=None) -> float:
    """FP64 lane-operations per second of a DFMA (kind 0) or DADD (kind 1)
    stream kernel filling the device: the reference issue rate."""
    r = C.c_double(0.0)
    _check(load().fv_debug_fp64_rate(int(kind), C.byref(r), _stream_handle(stream)), "fv_debug_fp64_rate")
    return r.value


def fv_debug_math(x, out_rsqrt, out_rcp, stream=None):
    _check(load().fv_debug_math(_ptr(x), _ptr(out_rsqrt), _ptr(out_rcp), x.numel(), _stream_handle(stream)),
           "fv_debug_math")


def torch_empty_like(U):
    return U.new_empty(U.shape)


# ----------------------------------------------------------------------------- convenience wrapper

class Solver:
    """A libfv context for one grid.

    Solver(grid, gamma=1.4, cfl=0.5, eps=1.0, kappa=-1.0, efix=0.1,
           launch=None (dict or fv_launch), stream=None (torch's current stream),
           limiter=FV_LIM_MINMOD | FV_LIM_VANLEER | FV_LIM_NONE,
           recon=FV_RECON_CONSERVED | FV_RECON_PRIMITIVE,
           mode=None | FV_FUSED | FV_SPLIT)
    mode, when given, selects the kernel structure: with launch=None it starts
    from the library's default launch; it overrides the mode of a given launch.
    """

    def __init__(self, grid, gamma=1.4, cfl=0.5, eps=1.0, kappa=-1.0, efix=0.1, launch=None, stream=None,
                 limiter=FV_LIM_MINMOD, recon=FV_RECON_CONSERVED, mode=None):
        self.batched = isinstance(grid, (list, tuple))
        self.grids = list(grid) if self.batched else [grid]
        self.grid = self.grids[0]
        self.ngrids = len(self.grids)
        self.scheme = make_scheme(gamma, cfl, eps, kappa, efix, limiter, recon)
        if isinstance(launch, dict):
            launch = launch_from_dict(launch)
        if mode is not None:
            if launch is None:
                launch = fv_default_launch(self.grid)
            launch.mode = mode
        self.ctx = fv_init(grid, self.scheme, launch, stream)
        self.offsets = fv_layout(self.ctx, self.ngrids)

    # shapes
    def _chk(self, U):
        shape = (self.offsets[-1],) if self.batched else tuple(self.grid.shape)
        if tuple(U.shape) != shape:
            raise ValueError(f"state shape {tuple(U.shape)} != expected {shape}")

    def pack(self, states, out=None):
        """Packed state of a batch from one array per grid (numpy or torch)."""
        import torch
        first = states[0]
        if out is None:
            out = (np.zeros(self.offsets[-1]) if isinstance(first, np.ndarray)
                   else torch.zeros(self.offsets[-1], dtype=torch.float64, device=first.device))
        for g, (S, gs) in enumerate(zip(states, self.grids)):
            out[self.offsets[g]:self.offsets[g] + S.numel() if not isinstance(S, np.ndarray) else
                self.offsets[g] + S.size] = S.reshape(-1)
        return out

    def unpack(self, U):
        """Views of each grid's state in a packed batch."""
        return [U[self.offsets[g]:self.offsets[g] + int(np.prod(gs.shape))].reshape(gs.shape)
                for g, gs in enumerate(self.grids)]

    @property
    def launch(self) -> dict:
        return launch_to_dict(fv_get_launch(self.ctx))

    @launch.setter
    def launch(self, d):
        fv_set_launch(self.ctx, launch_from_dict(d) if isinstance(d, dict) else d)

    def residual(self, U, R=None, norms: bool = False):
        """R_h of Eq. (5); with norms=True also returns sum_cells R_v^2 per variable."""
        self._chk(U)
        if R is None:
            R = U.new_empty(U.shape) if not isinstance(U, np.ndarray) else np.empty_like(U)
        nrm = None
        if norms:
            nrm = np.zeros(self.grid.nvar) if isinstance(U, np.ndarray) else U.new_zeros(self.grid.nvar)
        fv_residual(self.ctx, U, R, nrm)
        return (R, nrm) if norms else R

    def time_step(self, U) -> float:
        self._chk(U)
        return fv_time_step(self.ctx, U)

    def rk_step(self, U, dt: float = 0.0, return_dt: bool = False):
        self._chk(U)
        return fv_rk_step(self.ctx, U, dt, want_dt=return_dt)

    def run(self, U, nsteps: int, dt_fixed: float = 0.0, return_time: bool = False):
        self._chk(U)
        return fv_run(self.ctx, U, nsteps, dt_fixed, want_time=return_time, ngrids=self.ngrids)

    def residual_vjp(self, U, lam, out=None):
        """(dR/dU)^T lam."""
        out = torch_empty_like(U) if out is None else out
        fv_adjoint_vjp(self.ctx, FV_VJP_RESIDUAL, U, lam, 0.0, out)
        return out

    def rk_step_vjp(self, U, lam, dt: float, out=None):
        """(dU_{n+1}/dU_n)^T lam for one fixed-dt SSP-RK3 step taken from U."""
        out = torch_empty_like(U) if out is None else out
        fv_adjoint_vjp(self.ctx, FV_VJP_RKSTEP, U, lam, dt, out)
        return out

    def rk_step_stages(self, U, dt: float, U1, U2):
        """One fixed-dt SSP-RK3 step in place on U, also writing its stage
        states into U1 and U2."""
        self._chk(U)
        fv_rk_step_stages(self.ctx, U, dt, U1, U2)

    def rk_step_vjp_stages(self, U, U1, U2, lam, dt: float, out=None):
        """rk_step_vjp from the step's stage states (as rk_step_stages wrote
        them): the same values without recomputing the stages."""
        out = torch_empty_like(U) if out is None else out
        fv_adjoint_vjp_stages(self.ctx, U, U1, U2, lam, dt, out)
        return out

    def set_source(self, S):
        """Cell-averaged source S_h of Eq. (5) (a device tensor shaped like the
        state, kept referenced here), or None for S = 0."""
        if S is not None:
            self._chk(S)
            if not S.is_contiguous() or not S.is_cuda:
                raise ValueError("the source must be a contiguous CUDA tensor")
        fv_set_source(self.ctx, S)
        self._source = S

    def tune(self, U, **opts):
        """Run the autotuner on state U; installs and returns the tuned launch."""
        self._chk(U)
        return fv_tune(self.ctx, U, **opts)

    def sync(self):
        fv_sync(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            fv_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
