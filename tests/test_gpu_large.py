"""GPU parity on a grid whose state has more than 2^31 elements.

A 24576 x 24576 periodic grid holds 6.0e8 cells and 2.4e9 doubles per state,
so offsets into the last variables exceed 2^31 and any 32-bit index on the
path would wrap.  The state is built on the device (a smooth analytic field);
the residual and one fixed-dt SSP-RK3 step are checked on sampled cells --
the last cells of the array among them -- against the oracle evaluated on
small windows around each cell (the stencil reaches 2 cells per stage along
each axis, so a window of half-width 2 for the residual, 8 for three stages,
reproduces the full-grid values at its centre).  About 100 GB of device
memory.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2306_14011_gb300 import fv  # noqa: E402
from paper_2306_14011_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu

N = 24576
GAMMA = 1.4


def _state(n):
    """rho, m_x, m_y, E of a smooth periodic field, float64 on the device."""
    U = torch.empty((4, n, n), dtype=torch.float64, device="cuda")
    x = (torch.arange(n, dtype=torch.float64, device="cuda") + 0.5) / n
    sx, cx = torch.sin(2 * np.pi * x), torch.cos(2 * np.pi * x)
    X, Y = sx.view(1, n), cx.view(n, 1)
    U[0] = 1.0 + 0.2 * X * Y                                   # rho
    U[1] = U[0] * (0.3 + 0.1 * cx.view(1, n) * sx.view(n, 1))  # rho u
    U[2] = U[0] * (-0.2 + 0.1 * X * sx.view(n, 1))             # rho v
    p = 1.0 + 0.1 * cx.view(1, n) * Y
    U[3] = p / (GAMMA - 1.0) + 0.5 * (U[1] ** 2 + U[2] ** 2) / U[0]
    return U


def _windows(U, ys, xs, w):
    """(S, 4, 2w+1, 2w+1) periodic windows of the device state around (y, x)."""
    n = U.shape[-1]
    off = torch.arange(-w, w + 1, device="cuda")
    iy = (torch.as_tensor(ys, device="cuda").view(-1, 1) + off) % n
    ix = (torch.as_tensor(xs, device="cuda").view(-1, 1) + off) % n
    return U[:, iy[:, :, None], ix[:, None, :]].permute(1, 0, 2, 3).cpu().numpy()


def test_grid_beyond_int32_element_offsets():
    g = I.grid2d(N, N, 1.0, 1.0)
    assert g.nvar * g.ncells > 2 ** 31
    rng = np.random.default_rng(5)
    cells = np.concatenate([rng.integers(0, g.ncells, 1500), np.arange(g.ncells - 64, g.ncells),
                            np.arange(0, 32), [N * 31 + 31, N * 32 + 32, N * 4095 + 4096]])
    ys, xs = np.divmod(cells, N)
    U = _state(N)
    h = 1.0 / N
    with fv.Solver(g) as s:
        R = s.residual(U)
        Rs = R[:, torch.as_tensor(ys, device="cuda"), torch.as_tensor(xs, device="cuda")].cpu().numpy()
        del R
        torch.cuda.empty_cache()
        # residual: 5 x 5 windows
        Uw = _windows(U, ys, xs, 2)
        gw = I.grid2d(5, 5, 5 * h, 5 * h)
        Ro = np.stack([O.residual(gw, np.ascontiguousarray(u))[:, 2, 2] for u in Uw], axis=1)
        Rx = np.stack([O.residual_ext(gw, np.ascontiguousarray(u))[:, 2, 2] for u in Uw], axis=1)
        for v in range(g.nvar):
            scale = np.abs(Rx[v]).max()
            e_orc = np.abs(Ro[v] - Rx[v]).max()
            tol = max(1e-12 * scale, 4.0 * e_orc)
            assert np.abs(Rs[v] - Ro[v]).max() <= tol, (v, np.abs(Rs[v] - Ro[v]).max() / scale)
            assert np.abs(Rs[v] - Rx[v]).max() <= tol
        # one fixed-dt SSP-RK3 step: 17 x 17 windows
        dt = 0.1 * h
        pick = np.concatenate([rng.choice(len(cells) - 100, 200, replace=False), np.arange(len(cells) - 100,
                                                                                          len(cells))])
        Uw = _windows(U, ys[pick], xs[pick], 8)
        s.rk_step(U, dt)
        got = U[:, torch.as_tensor(ys[pick], device="cuda"), torch.as_tensor(xs[pick], device="cuda")].cpu().numpy()
    W = 8
    gw = I.grid2d(2 * W + 1, 2 * W + 1, (2 * W + 1) * h, (2 * W + 1) * h)
    exp = np.stack([O.rk3_step(gw, np.ascontiguousarray(u), dt)[0][:, W, W] for u in Uw], axis=1)
    scale = np.abs(exp).max(axis=1, keepdims=True)
    assert np.all(np.abs(got - exp) <= 1e-12 * scale)
