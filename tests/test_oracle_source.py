"""Oracle pins for the source term of Eq. (5), R = sum_f F.n ds - |Omega| S.

* a uniform state has exactly zero flux differences, so with a constant
  source R = -|Omega| S bit for bit, and one SSP-RK3 step integrates the
  constant derivative S exactly: U + dt S;
* a manufactured steady solution U_m with S = div F(U_m) (derived
  symbolically) makes R(U_m)/|Omega| the scheme's truncation error, which
  must fall as h^2 for the unlimited second-order reconstruction, in 2D and
  3D -- a check of the source term and of the flux's consistency together.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2306_14011_gb300 import inputs as I

sp = pytest.importorskip("sympy")

GAMMA = 1.4


@pytest.mark.parametrize("dim", [2, 3])
def test_constant_source_on_uniform_state(dim):
    g = I.grid2d(12, 10, 1.0, 0.8) if dim == 2 else I.grid3d(8, 7, 6, 1.0, 0.9, 0.7)
    U = I.uniform_state(g)
    rng = np.random.default_rng(1)
    s_val = rng.normal(size=g.nvar)
    S = np.broadcast_to(s_val.reshape((g.nvar,) + (1,) * g.dim), U.shape).copy()
    vol = np.prod([g.length[d] / g.n[d] for d in range(g.dim)])
    R = O.residual(g, U, S=S)
    assert np.array_equal(R, -vol * S)
    assert np.array_equal(O.residual(g, U), np.zeros_like(U))
    dt = 1e-3
    U1, used = O.rk3_step(g, U, dt, S=0.01 * S)
    assert used == dt
    assert np.allclose(U1, U + dt * 0.01 * S, rtol=1e-14, atol=1e-16)


def _manufactured(dim):
    """Symbols, conserved state and source S = div F of a smooth periodic state."""
    X = sp.symbols("x y z")[:dim]
    tp = 2 * sp.pi
    x, y = X[0], X[1]
    z = X[2] if dim == 3 else 0
    rho = 1 + sp.Rational(1, 5) * sp.sin(tp * x) * sp.cos(tp * y) + sp.Rational(1, 10) * sp.sin(tp * z)
    vel = [sp.Rational(3, 10) + sp.Rational(1, 10) * sp.cos(tp * x) * sp.sin(tp * y),
           -sp.Rational(1, 5) + sp.Rational(1, 10) * sp.sin(tp * (x + y + z)),
           sp.Rational(1, 10) + sp.Rational(1, 20) * sp.cos(tp * (x - z))][:dim]
    p = 1 + sp.Rational(1, 10) * sp.sin(tp * (x + y)) * sp.cos(tp * z)
    E = p / (GAMMA - 1) + rho * sum(u * u for u in vel) / 2
    Ucons = [rho] + [rho * u for u in vel] + [E]
    S = [0] * (dim + 2)
    for d in range(dim):
        un = vel[d]
        flux = [rho * un] + [rho * u * un + (p if a == d else 0) for a, u in enumerate(vel)] + [un * (E + p)]
        for v in range(dim + 2):
            S[v] = S[v] + sp.diff(flux[v], X[d])
    return X, Ucons, S


def _truncation_error(dim, n, X, Ucons, S, s):
    g = I.grid2d(n, n, 1.0, 1.0) if dim == 2 else I.grid3d(n, n, n, 1.0, 1.0, 1.0)
    c = (np.arange(n) + 0.5) / n
    grids = np.meshgrid(*([c] * dim), indexing="ij")[::-1]  # arrays indexed [(z,) y, x]
    args = grids if dim == 3 else grids[:2]
    U = np.stack([np.broadcast_to(sp.lambdify(X, e, "numpy")(*args), grids[0].shape) for e in Ucons])
    Sv = np.stack([np.broadcast_to(sp.lambdify(X, e, "numpy")(*args), grids[0].shape) for e in S])
    vol = (1.0 / n) ** dim
    R = O.residual(g, np.ascontiguousarray(U), s, S=np.ascontiguousarray(Sv))
    return np.abs(R / vol).reshape(g.nvar, -1).mean(axis=1)


@pytest.mark.parametrize("dim,ns", [(2, (32, 64, 128)), (3, (12, 24, 48))])
def test_manufactured_solution_truncation_error_is_second_order(dim, ns):
    X, Ucons, S = _manufactured(dim)
    s = O.scheme(limiter=O.LIM_NONE, kappa=-1.0)
    errs = [_truncation_error(dim, n, X, Ucons, S, s) for n in ns]
    for coarse, fine in zip(errs[:-1], errs[1:]):
        order = np.log2(coarse / fine)
        assert np.all(order > 1.85), order
    # without the source the residual is O(1): the source is what cancels it
    assert errs[-1].max() < 0.05 * _truncation_error(dim, ns[-1], X, Ucons, [0] * (dim + 2), s).max()
