"""Oracle pins for reconstruction in primitive variables (Eq. (6) applied to
rho, u, p; the face states converted back to conserved variables).

* a uniform state has identical face states everywhere: R = 0 exactly;
* a stationary contact with arbitrary shear -- u_n = 0, p uniform, density
  and tangential velocity varying along the normal -- is an exact steady
  state of the primitive scheme (u_n and p reach every face unchanged, the
  Roe flux then carries only p), while the conserved scheme, whose face
  pressure is recomputed from separately limited rho, m and E, produces a
  residual many orders above rounding;
* for smooth manufactured solutions the truncation error still falls as h^2.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2306_14011_gb300 import inputs as I


@pytest.mark.parametrize("dim", [2, 3])
def test_free_stream_is_exact(dim):
    g = I.grid2d(12, 9, 1.0, 0.7) if dim == 2 else I.grid3d(8, 7, 6, 1.0, 0.9, 0.7)
    U = I.uniform_state(g)
    assert np.array_equal(O.residual(g, U, O.scheme(recon=O.RECON_PRIMITIVE)), np.zeros_like(U))


def _contact_shear(dim):
    n = 64
    g = I.grid2d(n, 8, 1.0, 0.125) if dim == 2 else I.grid3d(n, 6, 5, 1.0, 0.1, 0.08)
    x = (np.arange(n) + 0.5) / n
    shape = g.shape[1:]
    rho = np.broadcast_to(1.0 + 0.5 * np.sin(2 * np.pi * x) + 0.3 * (x > 0.5), shape)
    v = np.broadcast_to(0.4 * np.cos(6 * np.pi * x) + 0.2 * (x > 0.3), shape)
    vel = (np.zeros(shape), v) + ((np.broadcast_to(-0.3 * np.sin(4 * np.pi * x), shape),) if dim == 3 else ())
    return g, I.conserved(rho, vel, np.ones(shape))


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("lim", [O.LIM_MINMOD, O.LIM_VANLEER])
def test_stationary_contact_with_shear_is_steady_in_primitive_variables(dim, lim):
    g, U = _contact_shear(dim)
    Rp = O.residual(g, U, O.scheme(limiter=lim, recon=O.RECON_PRIMITIVE))
    Rc = O.residual(g, U, O.scheme(limiter=lim, recon=O.RECON_CONSERVED))
    flux_scale = 1.0 * np.prod([g.length[d] / g.n[d] for d in range(1, g.dim)])  # p * face area
    assert np.abs(Rp).max() <= 1e-13 * flux_scale
    assert np.abs(Rc).max() >= 1e-6 * flux_scale


def test_smooth_solution_truncation_error_is_second_order():
    from test_oracle_source import _manufactured, _truncation_error
    X, Ucons, S = _manufactured(2)
    s = O.scheme(limiter=O.LIM_NONE, kappa=-1.0, recon=O.RECON_PRIMITIVE)
    errs = [_truncation_error(2, n, X, Ucons, S, s) for n in (32, 64, 128)]
    for coarse, fine in zip(errs[:-1], errs[1:]):
        assert np.all(np.log2(coarse / fine) > 1.85)


def test_conserved_reconstruction_is_the_default():
    g, U = I.isentropic_vortex(24, seed=1)
    assert np.array_equal(O.residual(g, U), O.residual(g, U, O.scheme(recon=O.RECON_CONSERVED)))
    assert not np.array_equal(O.residual(g, U), O.residual(g, U, O.scheme(recon=O.RECON_PRIMITIVE)))
