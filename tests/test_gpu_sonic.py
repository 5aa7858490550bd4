"""Sonic points: the entropy fix of the Roe flux on the GPU against the
oracle.  A smooth periodic flow whose normal velocities sweep through -c..+c
puts many faces inside the fix's band |lambda| < efix c~ on both acoustic
waves, for both signs of u~_n (the kernels evaluate the flux from the upwind
side, where one acoustic wave remains).  Same bars as the parity tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2306_14011_gb300 import fv  # noqa: E402
from paper_2306_14011_gb300 import inputs as I  # noqa: E402
from test_gpu_parity import assert_residual_parity, dev, relerr, TOL_RES  # noqa: E402

pytestmark = pytest.mark.gpu


def _transonic(dim):
    g = I.grid2d(96, 80, 1.0, 0.8) if dim == 2 else I.grid3d(40, 36, 32, 1.0, 0.9, 0.8)
    X = np.meshgrid(*I.cell_centres(g)[::-1], indexing="ij")[::-1]  # X[0] = x, ...
    tp = 2 * np.pi
    rho = 1.0 + 0.2 * np.sin(tp * X[0]) * np.cos(tp * X[1] / g.length[1])
    p = 1.0 + 0.1 * np.cos(tp * X[1] / g.length[1])
    c = np.sqrt(1.4 * p / rho)
    vel = [1.3 * c * np.sin(tp * X[0] + 0.3), 1.2 * c * np.cos(tp * X[1] / g.length[1] + 0.7)]
    if dim == 3:
        vel.append(1.1 * c * np.sin(tp * X[2] / g.length[2] + 1.1))
    return g, I.conserved(rho, vel, p)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("efix", [0.0, 0.1, 0.3, 0.9])
def test_entropy_fix_matches_oracle_at_sonic_points(dim, efix):
    g, U = _transonic(dim)
    so = O.scheme(efix=efix)
    if efix > 0:  # the fix is active on this state
        assert not np.array_equal(O.residual(g, U, so), O.residual(g, U, O.scheme(efix=0.0)))
    dto = O.time_step(g, U, so)
    with fv.Solver(g, efix=efix) as s:
        R = s.residual(dev(U)).cpu().numpy()
        Ud = dev(U)
        s.rk_step(Ud, dto)
        U1 = Ud.cpu().numpy()
    with fv.Solver(g, efix=efix, mode=fv.FV_SPLIT) as s:
        Rs = s.residual(dev(U)).cpu().numpy()
    assert_residual_parity(g, U, R, tag=f"sonic{dim}d-efix{efix}", s=so)
    assert_residual_parity(g, U, Rs, tag=f"sonic{dim}d-efix{efix}-split", s=so)
    assert relerr(U1, O.rk3_step(g, U, dto, so)[0]) <= TOL_RES


def test_entropy_fix_width_of_one_or_more_is_rejected():
    g, U = _transonic(2)
    for efix in (1.0, 2.5, float("nan"), -0.1):
        with pytest.raises(fv.FvError) as e:
            fv.Solver(g, efix=efix)
        assert e.value.status == fv.FV_EINVAL
