"""Reconstruction in primitive variables (scheme recon = FV_RECON_PRIMITIVE)
on the GPU against the oracle, with the bars of the conserved path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2306_14011_gb300 import fv  # noqa: E402
from paper_2306_14011_gb300 import inputs as I  # noqa: E402
from test_gpu_parity import CASES, assert_residual_parity, dev, relerr, TOL_RES, TOL_100  # noqa: E402
from test_oracle_recon import _contact_shear  # noqa: E402

pytestmark = pytest.mark.gpu

PRIM = fv.FV_RECON_PRIMITIVE


@pytest.mark.parametrize("lim,kappa", [(fv.FV_LIM_MINMOD, -1.0), (fv.FV_LIM_VANLEER, -1.0), (fv.FV_LIM_NONE, 1.0 / 3.0)])
@pytest.mark.parametrize("case", ["vortex128", "kh256", "ragged70x45_mixed_bc", "sod_rot64_transmissive", "tgv24",
                                  "box3d_36x20x14_mixed"])
def test_residual_and_step_match_oracle(case, lim, kappa):
    if lim == fv.FV_LIM_NONE and case.startswith("sod"):
        pytest.skip("unlimited extrapolation across the Sod jumps gives negative face pressures (NaN in both)")
    g, U = CASES[case]()
    so = O.scheme(limiter=lim, kappa=kappa, recon=O.RECON_PRIMITIVE)
    dto = O.time_step(g, U, so)
    with fv.Solver(g, limiter=lim, kappa=kappa, recon=PRIM) as s:
        R = s.residual(dev(U)).cpu().numpy()
        Ud = dev(U)
        s.rk_step(Ud, dto)
        U1 = Ud.cpu().numpy()
        Rn = torch.empty_like(dev(U))
        fv.fv_residual_noalloc(g, s.scheme, dev(U), Rn)
        torch.cuda.synchronize()
    assert_residual_parity(g, U, R, tag=f"prim-{case}-{lim}", s=so)
    assert relerr(U1, O.rk3_step(g, U, dto, so)[0]) <= TOL_RES
    assert np.array_equal(Rn.cpu().numpy(), R)


def test_hundred_steps_match_oracle():
    g, U = I.isentropic_vortex(64, seed=6)
    so = O.scheme(recon=O.RECON_PRIMITIVE)
    with fv.Solver(g, recon=PRIM) as s:
        Ud = dev(U)
        t = s.run(Ud, 100, return_time=True)
    Uo, to = O.run(g, U, 100, s=so)
    assert relerr(Ud.cpu().numpy(), Uo) <= TOL_100
    assert abs(t - to) <= 1e-12 * to


@pytest.mark.parametrize("dim", [2, 3])
def test_stationary_contact_with_shear_stays_steady(dim):
    g, U = _contact_shear(dim)
    flux_scale = np.prod([g.length[d] / g.n[d] for d in range(1, g.dim)])
    with fv.Solver(g, recon=PRIM) as s:
        R = s.residual(dev(U)).cpu().numpy()
        Ud = dev(U)
        s.run(Ud, 10)
    assert np.abs(R).max() <= 1e-13 * flux_scale
    U10 = Ud.cpu().numpy()
    u_n = U10[1] / U10[0]
    p = 0.4 * (U10[-1] - 0.5 * sum(U10[1 + d] ** 2 for d in range(g.dim)) / U10[0])
    assert np.abs(u_n).max() <= 1e-13 and np.abs(p - 1.0).max() <= 1e-13


def test_launch_invariance():
    g, U = I.kelvin_helmholtz(96, seed=2)
    outs = []
    for tile, thr, loader in [((32, 32, 1), 160, fv.FV_LOADER_TMA), ((16, 8, 1), 64, fv.FV_LOADER_PLAIN),
                              ((64, 4, 1), 192, fv.FV_LOADER_TMA)]:
        d = fv.launch_to_dict(fv.fv_default_launch(g))
        for st in range(3):
            d["stage"][st].update(tile=tile, threads=thr, loader=loader)
        with fv.Solver(g, launch=d, recon=PRIM) as s:
            Ud = dev(U)
            s.run(Ud, 3)
            outs.append(Ud.cpu().numpy())
    assert all(np.array_equal(o, outs[0]) for o in outs[1:])


def test_unsupported_combinations_are_rejected():
    g, U = I.isentropic_vortex(32)
    with pytest.raises(fv.FvError) as e:
        fv.Solver([g, g], recon=PRIM)
    assert e.value.status == fv.FV_EUNSUPPORTED
    with fv.Solver(g, recon=PRIM) as s:
        with pytest.raises(fv.FvError) as e:
            s.residual_vjp(dev(U), dev(U))
        assert e.value.status == fv.FV_EUNSUPPORTED
    g3, U3 = I.taylor_green(24, seed=2)
    d = fv.launch_to_dict(fv.fv_default_launch(g3))
    for st in range(3):
        d["stage"][st].update(tile=(16, 15, 8), threads=256, march=1)
    with pytest.raises(fv.FvError) as e:
        fv.Solver(g3, launch=d, recon=PRIM)
    assert e.value.status == fv.FV_EINVAL
    with pytest.raises(fv.FvError) as e:
        fv.Solver(g, recon=7)
    assert e.value.status == fv.FV_EINVAL
