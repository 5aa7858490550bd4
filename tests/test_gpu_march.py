"""GPU parity of the z-marching 3D stage kernel (launch field march = 1).

The marching kernel evaluates every face flux from the same stencil values
with the same arithmetic as the box-tiled kernel and accumulates the cell
residual in the same axis order, so its residuals and states must equal the
box-tiled kernel's bit for bit, for any tile, chunk length, thread count and
loader; the box-tiled kernel itself is held to the oracle in
test_gpu_parity.py, and the oracle comparison is repeated here directly.
Residual norms differ from the box kernel's only in summation order.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2306_14011_gb300 import fv  # noqa: E402
from paper_2306_14011_gb300 import inputs as I  # noqa: E402
from test_gpu_parity import assert_residual_parity, dev, relerr, TOL_RES  # noqa: E402

pytestmark = pytest.mark.gpu


def launch(g, tile, threads=256, loader=fv.FV_LOADER_TMA, march=1):
    d = fv.launch_to_dict(fv.fv_default_launch(g))
    for s in range(3):
        d["stage"][s].update(tile=tile, threads=threads, loader=loader, march=march)
    return d


BOX = ((16, 8, 4), 192)


def _grid(n, lens, bc, seed):
    g = I.grid3d(*n, *lens, bc)
    return g, I.random_smooth(g, seed=seed)


CASES = {
    "tgv24": lambda: I.taylor_green(24, seed=2),
    "transmissive_10x7x9": lambda: _grid((10, 7, 9), (1.0, 0.7, 0.9), I.BC_TRANSMISSIVE, 5),
    "mixed_36x20x14": lambda: _grid((36, 20, 14), (1.0, 0.6, 0.5), ((0, 0), (1, 1), (0, 0)), 6),
    "mixed_40x34x11": lambda: _grid((40, 34, 11), (1.0, 0.9, 0.3), ((1, 1), (0, 0), (1, 1)), 7),
    "nz1_periodic": lambda: _grid((18, 12, 1), (1.0, 0.7, 0.1), I.BC_PERIODIC, 8),
    "nz2_transmissive": lambda: _grid((12, 10, 2), (1.0, 0.7, 0.2), I.BC_TRANSMISSIVE, 9),
    "nz3_mixed": lambda: _grid((22, 9, 3), (1.0, 0.4, 0.2), ((0, 0), (0, 0), (1, 1)), 10),
}

# (tile x, tile y, planes per chunk), threads
MARCH_CFGS = [((16, 15, 32), 256), ((16, 15, 1), 256), ((8, 4, 3), 32), ((20, 6, 5), 160), ((16, 16, 7), 128),
              ((2, 2, 2), 64), ((32, 8, 100), 256)]


def _box_reference(g, U):
    with fv.Solver(g, launch=launch(g, BOX[0], BOX[1], march=0)) as s:
        R = s.residual(dev(U)).cpu().numpy()
        Ud = dev(U)
        s.run(Ud, 3)
        return R, Ud.cpu().numpy()


@pytest.mark.parametrize("case", sorted(CASES))
def test_march_equals_box_kernel_bitwise(case):
    g, U = CASES[case]()
    R0, U0 = _box_reference(g, U)
    for tile, thr in MARCH_CFGS:
        for loader in (fv.FV_LOADER_TMA, fv.FV_LOADER_PLAIN):
            with fv.Solver(g, launch=launch(g, tile, thr, loader)) as s:
                R = s.residual(dev(U)).cpu().numpy()
                Ud = dev(U)
                s.run(Ud, 3)
            assert np.array_equal(R, R0), (case, tile, thr, loader)
            assert np.array_equal(Ud.cpu().numpy(), U0), (case, tile, thr, loader)


@pytest.mark.parametrize("case", ["tgv24", "mixed_40x34x11", "nz2_transmissive"])
def test_march_matches_oracle(case):
    g, U = CASES[case]()
    with fv.Solver(g, launch=launch(g, (16, 15, 6))) as s:
        Rd, nrm = s.residual(dev(U), norms=True)
        R = Rd.cpu().numpy()
        dto = O.time_step(g, U, O.scheme())
        Ud = dev(U)
        s.rk_step(Ud, dto)
        U1 = Ud.cpu().numpy()
    assert_residual_parity(g, U, R, tag=f"march-{case}")
    Ro = O.residual(g, U).reshape(g.nvar, -1)
    n_exp = (Ro ** 2).sum(axis=1)
    assert np.allclose(nrm.cpu().numpy(), n_exp, rtol=1e-11, atol=0.0)
    Uo, _ = O.rk3_step(g, U, dto)
    assert relerr(U1, Uo) <= TOL_RES


@pytest.mark.parametrize("lim,kappa", [(fv.FV_LIM_VANLEER, -1.0), (fv.FV_LIM_NONE, 1.0 / 3.0)])
def test_march_limiter_variants_equal_box_kernel(lim, kappa):
    g, U = CASES["mixed_36x20x14"]()
    out = []
    for tile, thr, m in [(BOX[0], BOX[1], 0), ((16, 15, 5), 256, 1), ((8, 6, 2), 96, 1)]:
        with fv.Solver(g, launch=launch(g, tile, thr, march=m), limiter=lim, kappa=kappa) as s:
            R = s.residual(dev(U)).cpu().numpy()
            Ud = dev(U)
            s.run(Ud, 2)
            out.append((R, Ud.cpu().numpy()))
    for R, Un in out[1:]:
        assert np.array_equal(R, out[0][0])
        assert np.array_equal(Un, out[0][1])


def test_march_cfl_run_and_time_equal_box_kernel():
    g, U = I.taylor_green(32, seed=3)
    res = []
    for tile, thr, m in [(BOX[0], BOX[1], 0), ((16, 15, 8), 256, 1)]:
        with fv.Solver(g, launch=launch(g, tile, thr, march=m)) as s:
            Ud = dev(U)
            t = s.run(Ud, 20, return_time=True)
            res.append((Ud.cpu().numpy(), t))
    assert np.array_equal(res[0][0], res[1][0])
    assert res[0][1] == res[1][1]


def test_march_launch_validation():
    g3, _ = CASES["tgv24"]()
    g2, _ = I.isentropic_vortex(32)
    bad = [(g2, dict(tile=(16, 16, 1), march=1)), (g3, dict(tile=(16, 15, 4), march=2)),
           (g3, dict(tile=(16, 15, 0), march=1)), (g3, dict(tile=(15, 16, 4), march=1)),
           (g3, dict(tile=(252, 252, 4), march=1)), (g3, dict(tile=(8, 8, 8), threads=224, march=0))]
    for g, b in bad:
        d = fv.launch_to_dict(fv.fv_default_launch(g))
        for s_ in range(3):
            d["stage"][s_].update(b)
        with pytest.raises(fv.FvError) as e:
            fv.Solver(g, launch=d)
        assert e.value.status == fv.FV_EINVAL, b
