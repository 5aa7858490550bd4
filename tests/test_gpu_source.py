"""The source term of Eq. (5) on the GPU (fv_set_source) against the oracle.

R = sum_f F.n ds - |Omega| S and dU/dt = -R/|Omega| with a cell-averaged
source S in the layout of U.  Same bars as without a source (residual
1e-12 of max|R_v| or 4x the oracle's own rounding error; one RK step 1e-12;
100 steps 1e-9); the box-tiled and z-marching kernels stay bitwise equal.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2306_14011_gb300 import fv  # noqa: E402
from paper_2306_14011_gb300 import inputs as I  # noqa: E402
from test_gpu_parity import CASES, EPS, dev, relerr, TOL_RES, TOL_100  # noqa: E402

pytestmark = pytest.mark.gpu


def _source(g, U, seed):
    """A smooth source of the size of the flux differences, plus noise."""
    rng = np.random.default_rng(seed)
    scale = np.abs(O.residual(g, U)).reshape(g.nvar, -1).max(axis=1)
    vol = np.prod([g.length[d] / g.n[d] for d in range(g.dim)])
    S = I.random_smooth(g, seed=seed + 100) - I.random_smooth(g, seed=seed + 200)
    S = S * (scale / vol / np.maximum(np.abs(S).reshape(g.nvar, -1).max(axis=1), 1e-300)).reshape(
        (g.nvar,) + (1,) * g.dim)
    return np.ascontiguousarray(S + 1e-3 * rng.standard_normal(U.shape) * S.std())


def _residual_parity(g, U, S, R, tag):
    Ro = O.residual(g, U, S=S).reshape(g.nvar, -1)
    Rx = O.residual_ext(g, U, S=S).reshape(g.nvar, -1)
    Rg = np.asarray(R).reshape(g.nvar, -1)
    floor = 8 * EPS * O.residual_terms(g, U, S=S).reshape(g.nvar, -1).max(axis=1)
    for v in range(g.nvar):
        scale = np.abs(Rx[v]).max()
        e_orc = np.abs(Ro[v] - Rx[v]).max()
        tol = max(TOL_RES * scale, 4.0 * e_orc, floor[v])
        assert np.abs(Rg[v] - Ro[v]).max() <= tol, (tag, v, np.abs(Rg[v] - Ro[v]).max() / scale)
        assert np.abs(Rg[v] - Rx[v]).max() <= tol, (tag, v)


@pytest.mark.parametrize("case", ["vortex128", "ragged70x45_mixed_bc", "sod_rot64_transmissive", "tgv24",
                                  "box3d_36x20x14_mixed"])
def test_residual_and_step_with_source_match_oracle(case):
    g, U = CASES[case]()
    S = _source(g, U, 3)
    dto = O.time_step(g, U)
    with fv.Solver(g) as s:
        Sd = dev(S)
        s.set_source(Sd)
        R = s.residual(dev(U)).cpu().numpy()
        Ud = dev(U)
        s.rk_step(Ud, dto)
        U1 = Ud.cpu().numpy()
        Uc = dev(U)
        used = s.rk_step(Uc, 0.0, return_dt=True)
        Uc = Uc.cpu().numpy()
        s.set_source(None)
        R0 = s.residual(dev(U)).cpu().numpy()
    with fv.Solver(g) as s2:
        R_ref = s2.residual(dev(U)).cpu().numpy()
    _residual_parity(g, U, S, R, case)
    assert relerr(U1, O.rk3_step(g, U, dto, S=S)[0]) <= TOL_RES
    assert abs(used - dto) <= 2e-15 * dto  # the CFL step does not see the source
    assert relerr(Uc, O.rk3_step(g, U, used, S=S)[0]) <= TOL_RES
    assert np.array_equal(R0, R_ref)  # cleared: S = 0 again


def test_hundred_steps_with_source_match_oracle():
    g, U = I.isentropic_vortex(64, seed=4)
    S = 0.01 * _source(g, U, 5)
    dto = O.time_step(g, U)
    with fv.Solver(g) as s:
        s.set_source(dev(S))
        Ud = dev(U)
        s.run(Ud, 100, dt_fixed=dto)
        Ug = Ud.cpu().numpy()
        Uh = U.copy()
        s.run(Uh, 100, dt_fixed=dto)  # host path: banded last step
    Uo, _ = O.run(g, U, 100, dt_fixed=dto, S=S)
    assert relerr(Ug, Uo) <= TOL_100
    assert np.array_equal(Ug, Uh)


def test_constant_source_on_free_stream_is_exact():
    g = I.grid3d(20, 18, 12, 1.0, 2.0, 3.0)
    U = I.uniform_state(g)
    s_val = np.array([0.5, -0.25, 0.125, 2.0, -1.0])
    S = np.ascontiguousarray(np.broadcast_to(s_val.reshape(5, 1, 1, 1), U.shape))
    vol = (1.0 / 20) * (2.0 / 18) * (3.0 / 12)
    with fv.Solver(g) as s:
        s.set_source(dev(S))
        R = s.residual(dev(U)).cpu().numpy()
    assert np.array_equal(R, -vol * S)


def test_marching_kernel_with_source_equals_box_kernel():
    g, U = CASES["box3d_36x20x14_mixed"]()
    S = _source(g, U, 7)
    outs = []
    for tile, thr, m in [((8, 8, 8), 192, 0), ((16, 15, 5), 256, 1)]:
        d = fv.launch_to_dict(fv.fv_default_launch(g))
        for st in range(3):
            d["stage"][st].update(tile=tile, threads=thr, march=m)
        with fv.Solver(g, launch=d) as s:
            s.set_source(dev(S))
            R = s.residual(dev(U)).cpu().numpy()
            Ud = dev(U)
            s.run(Ud, 3)
            outs.append((R, Ud.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("case,scheme,dt_fixed", [
    ("ragged70x45_mixed_bc", {}, 0.0), ("kh256", dict(limiter=fv.FV_LIM_VANLEER), 0.0),
    ("box3d_36x20x14_mixed", dict(recon=fv.FV_RECON_PRIMITIVE), 0.0), ("kh256", {}, 1e-4)])
@pytest.mark.parametrize("nsteps", [1, 3])
def test_host_state_runs_with_source_equal_device_runs(case, scheme, dt_fixed, nsteps):
    """On a host state the first stage overlaps the copy in (per-axis flux
    differences band by band, then the stage-1 update formed from them):
    with a source, other scheme options and a fixed step the run still
    equals the device run bit for bit (page-locked and pageable host memory)."""
    g, U = CASES[case]()
    S = _source(g, U, 3)
    with fv.Solver(g, **scheme) as s:
        s.set_source(dev(S))
        Ud = dev(U)
        td = s.run(Ud, nsteps, dt_fixed, return_time=True)
        Uh = torch.from_numpy(U.copy()).pin_memory().numpy()
        th = s.run(Uh, nsteps, dt_fixed, return_time=True)
        Up = U.copy()
        tp = s.run(Up, nsteps, dt_fixed, return_time=True)
    assert np.array_equal(Ud.cpu().numpy(), Uh) and np.array_equal(Uh, Up)
    assert td == th == tp


def test_source_is_rejected_where_unsupported():
    g, U = I.isentropic_vortex(32)
    with fv.Solver([g, g]) as s:
        P = s.pack([dev(U), dev(U)])
        with pytest.raises(fv.FvError) as e:
            fv.fv_set_source(s.ctx, P)
        assert e.value.status == fv.FV_EUNSUPPORTED
    with fv.Solver(g) as s:
        with pytest.raises(fv.FvError) as e:
            fv.fv_set_source(s.ctx, U)  # a host array
        assert e.value.status == fv.FV_EINVAL


def test_fullsize_kh4096_primitive_reconstruction_with_source_sampled():
    """Kelvin-Helmholtz 4096x4096 (the benchmark grid) with reconstruction in
    primitive variables and a source set: the GPU residual on ~2100 sampled
    cells (domain edges and tile boundaries included) against the oracle's
    sampled residual with the same scheme and source, at the parity bar of
    the residual tests."""
    from test_gpu_parity import _sample_cells, assert_residual_parity
    g, U = I.kelvin_helmholtz(4096, seed=1)
    rng = np.random.default_rng(3)
    cells = _sample_cells(g, rng, 2000)
    so = O.scheme(recon=O.RECON_PRIMITIVE)
    scale = np.abs(O.residual_cells(g, U, cells, so)).max(axis=0)  # per variable
    vol = (g.length[0] / g.n[0]) * (g.length[1] / g.n[1])
    x = (np.arange(g.n[0]) + 0.5) / g.n[0]
    y = (np.arange(g.n[1]) + 0.5) / g.n[1]
    shape = np.sin(2 * np.pi * x)[None, :] * np.cos(4 * np.pi * y)[:, None]
    S = np.ascontiguousarray(np.stack([0.5 * scale[v] / vol * shape for v in range(g.nvar)]))
    with fv.Solver(g, recon=fv.FV_RECON_PRIMITIVE) as s:
        Sd = dev(S)
        s.set_source(Sd)
        R = s.residual(dev(U)).cpu().numpy().reshape(g.nvar, -1)[:, cells].T
    assert_residual_parity(g, U, R, cells, tag="kh4096-prim-source-sampled", s=so, S=S)
