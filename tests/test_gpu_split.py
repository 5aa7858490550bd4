"""The split kernel structure (launch mode FV_SPLIT: per axis a limiter and a
flux kernel, then source, right-hand-side and update kernels, Sec. 3.4)
against the oracle, with the bars of the fused path: residual 1e-12 of
max|R_v| (or 4x the oracle's own rounding error), one RK step 1e-12, 100
steps 1e-9.  Each face and cell is computed by one thread from the same
operands whatever the gang count and vector length, so results are bitwise
independent of the split launch parameters.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2306_14011_gb300 import fv  # noqa: E402
from paper_2306_14011_gb300 import inputs as I  # noqa: E402
from test_gpu_parity import CASES, _sample_cells, assert_residual_parity, dev, relerr, TOL_RES, TOL_100  # noqa: E402
from test_gpu_source import _source  # noqa: E402

pytestmark = pytest.mark.gpu

GANG = list(range(100, 1001, 100))
VECTOR = list(range(32, 385, 32))


def split_launch(g, grid=None, threads=None, rng=None):
    """The default launch in FV_SPLIT mode; grid/threads set every split
    kernel, rng draws each kernel's pair from the paper's value sets (and
    grid 0)."""
    d = fv.launch_to_dict(fv.fv_default_launch(g))
    d["mode"] = fv.FV_SPLIT
    for k in range(fv.FV_SK_COUNT):
        if rng is not None:
            d["split"][k] = dict(grid=int(rng.choice(GANG + [0])), threads=int(rng.choice(VECTOR + [512])))
        else:
            if grid is not None:
                d["split"][k]["grid"] = grid
            if threads is not None:
                d["split"][k]["threads"] = threads
    return d


@pytest.mark.parametrize("case", sorted(CASES))
def test_residual_matches_oracle(case):
    g, U = CASES[case]()
    with fv.Solver(g, mode=fv.FV_SPLIT) as s:
        R = s.residual(dev(U)).cpu().numpy()
    assert_residual_parity(g, U, R, tag=f"split-{case}")


@pytest.mark.parametrize("case", ["vortex128", "kh256", "sod_rot64_transmissive", "ragged70x45_mixed_bc", "tgv24",
                                  "box3d_36x20x14_mixed"])
@pytest.mark.parametrize("cfl_dt", [False, True])
def test_rk_step_matches_oracle(case, cfl_dt):
    g, U = CASES[case]()
    dto = O.time_step(g, U)
    Uo, _ = O.rk3_step(g, U, dto)
    with fv.Solver(g, mode=fv.FV_SPLIT) as s:
        Ud = dev(U)
        used = s.rk_step(Ud, 0.0 if cfl_dt else dto, return_dt=True)
        U1 = Ud.cpu().numpy()
    assert abs(used - dto) <= 2e-15 * dto
    assert relerr(U1, Uo) <= TOL_RES


def test_config1_vortex_100_steps_matches_oracle():
    g, U = I.isentropic_vortex(128, seed=0)
    Uo, to = O.run(g, U, 100)
    with fv.Solver(g, mode=fv.FV_SPLIT) as s:
        Ud = dev(U)
        t = s.run(Ud, 100, return_time=True)
        Uh = U.copy()
        th = s.run(Uh, 100, return_time=True)  # host state: the same graphs, copy in and out
    assert abs(t - to) <= 1e-12 * to
    assert relerr(Ud.cpu().numpy(), Uo) <= TOL_100
    assert np.array_equal(Ud.cpu().numpy(), Uh) and t == th


@pytest.mark.parametrize("lim,kappa,recon", [(fv.FV_LIM_VANLEER, -1.0, fv.FV_RECON_CONSERVED),
                                             (fv.FV_LIM_NONE, 1.0 / 3.0, fv.FV_RECON_CONSERVED),
                                             (fv.FV_LIM_NONE, 1.0, fv.FV_RECON_CONSERVED),
                                             (fv.FV_LIM_MINMOD, -1.0, fv.FV_RECON_PRIMITIVE),
                                             (fv.FV_LIM_VANLEER, -1.0, fv.FV_RECON_PRIMITIVE)])
@pytest.mark.parametrize("case", ["vortex128", "ragged70x45_mixed_bc", "tgv24", "box3d_10x7x9_transmissive"])
def test_scheme_variants_match_oracle(case, lim, kappa, recon):
    g, U = CASES[case]()
    so = O.scheme(limiter=lim, kappa=kappa, recon=recon)
    dto = O.time_step(g, U, so)
    with fv.Solver(g, limiter=lim, kappa=kappa, recon=recon, mode=fv.FV_SPLIT) as s:
        R = s.residual(dev(U)).cpu().numpy()
        Ud = dev(U)
        s.rk_step(Ud, dto)
        U1 = Ud.cpu().numpy()
    assert_residual_parity(g, U, R, tag=f"split-{case}-lim{lim}-k{kappa}-r{recon}", s=so)
    assert relerr(U1, O.rk3_step(g, U, dto, so)[0]) <= TOL_RES


@pytest.mark.parametrize("case", ["vortex128", "ragged70x45_mixed_bc", "box3d_36x20x14_mixed"])
def test_source_term_matches_oracle(case):
    g, U = CASES[case]()
    S = _source(g, U, 11)
    dto = O.time_step(g, U)
    with fv.Solver(g, mode=fv.FV_SPLIT) as s:
        s.set_source(dev(S))
        R = s.residual(dev(U)).cpu().numpy()
        Ud = dev(U)
        s.rk_step(Ud, dto)
        U1 = Ud.cpu().numpy()
    Ro = O.residual(g, U, S=S).reshape(g.nvar, -1)
    scale = np.abs(Ro).max(axis=1)
    assert np.all(np.abs(R.reshape(g.nvar, -1) - Ro).max(axis=1) <= 4 * TOL_RES * scale)
    assert relerr(U1, O.rk3_step(g, U, dto, S=S)[0]) <= TOL_RES


def test_residual_norms_are_the_sums_of_squares():
    g, U = I.kelvin_helmholtz(256, seed=1)
    with fv.Solver(g, launch=split_launch(g, grid=300, threads=96)) as s:
        R, nrm = s.residual(dev(U), norms=True)
    own = (R.cpu().numpy().reshape(g.nvar, -1) ** 2).sum(axis=1)
    assert np.max(np.abs(nrm.cpu().numpy() - own) / own) <= 1e-13


@pytest.mark.parametrize("dim,seed", [(2, 0), (3, 1)])
def test_split_launch_parameters_do_not_change_results(dim, seed):
    """Random (gang, vector) per kernel from the paper's value sets: bitwise
    the same residual, states and simulated time; and within rounding of the
    fused kernels."""
    if dim == 2:
        g = I.grid2d(70, 53, 1.0, 0.8, ((0, 0), (1, 1), (0, 0)))
    else:
        g = I.grid3d(26, 19, 13, 1.0, 0.7, 0.5, ((1, 1), (0, 0), (1, 1)))
    U = I.random_smooth(g, seed=seed)
    rng = np.random.default_rng(seed)
    outs = []
    for q in range(8):
        launch = split_launch(g) if q == 0 else split_launch(g, rng=rng)
        with fv.Solver(g, launch=launch) as s:
            R = s.residual(dev(U)).cpu().numpy()
            Ud = dev(U)
            t = s.run(Ud, 3, return_time=True)
            outs.append((R, Ud.cpu().numpy(), t))
    for R, U3, t in outs[1:]:
        assert np.array_equal(R, outs[0][0]) and np.array_equal(U3, outs[0][1]) and t == outs[0][2]
    with fv.Solver(g) as s:
        Rf = s.residual(dev(U)).cpu().numpy()
        Uf = dev(U)
        tf = s.run(Uf, 3, return_time=True)
    assert relerr(outs[0][0], Rf) <= 1e-12 and relerr(outs[0][1], Uf.cpu().numpy()) <= 1e-13
    assert abs(tf - outs[0][2]) <= 1e-14 * tf  # same time-step kernels on nearly the same states


def test_switching_modes_on_one_context():
    g, U = I.isentropic_vortex(96, seed=3)
    with fv.Solver(g) as s:
        Rf = s.residual(dev(U)).cpu().numpy()
        s.launch = split_launch(g, grid=200, threads=64)
        assert s.launch["mode"] == fv.FV_SPLIT
        Rs = s.residual(dev(U)).cpu().numpy()
        Ud = dev(U)
        s.run(Ud, 4)
        s.launch = fv.launch_to_dict(fv.fv_default_launch(g))
        Rf2 = s.residual(dev(U)).cpu().numpy()
    with fv.Solver(g, launch=split_launch(g)) as s2:
        Ud2 = dev(U)
        s2.run(Ud2, 4)
    assert np.array_equal(Rf, Rf2)
    assert relerr(Rs, Rf) <= 1e-12
    assert torch.equal(Ud, Ud2)


def test_fullsize_kh4096_residual_and_step_sampled():
    """KH 4096^2 with the split kernels at their default launch: residual on
    sampled cells, and a CFL step against the fused kernels' step."""
    g, U = I.kelvin_helmholtz(4096, seed=1)
    rng = np.random.default_rng(2)
    cells = _sample_cells(g, rng, 2000)
    with fv.Solver(g, mode=fv.FV_SPLIT) as s:
        Ud = dev(U)
        R = s.residual(Ud).cpu().numpy().reshape(g.nvar, -1)[:, cells].T
        used = s.rk_step(Ud, 0.0, return_dt=True)
        U1s = Ud.cpu().numpy()
    assert_residual_parity(g, U, R, cells, tag="split-kh4096-sampled")
    with fv.Solver(g) as s:
        Uf = dev(U)
        usedf = s.rk_step(Uf, 0.0, return_dt=True)
        U1f = Uf.cpu().numpy()
    assert used == usedf
    assert relerr(U1s, U1f) <= 1e-13


def test_split_mode_rejections():
    g, U = I.isentropic_vortex(32)
    for bad in [dict(threads=48), dict(threads=544), dict(threads=0), dict(grid=-1)]:
        d = split_launch(g)
        d["split"][fv.FV_SK_FLUX].update(bad)
        with pytest.raises(fv.FvError) as e:
            fv.Solver(g, launch=d)
        assert e.value.status == fv.FV_EINVAL
    d = split_launch(g)
    d["mode"] = 2
    with pytest.raises(fv.FvError) as e:
        fv.Solver(g, launch=d)
    assert e.value.status == fv.FV_EINVAL
    with fv.Solver([g, g]) as s:  # batched contexts run the fused persistent kernel only
        with pytest.raises(fv.FvError) as e:
            s.launch = split_launch(g)
        assert e.value.status == fv.FV_EUNSUPPORTED


def test_tuner_searches_the_papers_space():
    """The tuner on the split kernels: the paper's 14 parameters and 10^7 x
    12^7 points; the exhaustive search times 120 shared (gang, vector) pairs; the
    returned launch is a valid split launch no slower than the default."""
    g, U = I.kelvin_helmholtz(256, seed=1)
    with fv.Solver(g, mode=fv.FV_SPLIT) as s:
        best, rep = s.tune(dev(U), samples=60, candidates=2000, top=4, rounds=2, refine=1, exhaustive=1,
                           steps=2, final_repeats=3, seed=5)
        assert rep["n_params"] == 14 and rep["space_size"] == float(10 ** 7 * 12 ** 7)
        assert rep["n_exhaustive"] == 120
        assert best["mode"] == fv.FV_SPLIT and s.launch == best
        assert rep["t_tuned"] <= rep["t_default"]
        if rep["chosen"] == 0:
            for slot in [0, 1, 3, 4, 6, 7, 8]:
                assert best["split"][slot]["grid"] in GANG and best["split"][slot]["threads"] in VECTOR
        R = s.residual(dev(U)).cpu().numpy()
    assert_residual_parity(g, U, R, tag="split-tuned")
