"""Batched grids (many independent 2D problems, one persistent cooperative
launch per call, per-problem CFL steps) against single-grid runs of the same
problems (bitwise: the same tile routine and exact max reductions) and the
CPU oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2306_14011_gb300 import fv  # noqa: E402
from paper_2306_14011_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


def _relerr(a, b):
    return max(np.abs(a[v] - b[v]).max() / np.abs(b[v]).max() for v in range(b.shape[0]))


def _problems(sizes_angles):
    return [I.sod_rotated(n, th) for n, th in sizes_angles]


def _single(g, U, nsteps, dt_fixed=0.0):
    with fv.Solver(g) as s:
        Ud = torch.from_numpy(U).cuda()
        t = s.run(Ud, nsteps, dt_fixed, return_time=True)
        return Ud.cpu().numpy(), t


@pytest.mark.parametrize("loader", [fv.FV_LOADER_TMA, fv.FV_LOADER_PLAIN])
@pytest.mark.parametrize("dt_fixed", [0.0, 2e-4])
def test_small_batch_matches_single_grid_runs_and_oracle(dt_fixed, loader):
    """Sizes below, at and above the 36-cell tile + halo box of the 32x32
    tiles, odd and even widths: with the TMA loader the even ones of at least
    36 cells load by TMA (36: the box spans the whole grid), the others by
    plain loads; with the plain loader all of them."""
    rng = np.random.default_rng(11)
    sizes = [8, 13, 16, 31, 40, 47, 64, 70, 5, 36, 35]
    specs = [(int(n), float(th)) for n, th in zip(sizes, rng.uniform(0, 2 * np.pi, len(sizes)))]
    probs = _problems(specs)
    grids = [g for g, _ in probs]
    with fv.Solver(grids) as s:
        d = s.launch
        for st in d["stage"]:
            st["loader"] = loader
        s.launch = d
        assert s.offsets[0] == 0 and all(o % 32 == 0 for o in s.offsets)
        U = s.pack([torch.from_numpy(u).cuda() for _, u in probs])
        t = s.run(U, 10, dt_fixed, return_time=True)
        outs = [x.cpu().numpy() for x in s.unpack(U)]
    for (g, u0), out, tb in zip(probs, outs, t):
        ref, ts = _single(g, u0, 10, dt_fixed)
        assert np.array_equal(out, ref)
        assert tb == ts
        uo, to = O.run(g, u0, 10, dt_fixed)
        assert abs(tb - to) <= 1e-13 * to
        assert _relerr(out, uo) <= 1e-11


def test_batched_sod_config_96_problems_50_steps():
    """96 rotated Sod problems, sizes log-uniform in [64, 2048] (seed 3),
    transmissive boundaries, 50 CFL steps in one persistent launch (the
    default launch: TMA tile loads for the even widths)."""
    specs = I.batched_sod(96, seed=3)
    probs = _problems(specs)
    grids = [g for g, _ in probs]
    with fv.Solver(grids) as s:
        U = s.pack([torch.from_numpy(u).cuda() for _, u in probs])
        t = s.run(U, 50, return_time=True)
        outs = [x.cpu().numpy() for x in s.unpack(U)]
    order = np.argsort([n for n, _ in specs])
    # every problem equals its own single-grid run, bitwise (small ones and the largest)
    for i in list(order[:24]) + [order[-1]]:
        g, u0 = probs[i]
        ref, ts = _single(g, u0, 50)
        assert np.array_equal(outs[i], ref), i
        assert t[i] == ts
    # and the smallest against the oracle
    for i in order[:6]:
        g, u0 = probs[i]
        uo, to = O.run(g, u0, 50)
        assert abs(t[i] - to) <= 1e-12 * to
        assert _relerr(outs[i], uo) <= 1e-10
