"""GPU tests of the autotuner (paper Sec. 3.3-3.6): the surrogate network's
kernels against the NumPy oracle, and fv_tune against the default launch and
the exhaustive search of the reduced space."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp as M  # noqa: E402
from paper_2306_14011_gb300 import fv  # noqa: E402
from paper_2306_14011_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


def _data(n, nin, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, nin))
    y = np.tanh(X[:, 0] - 0.5 * X[:, 1]) + 0.3 * X[:, 2] * X[:, 3] + 0.05 * rng.normal(size=n)
    return X, y


def _pack(params):
    return np.concatenate([p.ravel() for p in params])


def _unpack(flat, sizes):
    out, k = [], 0
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        out.append(flat[k:k + fi * fo].reshape(fi, fo))
        k += fi * fo
        out.append(flat[k:k + fo])
        k += fo
    return out


@pytest.mark.parametrize("sizes,epochs,stop", [([14, 32, 16, 1], 6, 1000), ([14, 128, 64, 32, 1], 3, 1000),
                                               ([5, 8, 1], 60, 10)])
def test_mlp_training_matches_numpy_oracle(sizes, epochs, stop):
    n = 430
    X, y = _data(n, sizes[0], 1)
    rng = np.random.default_rng(2)
    init = M.glorot_init(sizes, rng.random(M.n_params(sizes)))
    order = np.stack([rng.permutation(n) for _ in range(epochs)]).astype(np.int32)
    hyper = dict(n_iter_no_change=stop)
    if stop == 10:
        hyper["lr"] = 1e-7  # the loss stalls: early stopping must fire at the same epoch on both sides
    ref = [p.copy() for p in init]
    losses_ref = M.train(ref, X, y, order, hyper)
    P = torch.from_numpy(_pack(init)).cuda()
    losses = fv.fv_mlp_train(sizes, P, torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(),
                             torch.from_numpy(order).cuda(), fv.mlp_hyper(**hyper))
    assert len(losses) == len(losses_ref)
    np.testing.assert_allclose(losses, losses_ref, rtol=1e-12)
    got = _unpack(P.cpu().numpy(), sizes)
    for a, b in zip(got, ref):
        assert np.abs(a - b).max() <= 1e-10 * max(np.abs(b).max(), 1e-3)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    fv.fv_mlp_predict(sizes, P, torch.from_numpy(X).cuda(), out)
    np.testing.assert_allclose(out.cpu().numpy(), M.predict(got, X), rtol=1e-13, atol=1e-13)


def test_tuner_beats_default_and_matches_exhaustive_search():
    g, U = I.kelvin_helmholtz(1024, seed=1)
    Ud = torch.from_numpy(U).cuda()
    with fv.Solver(g) as s:
        R_default = s.residual(Ud).clone()
        best, rep = s.tune(Ud, samples=300, candidates=50000, top=16, rounds=3, refine=2, exhaustive=1, steps=3,
                           final_repeats=7, seed=7)
        path = os.environ.get("FV_TUNE_REPORT")
        if path:
            with open(path, "a") as f:
                f.write(json.dumps({"workload": "kh1024", "best": best, "report": rep}) + "\n")
        assert rep["n_params"] == 14
        assert rep["space_size"] == float((5 * 5 * 7 * 2) ** 3 * 4 * 4)
        assert 0.15 < rep["n_test"] / 300 < 0.35 and rep["n_train"] + rep["n_test"] >= 300
        assert rep["rounds"] == 3 and rep["n_exhaustive"] > 100
        assert torch.equal(Ud, torch.from_numpy(U).cuda())  # tuning ran on a copy
        assert s.launch == best
        # the tuned launch changes speed only
        assert torch.equal(s.residual(Ud), R_default)
        # the surrogate predicts held-out configurations better than their mean does
        assert rep["r2_test"] > 0.0
        # the returned launch is the fastest of the search's pick, the default and
        # the exhaustive search; the search alone (which starts from the default)
        # is within 3% timing noise of both
        assert rep["t_tuned"] <= min(rep["t_default"], rep["t_search"])
        assert rep["chosen"] in (0, 1, 2)
        assert rep["t_search"] <= rep["t_default"] * 1.03
        assert rep["t_search"] <= rep["t_exhaustive"] * 1.03


def test_tuner_3d_space_includes_the_marching_kernel():
    """A short 3D search: 20 parameters (box or z-marching per stage); the
    installed launch changes speed only."""
    g, U = I.taylor_green(48, seed=2)
    Ud = torch.from_numpy(U).cuda()
    with fv.Solver(g) as s:
        R_default = s.residual(Ud).clone()
        best, rep = s.tune(Ud, samples=40, candidates=20000, top=8, rounds=1, refine=1, exhaustive=0, steps=2,
                           final_repeats=3, seed=3)
        assert rep["n_params"] == 20
        assert rep["space_size"] == float((3 * 3 * 3 * 7 * 2 * 2) ** 3 * 4 * 4)
        assert s.launch == best
        assert rep["t_tuned"] <= rep["t_default"]
        assert torch.equal(s.residual(Ud), R_default)
