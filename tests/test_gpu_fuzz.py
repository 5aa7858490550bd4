"""Launch-configuration fuzzing: every valid launch gives the same bits.

Random tile shapes, thread counts, loaders and (3D) kernels on ragged grids
with mixed boundaries; the residual and three RK steps must equal those of
the default launch bit for bit (every face flux is computed from the same
operands with the same arithmetic whatever the decomposition).  Catches
index arithmetic that only breaks at unusual tile/grid combinations.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2306_14011_gb300 import fv  # noqa: E402
from paper_2306_14011_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


def _random_launch(g, rng, dim):
    d = fv.launch_to_dict(fv.fv_default_launch(g))
    march = dim == 3 and rng.random() < 0.4
    tx = int(rng.choice([2, 4, 6, 8, 10, 16, 22, 32, 48, 64]))
    ty = int(rng.choice([1, 2, 3, 4, 5, 7, 8, 12, 16, 31, 32] if dim == 2 else [2, 3, 4, 5, 8, 15, 16]))
    ty = max(ty, 2)
    if dim == 2:
        tz = 1
    elif march:
        tz = int(rng.integers(1, 12))
    else:
        tz = int(rng.choice([2, 3, 4, 6, 8]))
    cap = 256 if (dim == 2 or march) else 192
    thr = int(rng.choice([t for t in (32, 64, 96, 128, 160, 192, 224, 256) if t <= cap]))
    loader = int(rng.integers(0, 2))
    for s in range(3):
        d["stage"][s].update(tile=(tx, ty, tz), threads=thr, loader=loader, march=int(march))
    d["dt"] = dict(threads=int(rng.choice([64, 128, 256, 512, 1024])), grid=int(rng.choice([0, 7, 152, 304])))
    return d


def _outputs(g, U, launch):
    with fv.Solver(g, launch=launch) as s:
        R = s.residual(torch.from_numpy(U).cuda()).cpu().numpy()
        Ud = torch.from_numpy(U).cuda()
        t = s.run(Ud, 3, return_time=True)
        return R, Ud.cpu().numpy(), t


@pytest.mark.parametrize("dim,seed", [(2, 0), (2, 1), (3, 2), (3, 3)])
def test_random_launches_give_identical_bits(dim, seed):
    rng = np.random.default_rng(seed)
    if dim == 2:
        g = I.grid2d(70, 53, 1.0, 0.8, ((0, 0), (1, 1), (0, 0)))
    else:
        g = I.grid3d(26, 19, 13, 1.0, 0.7, 0.5, ((1, 1), (0, 0), (1, 1)))
    U = I.random_smooth(g, seed=seed)
    R0, U0, t0 = _outputs(g, U, None)
    tried = 0
    while tried < 25:
        launch = _random_launch(g, rng, dim)
        try:
            R, U3, t = _outputs(g, U, launch)
        except fv.FvError as e:
            assert e.status == fv.FV_EINVAL, launch  # e.g. shared memory of a large tile
            continue
        tried += 1
        assert np.array_equal(R, R0), launch
        assert np.array_equal(U3, U0), launch
        assert t == t0, launch
