"""GPU time-step reduction (with its FP32 pre-selection) against the oracle.

The reduction evaluates in FP64 only the cells whose certified FP32 upper
bound reaches the largest certified lower bound, so its result must still be
the exact FP64 maximum.  These cases put the maximum where a wrong selection
would show: among near-ties, at cells whose FP32 evaluation is not certified
(cancellation in the pressure, a density outside the certified range), next
to a runner-up 1e-9 below it, and on a grid whose spacing switches the
pre-selection off.  A miss would change dt by at least the gap between the
two largest wave-speed sums (1e-12 and more here), far above the 2e-15 bar.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2306_14011_gb300 import fv  # noqa: E402
from paper_2306_14011_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 2e-15


def dev(U):
    return torch.from_numpy(np.ascontiguousarray(U)).cuda()


def check(g, U):
    with fv.Solver(g) as s:
        dt = s.time_step(dev(U))
        dtd = torch.zeros(1, dtype=torch.float64, device="cuda")
        fv.fv_time_step(s.ctx, dev(U), dtd)
        torch.cuda.synchronize()
    dto = O.time_step(g, U)
    assert abs(dt - dto) <= TOL * dto, (dt, dto)
    assert dtd.item() == dt
    return dt


def grid(dim, n=48):
    return I.grid2d(n, n - 5, 1.0, 0.9) if dim == 2 else I.grid3d(n // 2, n // 2 - 3, n // 2 - 5, 1.0, 0.9, 0.7)


def set_cell(g, U, idx, rho, vel, p):
    U[(slice(None),) + idx] = I.conserved(np.array(rho), tuple(np.array(v) for v in vel), np.array(p))


@pytest.mark.parametrize("dim", [2, 3])
def test_near_ties_everywhere(dim):
    """Uniform flow with 1e-12 pressure noise: every cell is a candidate."""
    g = grid(dim)
    rng = np.random.default_rng(1)
    p = 0.9 * (1.0 + 1e-12 * rng.standard_normal(g.shape[1:]))
    U = I.conserved(np.ones(g.shape[1:]), tuple(np.full(g.shape[1:], v) for v in (0.3, -0.2, 0.1)[:dim]), p)
    check(g, U)


@pytest.mark.parametrize("dim", [2, 3])
def test_maximum_at_cell_with_cancelling_pressure(dim):
    """A hypersonic cell (kinetic energy 1e9 times the internal energy): its
    FP32 pressure is not certified, and it holds the maximum."""
    g = grid(dim)
    U = I.random_smooth(g, seed=3)
    idx = (3, 5) if dim == 2 else (2, 3, 5)
    set_cell(g, U, idx, 1.0, (500.0, 0.0, 0.0)[:dim], 1e-4)
    check(g, U)


@pytest.mark.parametrize("dim", [2, 3])
def test_maximum_at_density_outside_certified_range(dim):
    g = grid(dim)
    U = I.random_smooth(g, seed=4)
    idx = (7, 11) if dim == 2 else (4, 6, 8)
    set_cell(g, U, idx, 1e-12, (0.1, 0.0, 0.0)[:dim], 1.0)
    check(g, U)


@pytest.mark.parametrize("dim", [2, 3])
def test_runner_up_within_1e_9(dim):
    """Two fast certified cells 1e-9 apart, the rest far below."""
    g = grid(dim)
    U = I.uniform_state(g)
    a = (10, 20) if dim == 2 else (3, 7, 9)
    b = (30, 2) if dim == 2 else (8, 2, 1)
    set_cell(g, U, a, 1.0, (2.0, 0.0, 0.0)[:dim], 0.9)
    set_cell(g, U, b, 1.0, (2.0 * (1.0 + 1e-9), 0.0, 0.0)[:dim], 0.9)
    dt_b = check(g, U)
    set_cell(g, U, b, 1.0, (2.0 * (1.0 - 1e-9), 0.0, 0.0)[:dim], 0.9)
    dt_a = check(g, U)
    assert dt_a > dt_b


def test_preselection_off_for_tiny_spacing():
    """1/dx above 2^30 switches the FP32 pre-selection off."""
    g = I.grid2d(40, 33, 40e-10, 33e-10)
    U = I.random_smooth(g, seed=5)
    check(g, U)


@pytest.mark.parametrize("n", [(1, 1), (3, 5), (7, 1), (1, 9)])
def test_tiny_and_ragged_grids(n):
    g = I.grid2d(n[0], n[1], 1.0, 1.0)
    check(g, I.random_smooth(g, seed=6))


def test_negative_pressure_behind_cancellation_is_reported():
    """E just below the kinetic energy: p < 0 in FP64, undecidable in FP32."""
    g = grid(2)
    U = I.random_smooth(g, seed=7)
    U[:, 4, 4] = [1.0, 100.0, 0.0, 0.5 * 100.0 ** 2 * (1.0 - 1e-13)]
    with fv.Solver(g) as s:
        with pytest.raises(fv.FvError) as e:
            s.time_step(dev(U))
        assert e.value.status == fv.FV_ENONPHYSICAL
