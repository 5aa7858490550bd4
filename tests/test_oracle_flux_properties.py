"""Property checks of the oracle's Roe flux on generated state pairs (CPU;
skipped where hypothesis is not installed).

* By Roe's property the central flux (F(QL) + F(QR))/2 - sum |lambda| alpha
  r / 2 equals the upwind physical flux plus the one acoustic wave that
  crosses from downwind (the form the GPU kernels evaluate), for density
  ratios up to 1e3, Mach numbers up to 5, both signs of the normal velocity
  and entropy-fix widths below 1;
* consistency: F(Q, Q) = F(Q) bitwise;
* mirror symmetry: reflecting both states across the face (swap sides, flip
  the normal velocity) flips the normal-momentum flux's partner signs:
  F_n(QL, QR) = -P F_n(P QR, P QL) with P the reflection.
"""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_2306_14011_gb300 import inputs as I  # noqa: E402

G = 1.4


def _state(rho, vel, p):
    return I.conserved(np.array(rho), tuple(np.array(v) for v in vel), np.array(p))


def _states(dim):
    rho = st.floats(1e-3, 1e3)
    pres = st.floats(1e-3, 1e3)
    mach = st.lists(st.floats(-5.0, 5.0), min_size=dim, max_size=dim)

    def build(r, m, p):
        c = np.sqrt(G * p / r)
        return _state(r, [mi * c for mi in m], p)

    return st.builds(build, rho, mach, pres)


def _one_wave(ql, qr, d, dim, efix):
    g1 = G - 1
    rl, rr = ql[0], qr[0]
    ul, ur = ql[1:1 + dim] / rl, qr[1:1 + dim] / rr
    pl = g1 * (ql[-1] - 0.5 * rl * ul @ ul)
    pr = g1 * (qr[-1] - 0.5 * rr * ur @ ur)
    Hl, Hr = (ql[-1] + pl) / rl, (qr[-1] + pr) / rr
    wl, wr = np.sqrt(rl), np.sqrt(rr)
    u = (wl * ul + wr * ur) / (wl + wr)
    H = (wl * Hl + wr * Hr) / (wl + wr)
    rho = wl * wr
    c = np.sqrt(g1 * (H - 0.5 * u @ u))
    un = u[d]
    sg = 1.0 if un >= 0 else -1.0
    x = abs(un) - c
    delta = efix * c
    k = (x - (x * x + delta * delta) / (2 * delta)) / 2 if abs(x) < delta else min(x, 0.0)
    alpha = (pr - pl) / (2 * c * c) - sg * rho * (ur[d] - ul[d]) / (2 * c)
    r = np.concatenate([[1.0], u, [H - c * abs(un)]])
    r[1 + d] = un - sg * c
    return O.physical_flux(ql if sg > 0 else qr, d) + k * alpha * r


@pytest.mark.parametrize("dim", [2, 3])
def test_upwind_one_wave_form_equals_the_oracle_flux(dim):
    @settings(max_examples=300, deadline=None)
    @given(_states(dim), _states(dim), st.integers(0, dim - 1), st.sampled_from([0.0, 0.05, 0.1, 0.5, 0.95]))
    def check(ql, qr, d, efix):
        Fo = O.roe_flux(ql, qr, d, dim, O.scheme(efix=efix))
        F = _one_wave(ql, qr, d, dim, efix)
        scale = max(np.abs(O.physical_flux(ql, d)).max(), np.abs(O.physical_flux(qr, d)).max(), np.abs(Fo).max())
        assert np.abs(F - Fo).max() <= 1e-11 * scale

    check()


@pytest.mark.parametrize("dim", [2, 3])
def test_consistency_and_mirror_symmetry(dim):
    @settings(max_examples=200, deadline=None)
    @given(_states(dim), _states(dim), st.integers(0, dim - 1))
    def check(ql, qr, d):
        s = O.scheme()
        np.testing.assert_array_equal(O.roe_flux(ql, ql, d, dim, s), O.physical_flux(ql, d))
        P = np.ones(dim + 2)
        P[1 + d] = -1.0  # reflection across the face
        F = O.roe_flux(ql, qr, d, dim, s)
        Fm = O.roe_flux(P * qr, P * ql, d, dim, s)
        scale = max(np.abs(F).max(), np.abs(O.physical_flux(ql, d)).max(), np.abs(O.physical_flux(qr, d)).max())
        assert np.abs(F + P * Fm).max() <= 1e-12 * scale

    check()
