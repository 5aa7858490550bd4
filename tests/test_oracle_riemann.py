"""Pins of the exact Riemann solver that the Sod convergence test relies on.

Checked against (a) the star state printed in Toro's textbook for Sod's
problem (tests/golden/sod_star_state.txt) and (b) the physics that fixes it:
Rankine-Hugoniot conditions across the shock, isentropy and the Riemann
invariant across the rarefaction, and continuity of p and u at the contact.
"""
import math
import os

import numpy as np
import pytest

from oracle import riemann_exact as RE

G = 1.4
SOD_L = (1.0, 0.0, 1.0)
SOD_R = (0.125, 0.0, 0.1)
HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    vals = {}
    with open(os.path.join(HERE, "golden", "sod_star_state.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_sod_star_state_matches_textbook():
    ref = _golden()
    p, u = RE.star_state(SOD_L, SOD_R, G)
    assert abs(p - ref["p_star"]) < 1e-5
    assert abs(u - ref["u_star"]) < 1e-5
    # densities next to the contact: sample just left / right of x/t = u*
    rho, uu, pp = RE.sample(SOD_L, SOD_R, np.array([u - 1e-9, u + 1e-9]), G)
    assert abs(rho[0] - ref["rho_star_left"]) < 1e-5
    assert abs(rho[1] - ref["rho_star_right"]) < 1e-5


def _energy(rho, u, p):
    return p / (G - 1) + 0.5 * rho * u * u


def test_rankine_hugoniot_across_right_shock():
    p, u = RE.star_state(SOD_L, SOD_R, G)
    rr, ur, pr = SOD_R
    cr = math.sqrt(G * pr / rr)
    S = ur + cr * math.sqrt((G + 1) / (2 * G) * p / pr + (G - 1) / (2 * G))
    rho, uu, pp = RE.sample(SOD_L, SOD_R, np.array([S - 1e-9, S + 1e-9]), G)
    # mass, momentum and energy fluxes in the shock frame are continuous
    a = (rho[0], uu[0], pp[0])
    b = (rho[1], uu[1], pp[1])
    for (r1, u1, p1), (r2, u2, p2) in [(a, b)]:
        m1, m2 = r1 * (u1 - S), r2 * (u2 - S)
        assert abs(m1 - m2) < 1e-12
        assert abs((r1 * u1 * (u1 - S) + p1) - (r2 * u2 * (u2 - S) + p2)) < 1e-12
        assert abs((_energy(r1, u1, p1) * (u1 - S) + p1 * u1) - (_energy(r2, u2, p2) * (u2 - S) + p2 * u2)) < 1e-12


def test_left_rarefaction_is_isentropic_with_constant_invariant():
    p, u = RE.star_state(SOD_L, SOD_R, G)
    rl, ul, pl = SOD_L
    cl = math.sqrt(G * pl / rl)
    cs = cl * (p / pl) ** ((G - 1) / (2 * G))
    xi = np.linspace(ul - cl, u - cs, 17)
    rho, uu, pp = RE.sample(SOD_L, SOD_R, xi, G)
    s = pp / rho ** G
    assert np.max(np.abs(s - pl / rl ** G)) < 1e-12
    c = np.sqrt(G * pp / rho)
    J = uu + 2 * c / (G - 1)
    assert np.max(np.abs(J - (ul + 2 * cl / (G - 1)))) < 1e-12
    # inside the fan the flow is sonic relative to the ray: u - c = x/t
    assert np.max(np.abs((uu - c)[1:-1] - xi[1:-1])) < 1e-12


def test_contact_continuity_and_far_field():
    p, u = RE.star_state(SOD_L, SOD_R, G)
    rho, uu, pp = RE.sample(SOD_L, SOD_R, np.array([u - 1e-7, u + 1e-7, -10.0, 10.0]), G)
    assert abs(pp[0] - pp[1]) < 1e-14 and abs(uu[0] - uu[1]) < 1e-14
    assert (rho[2], uu[2], pp[2]) == SOD_L
    assert (rho[3], uu[3], pp[3]) == SOD_R


@pytest.mark.parametrize("left,right", [((1.0, -2.0, 0.4), (1.0, 2.0, 0.4)),      # two rarefactions
                                        ((1.0, 2.0, 0.4), (1.0, -2.0, 0.4)),      # two shocks
                                        ((5.99924, 19.5975, 460.894), (5.99242, -6.19633, 46.0950))])
def test_star_state_solves_the_pressure_equation(left, right):
    p, u = RE.star_state(left, right, G)
    # both one-sided relations give the same star velocity
    fl, _ = RE._fk(p, left[0], left[2], math.sqrt(G * left[2] / left[0]), G)
    fr, _ = RE._fk(p, right[0], right[2], math.sqrt(G * right[2] / right[0]), G)
    assert abs((left[1] - fl) - u) < 1e-10 * max(1.0, abs(u))
    assert abs((right[1] + fr) - u) < 1e-10 * max(1.0, abs(u))
