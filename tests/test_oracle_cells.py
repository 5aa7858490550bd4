"""Pin of the oracle's sampled residual (residual_cells) against its full residual.

residual_cells is the checker of the GPU parity tests at full size (4096^2,
384^3), where the full oracle residual is too slow.  It evaluates each listed
cell's two faces per axis from their stencils, reading every stencil cell
through the boundary map instead of a ghost-padded copy, so a wrong stencil
offset or ghost index would show up here as a mismatch against the full
residual of Eq. (5) (which is pinned by test_oracle_pins.py).  Both sum the
same face fluxes in the same order, so they must agree bit for bit: every
cell of small and odd grids (every edge and corner cell, every boundary
combination), every scheme option the oracle has, with and without a source.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2306_14011_gb300 import inputs as I

T, P = I.BC_TRANSMISSIVE, I.BC_PERIODIC

GRIDS = {
    "2d_4x4_periodic": lambda: I.grid2d(4, 4, 1.0, 1.0),
    "2d_5x7_transmissive": lambda: I.grid2d(5, 7, 1.0, 1.4, T),
    "2d_6x5_mixed": lambda: I.grid2d(6, 5, 1.0, 0.7, ((T, T), (P, P), (P, P))),
    "2d_9x3_mixed_other": lambda: I.grid2d(9, 3, 1.3, 0.4, ((P, P), (T, T), (P, P))),
    "3d_4x4x4_periodic": lambda: I.grid3d(4, 4, 4, 1.0, 1.0, 1.0),
    "3d_10x7x9_transmissive": lambda: I.grid3d(10, 7, 9, 1.0, 0.7, 0.9, T),
    "3d_5x6x7_mixed": lambda: I.grid3d(5, 6, 7, 1.0, 0.6, 0.5, ((P, P), (T, T), (P, P))),
    "3d_6x5x4_mixed_z": lambda: I.grid3d(6, 5, 4, 0.6, 0.5, 0.4, ((T, T), (P, P), (T, T))),
}

SCHEMES = {
    "minmod": lambda: O.scheme(),
    "vanleer": lambda: O.scheme(limiter=O.LIM_VANLEER),
    "kappa_third": lambda: O.scheme(limiter=O.LIM_NONE, kappa=1.0 / 3.0),
    "central": lambda: O.scheme(limiter=O.LIM_NONE, kappa=1.0),
    "primitive": lambda: O.scheme(recon=O.RECON_PRIMITIVE),
    "first_order": lambda: O.scheme(eps=0.0),
    "no_entropy_fix": lambda: O.scheme(efix=0.0),
}


@pytest.mark.parametrize("scheme", sorted(SCHEMES))
@pytest.mark.parametrize("grid", sorted(GRIDS))
@pytest.mark.parametrize("with_source", [False, True])
def test_residual_cells_equal_the_full_residual_bitwise(grid, scheme, with_source):
    g = GRIDS[grid]()
    s = SCHEMES[scheme]()
    U = I.random_smooth(g, seed=11)
    S = np.random.default_rng(5).normal(size=U.shape) if with_source else None
    R = O.residual(g, U, s, S=S).reshape(g.nvar, -1)
    cells = np.arange(g.ncells, dtype=np.int64)
    Rc = O.residual_cells(g, U, cells, s, S=S)
    np.testing.assert_array_equal(Rc, R.T)
    # extended precision: the same agreement against the full long-double residual
    Rx = O.residual_ext(g, U, s, S=S).reshape(g.nvar, -1)
    np.testing.assert_array_equal(O.residual_cells(g, U, cells, s, extended=True, S=S), Rx.T)


def test_residual_cells_in_any_order_and_with_repeats():
    g = I.grid2d(11, 8, 1.0, 0.8, ((T, T), (P, P), (P, P)))
    U = I.random_smooth(g, seed=12)
    R = O.residual(g, U).reshape(g.nvar, -1)
    rng = np.random.default_rng(0)
    cells = rng.integers(0, g.ncells, 300)
    np.testing.assert_array_equal(O.residual_cells(g, U, cells), R[:, cells].T)
    assert O.residual_cells(g, U, np.zeros(0, dtype=np.int64)).shape == (0, g.nvar)


def test_residual_cells_rejects_indices_outside_the_grid():
    g = I.grid2d(5, 4, 1.0, 1.0)
    U = I.random_smooth(g, seed=1)
    for bad in ([-1], [g.ncells]):
        with pytest.raises(ValueError):
            O.residual_cells(g, U, np.array(bad, dtype=np.int64))
