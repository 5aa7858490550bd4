"""Algorithmic floating-point work of the method, counted on the oracle.

Runs the oracle with an operation-counting scalar type (each +, -, *, /, sqrt
is one FLOP; comparisons, fabs and negation are free) on small states of the
benchmark workloads and prints FLOPs per cell and RK stage:
  per cell-stage = (one SSP-RK3 step + one CFL time step) / (3 * cells).
These are the "algorithmic FLOPs" of the roofline the benchmark reports.
Usage: python -m oracle.count_flops
"""
from __future__ import annotations

import json

from paper_2306_14011_gb300 import inputs as I

from . import oracle as O


def per_cell_stage(g, U) -> dict:
    dt = O.time_step(g, U)
    c = O.count_ops(g, U, dt)
    cells = g.ncells
    out = {}
    for k in ("residual", "time_step", "rk3_step"):
        out[k] = sum(int(x) for x in c[k]) / cells
    out["per_cell_stage"] = (out["rk3_step"] + out["time_step"]) / 3.0
    out["breakdown_rk3_step"] = dict(zip(("add", "mul", "div", "sqrt"), (int(x) for x in c["rk3_step"])))
    return out


def extrapolate(make, n_small, n_large, n_target) -> float:
    """Per-cell-stage count at size n_target from two small sizes: the oracle
    evaluates n+1 faces per line, so the count is a + b/n in the line length."""
    a1 = per_cell_stage(*make(n_small))["per_cell_stage"]
    a2 = per_cell_stage(*make(n_large))["per_cell_stage"]
    b = (a1 - a2) / (1.0 / n_small - 1.0 / n_large)
    a = a2 - b / n_large
    return a + b / n_target


def main():
    res = {
        "2d_kelvin_helmholtz_128": per_cell_stage(*I.kelvin_helmholtz(128, seed=1)),
        "3d_taylor_green_32": per_cell_stage(*I.taylor_green(32, seed=2)),
        "2d_kelvin_helmholtz_4096_per_cell_stage": extrapolate(lambda n: I.kelvin_helmholtz(n, seed=1), 64, 128, 4096),
        "3d_taylor_green_384_per_cell_stage": extrapolate(lambda n: I.taylor_green(n, seed=2), 16, 32, 384),
    }
    print(json.dumps(res, indent=1))


if __name__ == "__main__":
    main()
