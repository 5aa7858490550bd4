"""Launch sweeps: time the SSP-RK3 step of a workload under explicit launch
configurations (the manual counterpart of the autotuner).

    python -m paper_2306_14011_gb300.sweep --workload kh --n 4096 \
        --config 32x32:160 --config 32x16:128 ...
    python -m paper_2306_14011_gb300.sweep --workload tgv --n 384 \
        --config 8x8x8:192 --config 16x15x32:256:march

Each --config is TILE:THREADS[:march] (TILE = XxY or XxYxZ; with `march` the
3D z-marching kernel, Z = planes per chunk).  Per configuration: a context
with that tile and thread count for all three stages, 3 untimed steps, then
the best of 3 timed runs of --steps steps (CUDA events on the solver's
stream).  Prints one JSON line per configuration: ms per step and
cell-stage/s, or the library's error for a configuration it rejects.
"""
from __future__ import annotations

import argparse
import json
import sys


def parse_config(text: str, dim: int):
    """'32x32:160' -> ((32, 32, 1), 160, 0); '16x15x32:256:march' -> (..., 1)."""
    parts = text.split(":")
    if len(parts) not in (2, 3) or (len(parts) == 3 and parts[2] != "march"):
        raise ValueError(f"bad config {text!r}: expected TILE:THREADS[:march]")
    tile = tuple(int(x) for x in parts[0].lower().split("x"))
    if len(tile) != dim:
        raise ValueError(f"bad config {text!r}: a {dim}D tile has {dim} extents")
    if dim == 2:
        tile = tile + (1,)
    march = 1 if len(parts) == 3 else 0
    if march and dim != 3:
        raise ValueError(f"bad config {text!r}: the marching kernel is 3D only")
    return tile, int(parts[1]), march


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", choices=("kh", "tgv"), default="kh",
                    help="kh: 2D Kelvin-Helmholtz (seed 1); tgv: 3D Taylor-Green (seed 2)")
    ap.add_argument("--n", type=int, default=None, help="cells per side (default 4096 for kh, 384 for tgv)")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--config", action="append", required=True)
    args = ap.parse_args(argv)
    dim = 2 if args.workload == "kh" else 3
    configs = [parse_config(c, dim) for c in args.config]

    import torch

    from . import fv
    from . import inputs as I

    n = args.n or (4096 if dim == 2 else 384)
    g, U0 = I.kelvin_helmholtz(n, seed=1) if dim == 2 else I.taylor_green(n, seed=2)
    Ud0 = torch.from_numpy(U0).cuda()
    st = torch.cuda.current_stream()
    for tile, thr, march in configs:
        d = fv.launch_to_dict(fv.fv_default_launch(g))
        for s in range(3):
            d["stage"][s].update(tile=tile, threads=thr, march=march)
        rec = dict(tile=list(tile), threads=thr, march=march)
        try:
            S = fv.Solver(g, launch=d, stream=st)
        except fv.FvError as e:
            print(json.dumps(dict(rec, error=str(e))), flush=True)
            continue
        U = Ud0.clone()
        S.run(U, 3)
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            S.run(U, args.steps)
            e1.record(st)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        S.sync()
        S.close()
        print(json.dumps(dict(rec, ms_per_step=best / args.steps,
                              rate=g.ncells * 3 * args.steps / (best / 1e3))), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
