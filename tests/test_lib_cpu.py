"""CPU-only checks of the C-ABI library: it builds for sm_103a, loads, and
exports every entry point include/fv.h declares; host-side validation works
without a GPU.  No kernel is launched here."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2306_14011_gb300 import fv
from paper_2306_14011_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(fv_\w+)\s*\(", txt, re.M))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = fv.load()
    names = _declared()
    assert "fv_run" in names and "fv_init" in names and len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", fv.library_path()], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}\b", out), n


def test_library_targets_sm_103a_only():
    out = subprocess.run(["cuobjdump", "--list-elf", fv.library_path()], capture_output=True, text=True).stdout
    arches = set(re.findall(r"sm_\d+a?", out))
    assert arches == {"sm_103a"}, arches


def test_strerror_and_default_launch_without_gpu():
    assert fv.strerror(fv.FV_EINVAL) == "invalid argument"
    assert fv.strerror(99) == "unknown status"
    l2 = fv.fv_default_launch(I.grid2d(64, 64, 1.0, 1.0))
    assert tuple(l2.stage[0].tile) == (64, 16, 1) and l2.stage[0].threads == 192
    assert l2.dt.threads == 512 and l2.dt.grid == 0
    l3 = fv.fv_default_launch(I.grid3d(16, 16, 16, 1.0, 1.0, 1.0))
    assert tuple(l3.stage[2].tile) == (8, 8, 8) and l3.stage[2].threads == 192 and l3.stage[2].march == 0
    # fused by default; the split kernels default to 128 threads, one item per thread
    for l in (l2, l3):
        assert l.mode == fv.FV_FUSED
        assert all(l.split[k].threads == 128 and l.split[k].grid == 0 for k in range(fv.FV_SK_COUNT))
    d = fv.launch_to_dict(l2)
    assert fv.launch_to_dict(fv.launch_from_dict(d)) == d


def test_invalid_grids_are_rejected_on_the_host():
    bad = [
        I.GridSpec(4, (8, 8, 1), (1.0, 1.0, 1.0)),          # dim
        I.GridSpec(2, (0, 8, 1), (1.0, 1.0, 1.0)),          # empty axis
        I.GridSpec(2, (8, 8, 1), (1.0, -1.0, 1.0)),         # length
        I.GridSpec(2, (8, 8, 1), (1.0, 1.0, 1.0), ((0, 1), (0, 0), (0, 0))),  # half-periodic axis
    ]
    for g in bad:
        with pytest.raises(fv.FvError) as e:
            fv.fv_default_launch(g)
        assert e.value.status == fv.FV_EINVAL
    lib = fv.load()
    G = fv.make_grid(I.grid2d(8, 8, 1.0, 1.0))
    G.n[2] = 2  # nz != 1 in 2D
    assert lib.fv_default_launch(C.byref(G), C.byref(fv.fv_launch())) == fv.FV_EINVAL
    # null context pointers are rejected before any CUDA call
    assert lib.fv_sync(None) == fv.FV_EINVAL
    assert lib.fv_residual(None, None, None, None) == fv.FV_EINVAL
    assert lib.fv_run(None, None, 1, 0.0, None) == fv.FV_EINVAL


def test_init_without_a_gpu_reports_an_error_not_a_crash():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = fv.load()
    ctx = C.c_void_p()
    G = fv.make_grid(I.grid2d(8, 8, 1.0, 1.0))
    S = fv.make_scheme()
    st = lib.fv_init(C.byref(ctx), C.byref(G), 1, C.byref(S), None, None)
    assert st in (fv.FV_ECUDA, fv.FV_ENOMEM)
    assert not ctx.value


def test_tuning_space_sizes():
    """The split kernels' space is the paper's (Sec. 3.4, Table
    "tuning-parameters": 7 kernels, each with 10 gang and 12 vector-length
    values; the paper states 14 parameters and 3.58e14 points); 3D adds a
    limiter and a flux kernel.  The fused space counts its own value sets."""
    n, size = fv.fv_tune_space(2, fv.FV_SPLIT)
    assert n == 14 and size == float(10 ** 7 * 12 ** 7) and f"{size:.2e}" == "3.58e+14"
    assert fv.fv_tune_space(3, fv.FV_SPLIT) == (18, float(10 ** 9 * 12 ** 9))
    assert fv.fv_tune_space(2) == (14, float((5 * 5 * 7 * 2) ** 3 * 4 * 4))
    assert fv.fv_tune_space(3, fv.FV_FUSED) == (20, float((3 * 3 * 3 * 7 * 2 * 2) ** 3 * 4 * 4))
    for dim, mode in [(4, fv.FV_FUSED), (2, 2), (3, -1)]:
        with pytest.raises(fv.FvError):
            fv.fv_tune_space(dim, mode)


def test_fp64_rate_rejects_bad_arguments_on_the_host():
    lib = fv.load()
    assert lib.fv_debug_fp64_rate(4, C.byref(C.c_double()), None) == fv.FV_EINVAL
    assert lib.fv_debug_fp64_rate(-1, C.byref(C.c_double()), None) == fv.FV_EINVAL
    assert lib.fv_debug_fp64_rate(0, None, None) == fv.FV_EINVAL


def test_debug_wait_rejects_bad_arguments_on_the_host():
    for kind, limit in [(2, 0.1), (-1, 0.1), (0, 0.0), (1, -1.0), (0, 11.0), (1, float("nan"))]:
        with pytest.raises(fv.FvError) as e:
            fv.fv_debug_wait(kind, limit, stream=0)
        assert e.value.status == fv.FV_EINVAL
