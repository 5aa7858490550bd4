"""The allocation-free residual entry point, fv_residual_noalloc.

Some callers cannot allocate device memory when they call into the library
(services with a fixed device-memory budget, plug-ins inside an application
that owns the device's memory, hosts that cannot take cudaFree's device-wide
synchronisation); for them the residual and its norms are available without a
context, using a fixed scratch array inside the library.  These tests check it against fv_residual (through a context) on
consecutive calls that share that scratch.  This file is collected last, so a
run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2306_14011_gb300 import fv  # noqa: E402
from paper_2306_14011_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the residual parity bar of the GPU tests


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    out = 0.0
    for v in range(b.shape[0]):
        den = np.abs(b[v]).max()
        num = np.abs(a[v] - b[v]).max()
        out = max(out, num / den if den > 0 else (np.inf if num > 0 else 0.0))
    return out


def test_noalloc_residual_matches_context_residual_on_consecutive_calls():
    cases = [I.kelvin_helmholtz(256, seed=1), I.taylor_green(24, seed=2), I.isentropic_vortex(128, seed=5)]
    sch = fv.make_scheme()
    for g, U in cases:  # consecutive calls share (and overwrite) the fixed scratch
        Ud = torch.from_numpy(U).cuda()
        with fv.Solver(g) as s:
            R_ref, n_ref = s.residual(Ud, norms=True)
            R_ref, n_ref = R_ref.cpu().numpy(), n_ref.cpu().numpy()
        R = torch.empty_like(Ud)
        nrm = torch.full((g.nvar,), -1.0, dtype=torch.float64, device="cuda")
        fv.fv_residual_noalloc(g, sch, Ud, R, nrm)
        torch.cuda.synchronize()
        assert _rel(R.cpu().numpy(), R_ref) <= TOL
        assert np.max(np.abs(nrm.cpu().numpy() - n_ref) / n_ref) <= TOL
        # without norms: same residual
        R2 = torch.empty_like(Ud)
        fv.fv_residual_noalloc(g, sch, Ud, R2)
        torch.cuda.synchronize()
        assert torch.equal(R2, R)


def test_noalloc_residual_allocates_nothing_after_first_use():
    g, U = I.kelvin_helmholtz(512, seed=1)
    Ud = torch.from_numpy(U).cuda()
    R = torch.empty_like(Ud)
    nrm = torch.zeros(g.nvar, dtype=torch.float64, device="cuda")
    sch = fv.make_scheme()
    fv.fv_residual_noalloc(g, sch, Ud, R, nrm)  # first call on this device: set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        fv.fv_residual_noalloc(g, sch, Ud, R, nrm)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_residual_rejects_oversized_grids_and_host_pointers():
    sch = fv.make_scheme()
    g = I.grid2d(5792, 5824, 1.0, 1.0)  # 91 x 364 = 33124 default tiles of 64x16: above the 32768 of the scratch
    U = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    R = torch.empty_like(U)
    nrm = torch.zeros(g.nvar, dtype=torch.float64, device="cuda")
    with pytest.raises(fv.FvError) as e:
        fv.fv_residual_noalloc(g, sch, U, R, nrm)
    assert e.value.status == fv.FV_EINVAL
    gs, Us = I.isentropic_vortex(32)
    with pytest.raises(fv.FvError) as e:
        fv.fv_residual_noalloc(gs, sch, Us, np.empty_like(Us))
    assert e.value.status == fv.FV_EINVAL
