"""Failure detection without a GPU fault: the library's bounded device waits
give up, report FV_ETIMEOUT and leave the device usable.

fv_debug_wait runs the same wait code as the tile loads (an mbarrier that no
copy completes) and the batched kernel's grid barrier (a word that nothing
changes) with a short limit; nothing traps, faults or hangs.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2306_14011_gb300 import fv  # noqa: E402
from paper_2306_14011_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", [0, 1])
def test_bounded_wait_times_out_and_device_stays_usable(kind):
    g, U = I.isentropic_vortex(64, seed=0)
    Ud = torch.from_numpy(U).cuda()
    with fv.Solver(g) as s:
        before = s.residual(Ud).clone()
        t0 = time.perf_counter()
        with pytest.raises(fv.FvError) as e:
            fv.fv_debug_wait(kind, 0.25)
        elapsed = time.perf_counter() - t0
        assert e.value.status == fv.FV_ETIMEOUT
        assert 0.2 <= elapsed < 5.0
        # the context and the device still work and give the same results
        assert torch.equal(s.residual(Ud), before)
        X = Ud.clone()
        s.run(X, 3)
        assert torch.isfinite(X).all()
