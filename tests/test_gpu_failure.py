"""Failure detection on the device without a GPU fault: a bounded wait that
runs out raises a flag the host reads, and the context keeps working."""
import time

import numpy as np
import pytest

from paper_2001_06444_gb300 import inputs, rtm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_context_survives():
    with rtm.Context(0) as ctx:
        t = time.perf_counter()
        assert ctx.selftest_wait(200) is True
        dt = time.perf_counter() - t
        assert 0.15 < dt < 5.0, dt
        # the context is still usable: a small modelling call succeeds
        nx, nz, nt = 60, 40, 50
        v = np.full((nz, nx), 2000.0, np.float32)
        keep = rtm._Keep()
        acq = rtm.make_acq(keep, [30], [5], np.arange(nx), np.full(nx, 5), inputs.ricker(20.0, 1e-3, nt))
        out = torch.zeros((nt, nx), dtype=torch.float32, device="cuda")
        ctx.model(rtm.make_grid(nx, nz, 10, 10.0, 10.0, 1e-3, nt), torch.from_numpy(v).cuda(), acq, 0, out)
        torch.cuda.synchronize()
        assert torch.isfinite(out).all() and out.abs().max() > 0
