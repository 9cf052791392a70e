"""Modelling without device allocation (rtm_model_noalloc), called through the
C ABI.  It is meant for callers that cannot allocate device memory while they
run; it works in a fixed scratch array the library holds on the device.  Two
calls in a row must each match the allocating entry point (rtm_model) within
the seismogram tolerance of the parity tests.  This file is collected last,
so a run that stops at the first failure has run every other test first."""
import ctypes

import numpy as np
import pytest

from conftest import rel_l2
from paper_2001_06444_gb300 import inputs, rtm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEIS_TOL = 1e-4


def test_noalloc_modelling_matches_rtm_model_on_two_calls():
    torch.cuda.set_device(0)
    nx, nz, nt = 230, 96, 700
    v = inputs.layered_faulted(nz, nx, 10.0, 10.0, seed=41, water_depth=90.0).astype(np.float32)
    s = inputs.Survey(nx, nz, 20, 10.0, 10.0, 1e-3, nt, v, np.array([40, 181], np.int32),
                      np.array([2, 1], np.int32), np.arange(nx, dtype=np.int32),
                      np.full(nx, 3, np.int32), inputs.ricker(15.0, 1e-3, nt))
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    grid = rtm.make_grid(*s.grid_tuple())
    vel = torch.from_numpy(v).cuda()
    fn = rtm.lib().rtm_model_noalloc
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    with rtm.Context(0) as ctx:
        for shot in (0, 1):  # two calls in a row share the scratch
            got = torch.full((nt, s.nrec), float("nan"), dtype=torch.float32, device="cuda")
            rc = fn(ctypes.byref(grid), ctypes.c_void_p(vel.data_ptr()), ctypes.byref(acq), shot,
                    ctypes.c_void_p(got.data_ptr()), stream)
            assert rc == rtm.RTM_OK
            want = torch.zeros_like(got)
            ctx.model(grid, vel, acq, shot, want)
            torch.cuda.synchronize()
            assert rel_l2(got.cpu().numpy(), want.cpu().numpy()) <= SEIS_TOL
