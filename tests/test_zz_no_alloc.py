"""Modelling without device allocation (rtm_model_noalloc), called through the
C ABI.  It serves callers that cannot allocate device memory while they run:
a host framework whose caching allocator already owns the device's memory, or
a real-time loop where an allocation could stall the device.  It works in a
fixed scratch array that the library holds on the device.

Checked here:
- two calls in a row, which share the scratch, each equal the allocating
  entry point rtm_model bit for bit (both run the same per-point arithmetic);
- a call after the first one changes neither the device's free memory nor
  the torch allocator's counters;
- the documented refusals: a grid larger than the scratch (RTM_ERR_NOMEM,
  output untouched), a velocity above the stability bound (RTM_ERR_CFL), a
  host velocity pointer and a shot outside the acquisition (RTM_ERR_ARG);
  a good call after them is still exact.

This file is collected last, so a run that stops at the first failure has
run every other test first."""
import ctypes

import numpy as np
import pytest

from paper_2001_06444_gb300 import inputs, rtm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problem():
    nx, nz, nt = 230, 96, 700
    v = inputs.layered_faulted(nz, nx, 10.0, 10.0, seed=41, water_depth=90.0).astype(np.float32)
    s = inputs.Survey(nx, nz, 20, 10.0, 10.0, 1e-3, nt, v, np.array([40, 181], np.int32),
                      np.array([2, 1], np.int32), np.arange(nx, dtype=np.int32),
                      np.full(nx, 3, np.int32), inputs.ricker(15.0, 1e-3, nt))
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    return s, v, keep, acq, rtm.make_grid(*s.grid_tuple())


def _call(grid, vel_ptr, acq, shot, out):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return rtm.lib().rtm_model_noalloc(ctypes.byref(grid), ctypes.c_void_p(vel_ptr),
                                       ctypes.byref(acq), shot,
                                       ctypes.c_void_p(out.data_ptr()), stream)


def test_noalloc_modelling_matches_rtm_model_on_two_calls():
    torch.cuda.set_device(0)
    s, v, keep, acq, grid = _problem()
    vel = torch.from_numpy(v).cuda()
    with rtm.Context(0) as ctx:
        for shot in (0, 1):  # two calls in a row share the scratch
            got = torch.full((s.nt, s.nrec), float("nan"), dtype=torch.float32, device="cuda")
            assert _call(grid, vel.data_ptr(), acq, shot, got) == rtm.RTM_OK
            want = torch.zeros_like(got)
            ctx.model(grid, vel, acq, shot, want)
            torch.cuda.synchronize()
            assert torch.equal(got, want), shot


def test_noalloc_call_allocates_no_device_memory():
    torch.cuda.set_device(0)
    s, v, keep, acq, grid = _problem()
    vel = torch.from_numpy(v).cuda()
    out = torch.zeros((s.nt, s.nrec), dtype=torch.float32, device="cuda")
    assert _call(grid, vel.data_ptr(), acq, 0, out) == rtm.RTM_OK  # first call: set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    alloc0 = torch.cuda.memory_allocated()
    reserved0 = torch.cuda.memory_reserved()
    for shot in (1, 0):
        assert _call(grid, vel.data_ptr(), acq, shot, out) == rtm.RTM_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.memory_reserved() == reserved0


def test_noalloc_refusals_then_exact_again():
    torch.cuda.set_device(0)
    s, v, keep, acq, grid = _problem()
    vel = torch.from_numpy(v).cuda()
    # a grid whose four padded planes (c and three fields) exceed the 32 MiB
    # scratch: 1701 x 1201 with a 20-cell sponge is 1241 x 1760 floats a plane
    big = inputs.Survey(1701, 1201, 20, 10.0, 10.0, 1e-3, 10, None, np.array([800], np.int32),
                        np.array([1], np.int32), np.array([5], np.int32),
                        np.array([1], np.int32), inputs.ricker(15.0, 1e-3, 10))
    bkeep = rtm._Keep()
    bacq = rtm.make_acq(bkeep, big.src_ix, big.src_iz, big.rec_ix, big.rec_iz,
                        big.wavelet.astype(np.float32))
    bvel = torch.full((1201, 1701), 2000.0, dtype=torch.float32, device="cuda")
    bout = torch.full((10, 1), float("nan"), dtype=torch.float32, device="cuda")
    assert _call(rtm.make_grid(*big.grid_tuple()), bvel.data_ptr(), bacq, 0, bout) == \
        rtm.RTM_ERR_NOMEM
    torch.cuda.synchronize()
    assert torch.isnan(bout).all()  # untouched
    out = torch.full((s.nt, s.nrec), float("nan"), dtype=torch.float32, device="cuda")
    fast = torch.full_like(vel, 1.05 * rtm.cfl_limit() * 10.0 / 1e-3)
    assert _call(grid, fast.data_ptr(), acq, 0, out) == rtm.RTM_ERR_CFL
    host_v = np.ascontiguousarray(v)
    assert _call(grid, host_v.ctypes.data, acq, 0, out) == rtm.RTM_ERR_ARG
    assert _call(grid, vel.data_ptr(), acq, 2, out) == rtm.RTM_ERR_ARG
    assert _call(grid, vel.data_ptr(), acq, -1, out) == rtm.RTM_ERR_ARG
    torch.cuda.synchronize()
    assert torch.isnan(out).all()  # no refused call wrote the output
    assert _call(grid, vel.data_ptr(), acq, 1, out) == rtm.RTM_OK
    want = torch.zeros_like(out)
    with rtm.Context(0) as ctx:
        ctx.model(grid, vel, acq, 1, want)
    torch.cuda.synchronize()
    assert torch.equal(out, want)
