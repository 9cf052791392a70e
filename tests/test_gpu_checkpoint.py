"""Checkpointed recomputation of the source wavefield (memory-lean mode):
keeping the state every C steps and recomputing each segment's snapshots
must give the same image, bit for bit, as keeping every snapshot, in every
snapshot format and for any segment length; and it must need less memory."""
import os

import numpy as np
import pytest

from paper_2001_06444_gb300 import inputs, rtm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problem(nt):
    nx, nz = 210, 80
    v = inputs.layered_faulted(nz, nx, 10.0, 10.0, seed=71, water_depth=90.0).astype(np.float32)
    s = inputs.Survey(nx, nz, 20, 10.0, 10.0, 1e-3, nt, v, np.array([15, 105, 190], np.int32),
                      np.array([1, 2, 1], np.int32), np.arange(nx, dtype=np.int32),
                      np.full(nx, 1, np.int32), inputs.ricker(16.0, 1e-3, nt))
    seis = (inputs.normal(9, 3 * nt * nx).reshape(3, nt, nx) * 1e-3).astype(np.float32)
    return s, v, seis


def _migrate(ctx, s, v, seis, opts):
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    img = torch.zeros((s.nz, s.nx), dtype=torch.float32, device="cuda")
    ctx.migrate(rtm.make_grid(*s.grid_tuple()), torch.from_numpy(v).cuda(), acq,
                torch.from_numpy(seis).cuda(), opts, img)
    torch.cuda.synchronize()
    return img.cpu().numpy()


@pytest.mark.parametrize("nt,isnap", [(400, 4), (331, 3)])
@pytest.mark.parametrize("dtype", [rtm.SNAP_F32, rtm.SNAP_F16, rtm.SNAP_BF16])
def test_checkpoint_mode_is_bitwise_identical(nt, isnap, dtype):
    s, v, seis = _problem(nt)
    with rtm.Context(0) as ctx:
        full = _migrate(ctx, s, v, seis, rtm.Opts(isnap, dtype, 1e-6, 1, 0))
        for cp in (8, 10, 26, -1):
            got = _migrate(ctx, s, v, seis, rtm.Opts(isnap, dtype, 1e-6, 1, cp))
            assert np.array_equal(got, full), (cp, isnap, dtype)


def test_checkpoint_mode_single_step_kernel_and_memory():
    s, v, seis = _problem(300)
    old = os.environ.get("RTM_STEP_KERNEL")
    os.environ["RTM_STEP_KERNEL"] = "1"
    try:
        one = rtm.Context(0)
    finally:
        if old is None:
            del os.environ["RTM_STEP_KERNEL"]
        else:
            os.environ["RTM_STEP_KERNEL"] = old
    try:
        with rtm.Context(0) as ctx:
            full = _migrate(ctx, s, v, seis, rtm.Opts(4, rtm.SNAP_F32, 1e-6, 1, 0))
        assert np.array_equal(_migrate(one, s, v, seis, rtm.Opts(4, rtm.SNAP_F32, 1e-6, 1, 12)), full)
    finally:
        one.close()
    # the full-size shot: 3.0 GB of FP32 snapshots against checkpoints + a ring
    big = inputs.full_size(nshot=1)
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, big.src_ix, big.src_iz, big.rec_ix, big.rec_iz, big.wavelet)
    g = rtm.make_grid(*big.grid_tuple())
    _, item_full = rtm.plan_bytes(g, acq, rtm.Opts(4, rtm.SNAP_F32, 1e-6, 1, 0))
    _, item_cp = rtm.plan_bytes(g, acq, rtm.Opts(4, rtm.SNAP_F32, 1e-6, 1, -1))
    assert item_cp < item_full / 5, (item_cp, item_full)


@pytest.mark.parametrize("cp", [0, 26])
def test_host_seismograms_uploaded_behind_the_forward_phase(cp):
    """Host seismograms are uploaded on a side stream behind the first
    forward phase; the image must equal the device-buffer image bit for bit,
    for pinned and pageable host memory, one shot per batch (the upload is
    issued once, in the first batch) and in checkpoint mode."""
    s, v, seis = _problem(400)
    opts = rtm.Opts(4, rtm.SNAP_F32, 1e-6, 1, cp)
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    grid = rtm.make_grid(*s.grid_tuple())
    with rtm.Context(0) as ctx:
        for batch in (0, 1):
            ctx.set_batch(batch)
            want = _migrate(ctx, s, v, seis, opts)
            for host in (torch.from_numpy(seis).pin_memory(), seis):
                img = np.zeros((s.nz, s.nx), np.float32)
                ctx.migrate(grid, v, acq, host, opts, img)
                assert np.array_equal(img, want), (batch, cp, type(host))


def test_host_seismograms_with_batches_across_samples():
    """Two velocity samples x 3 shots in batches of 2: the middle batch holds
    the last shot of sample 0 and the first of sample 1, so it waits for the
    whole upload.  Host and device seismograms give the same images."""
    s, v, seis = _problem(400)
    vels = np.stack([v, (v * 1.02).astype(np.float32)])
    opts = rtm.Opts(4, rtm.SNAP_F32, 1e-6, 1, 0)
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    grid = rtm.make_grid(*s.grid_tuple())
    with rtm.Context(0) as ctx:
        ctx.set_batch(2)
        want = torch.zeros((2, s.nz, s.nx), dtype=torch.float32, device="cuda")
        ctx.migrate_ensemble(grid, torch.from_numpy(vels).cuda(), acq,
                             torch.from_numpy(seis).cuda(), opts, want)
        torch.cuda.synchronize()
        got = np.zeros((2, s.nz, s.nx), np.float32)
        ctx.migrate_ensemble(grid, vels, acq, torch.from_numpy(seis).pin_memory(), opts, got)
        assert np.array_equal(got, want.cpu().numpy())
