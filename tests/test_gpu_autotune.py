"""The launch-configuration autotuner and graph-captured batches: every
candidate configuration (propagation kernel and tile height, items in
flight, CUDA graph capture) must give bit-identical images, so tuning never
changes a result."""
import os

import numpy as np
import pytest

from paper_2001_06444_gb300 import inputs, rtm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problem():
    nx, nz, nt = 190, 72, 330
    v = inputs.layered_faulted(nz, nx, 10.0, 10.0, seed=61, water_depth=80.0).astype(np.float32)
    s = inputs.Survey(nx, nz, 20, 10.0, 10.0, 1e-3, nt, v, np.array([20, 95, 170], np.int32),
                      np.full(3, 1, np.int32), np.arange(nx, dtype=np.int32),
                      np.full(nx, 1, np.int32), inputs.ricker(18.0, 1e-3, nt))
    seis = (inputs.normal(5, 3 * nt * nx).reshape(3, nt, nx) * 1e-3).astype(np.float32)
    return s, v, seis


def _migrate(ctx, s, v, seis, opts, stream=None):
    """Migrate on `stream` (None: the legacy default stream, where the
    library launches directly; a created stream lets it capture graphs)."""
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    with torch.cuda.stream(stream or torch.cuda.default_stream()):
        img = torch.zeros((s.nz, s.nx), dtype=torch.float32, device="cuda")
        ctx.migrate(rtm.make_grid(*s.grid_tuple()), torch.from_numpy(v).cuda(), acq,
                    torch.from_numpy(seis).cuda(), opts, img)
    torch.cuda.synchronize()
    return img.cpu().numpy()


@pytest.mark.parametrize("dtype", [rtm.SNAP_F32, rtm.SNAP_F16])
def test_autotune_and_graph_capture_are_bitwise_neutral(dtype):
    s, v, seis = _problem()
    opts = rtm.Opts(4, dtype, 1e-6, 1)
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    side = torch.cuda.Stream()
    with rtm.Context(0) as ctx:
        base = _migrate(ctx, s, v, seis, opts)
        choice = ctx.autotune(rtm.make_grid(*s.grid_tuple()), acq, opts, trial_steps=40)
        assert choice["step_kernel"] in (1, 2, 3, 4) and choice["graph"] in (0, 1)
        assert choice["tile_z"] in (16, 24, 32)
        assert choice["tile_z"] == 24 or (choice["step_kernel"], choice["tile_z"]) in ((3, 16),
                                                                                      (4, 32))
        assert choice["l2_ahead"] in (0, 1)
        assert choice["max_items"] >= 0
        assert np.array_equal(_migrate(ctx, s, v, seis, opts), base)
        assert np.array_equal(_migrate(ctx, s, v, seis, opts, side), base)
    old = os.environ.get("RTM_GRAPHS")
    os.environ["RTM_GRAPHS"] = "1"
    try:
        g = rtm.Context(0)
    finally:
        if old is None:
            del os.environ["RTM_GRAPHS"]
        else:
            os.environ["RTM_GRAPHS"] = old
    try:
        g.set_batch(2)  # two batches, each phase captured and replayed as a graph
        g.set_profiling(True)
        g.stats(reset=True)
        assert np.array_equal(_migrate(g, s, v, seis, opts, side), base)
        st = g.stats(reset=True)
        assert st["graph_launches"] >= 4, st  # 2 batches x (forward, backward)
    finally:
        g.close()
