"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances: seismograms 1e-4 relative L2, images 1e-3 with FP32 snapshots
and 1e-2 with half-precision snapshots; source and receiver indexing
bit-exact.  Inputs are generated once, rounded to float32, and given to both
sides; the oracle never sees anything the GPU computed.
"""
import numpy as np
import pytest

import oracle
from conftest import rel_l2
from paper_2001_06444_gb300 import inputs
from paper_2001_06444_gb300 import rtm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SEIS_TOL, IMG_TOL, HALF_IMG_TOL = 1e-4, 1e-3, 1e-2


@pytest.fixture(scope="module")
def ctx():
    c = rtm.Context(0)
    yield c
    c.close()


def f32(a):
    return np.ascontiguousarray(np.asarray(a, np.float32))


def dev(a):
    return torch.from_numpy(f32(a)).cuda()


def gpu_model(ctx, s, vel, shot=0, rec=None):
    rec_ix, rec_iz = (s.rec_ix, s.rec_iz) if rec is None else rec
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, rec_ix, rec_iz, f32(s.wavelet))
    out = torch.zeros((s.nt, np.size(rec_ix)), dtype=torch.float32, device="cuda")
    ctx.model(rtm.make_grid(*s.grid_tuple()), dev(vel), acq, shot, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def ora_model(s, vel, shot=0, rec=None):
    rec_ix, rec_iz = (s.rec_ix, s.rec_iz) if rec is None else rec
    return oracle.model(oracle.grid(*s.grid_tuple()), f32(vel).astype(np.float64),
                        s.src_ix[shot], s.src_iz[shot], rec_ix, rec_iz,
                        f32(s.wavelet).astype(np.float64))


def _graph_context():
    """A context that captures each phase of a batch as a CUDA graph (on any
    stream but the legacy default one)."""
    import os

    old = os.environ.get("RTM_GRAPHS")
    os.environ["RTM_GRAPHS"] = "1"
    try:
        return rtm.Context(0)
    finally:
        if old is None:
            del os.environ["RTM_GRAPHS"]
        else:
            os.environ["RTM_GRAPHS"] = old


def gpu_migrate(ctx, s, vel, seis, isnap=1, dtype=rtm.SNAP_F32, lap=True, batch=0):
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, f32(s.wavelet))
    img = torch.zeros((s.nz, s.nx), dtype=torch.float32, device="cuda")
    ctx.set_batch(batch)
    ctx.migrate(rtm.make_grid(*s.grid_tuple()), dev(vel), acq, dev(seis),
                rtm.Opts(isnap, dtype, 1e-6, int(lap)), img)
    ctx.set_batch(0)
    torch.cuda.synchronize()
    return img.cpu().numpy()


def ora_migrate(s, vel, seis, isnap=1, mode=0, lap=True):
    return oracle.migrate(oracle.grid(*s.grid_tuple()), f32(vel).astype(np.float64), s.src_ix,
                          s.src_iz, s.rec_ix, s.rec_iz, f32(s.wavelet).astype(np.float64),
                          f32(seis).astype(np.float64), isnap=isnap, snap_mode=mode, laplacian=lap)


@pytest.fixture(scope="module")
def flat():
    """Flat-reflector workload (201 x 101, 1000 steps) with oracle data."""
    s = inputs.flat_reflector()
    d_two = ora_model(s, s.vel)
    d_dir = ora_model(s, np.full_like(s.vel, 1500.0))
    return s, f32(d_two - d_dir)


def test_flat_reflector_seismogram(ctx, flat):
    s, _ = flat
    got = gpu_model(ctx, s, s.vel)
    want = ora_model(s, s.vel)
    assert rel_l2(got, want) <= SEIS_TOL


def test_flat_reflector_image(ctx, flat):
    s, data = flat
    got = gpu_migrate(ctx, s, s.vel, data[None])
    want = ora_migrate(s, s.vel, data[None])
    assert rel_l2(got, want) <= IMG_TOL


def test_flat_reflector_depth_on_gpu(ctx, flat):
    from scipy.signal import hilbert

    s, data = flat
    img = gpu_migrate(ctx, s, np.full_like(s.vel, 1500.0), data[None])
    prof = img[:, 50:151].astype(np.float64).mean(axis=1)
    env = np.abs(hilbert(prof))
    pick = 10 + int(np.argmax(env[10:91]))
    assert abs(pick * s.dz - 495.0) <= 10.0


def test_source_and_receiver_indices_bit_exact(ctx):
    """After one update the field is non-zero at the source cell only; after
    two, exactly on the 8th-order cross around it."""
    nx, nz = 37, 29
    s = inputs.Survey(nx, nz, 7, 10.0, 10.0, 1e-3, 2, np.full((nz, nx), 2000.0),
                      np.array([11], np.int32), np.array([17], np.int32),
                      np.repeat(np.arange(nx), nz).astype(np.int32),
                      np.tile(np.arange(nz), nx).astype(np.int32),
                      np.array([1.0, 0.0]))
    d = gpu_model(ctx, s, s.vel)
    first = d[0].reshape(nx, nz).T
    nzr = np.argwhere(first != 0)
    assert nzr.tolist() == [[17, 11]]
    second = d[1].reshape(nx, nz).T != 0
    cross = np.zeros((nz, nx), bool)
    cross[17, 11 - 4:11 + 5] = True
    cross[17 - 4:17 + 5, 11] = True
    assert np.array_equal(second, cross)


@pytest.mark.parametrize("nx,nz,nb,dx,dz", [(300, 75, 20, 10.0, 10.0), (263, 141, 13, 8.0, 12.0),
                                             (130, 40, 3, 10.0, 10.0)])
def test_ragged_grids_model_and_migrate(ctx, nx, nz, nb, dx, dz):
    """Several tiles with ragged tails, sponge widths that are not multiples of
    4 (unaligned padded origin), rectangular cells, three shots."""
    nt = 400
    v = inputs.layered_faulted(nz, nx, dx, dz, seed=77, water_depth=60.0)
    s = inputs.Survey(nx, nz, nb, dx, dz, 1e-3, nt, v,
                      np.array([5, nx // 2, nx - 3], np.int32), np.array([1, 2, 0], np.int32),
                      np.arange(0, nx, 2, dtype=np.int32), np.full((nx + 1) // 2, 1, np.int32),
                      inputs.ricker(18.0, 1e-3, nt))
    for shot in range(3):
        assert rel_l2(gpu_model(ctx, s, v, shot), ora_model(s, v, shot)) <= SEIS_TOL
    vm = inputs.smooth(v, dx, dz, 40.0)
    data = np.stack([ora_model(s, v, k) for k in range(3)])
    assert rel_l2(gpu_migrate(ctx, s, vm, data, isnap=3), ora_migrate(s, vm, data, isnap=3)) <= IMG_TOL


def test_batch_size_does_not_change_the_image(ctx, flat):
    s0, _ = flat
    nt = 300
    s = inputs.Survey(s0.nx, s0.nz, 20, 10.0, 10.0, 1e-3, nt, s0.vel,
                      np.array([20, 60, 100, 140, 180], np.int32), np.full(5, 2, np.int32),
                      s0.rec_ix, s0.rec_iz, inputs.ricker(15.0, 1e-3, nt))
    data = np.stack([ora_model(s, s.vel, k) for k in range(5)])
    a = gpu_migrate(ctx, s, s.vel, data, isnap=2, batch=1)
    b = gpu_migrate(ctx, s, s.vel, data, isnap=2, batch=2)
    c = gpu_migrate(ctx, s, s.vel, data, isnap=2, batch=0)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    assert rel_l2(a, ora_migrate(s, s.vel, data, isnap=2)) <= IMG_TOL


# Image error of the snapshot format itself (oracle with the quantisation
# replayed vs exact snapshots, Laplacian-filtered flat-reflector image):
# BF16 6.1e-3 / 1.20e-2 / 1.69e-2 and FP16 7.6e-4 / 1.5e-3 / 2.1e-3 at
# isnap 1 / 4 / 8.  The filter amplifies the white quantisation noise ~14x,
# so BF16's 8-bit significand cannot meet 1e-2 against exact snapshots at
# isnap >= 4; FP16 with per-snapshot scaling can.
EXACT_TOL = {(rtm.SNAP_F16, 1): 1e-2, (rtm.SNAP_F16, 4): 1e-2, (rtm.SNAP_F16, 8): 1e-2,
             (rtm.SNAP_BF16, 1): 1e-2, (rtm.SNAP_BF16, 4): 1.5e-2, (rtm.SNAP_BF16, 8): 2e-2}


@pytest.mark.parametrize("mode", [rtm.SNAP_BF16, rtm.SNAP_F16])
@pytest.mark.parametrize("isnap", [1, 4, 8])
def test_half_precision_snapshots(ctx, flat, mode, isnap):
    s, data = flat
    got = gpu_migrate(ctx, s, s.vel, data[None], isnap=isnap, dtype=mode)
    want_q = ora_migrate(s, s.vel, data[None], isnap=isnap, mode=mode)
    want_x = ora_migrate(s, s.vel, data[None], isnap=isnap, mode=0)
    assert rel_l2(got, want_q) <= HALF_IMG_TOL
    assert rel_l2(got, want_x) <= EXACT_TOL[(mode, isnap)]


def test_reciprocity_fp32(ctx):
    nx, nz, nt = 160, 90, 500
    v = inputs.layered_faulted(nz, nx, 10.0, 10.0, seed=5, water_depth=100.0)
    a, b = (12, 3), (141, 70)
    w = inputs.ricker(15.0, 1e-3, nt)

    def trace(src, rec):
        s = inputs.Survey(nx, nz, 20, 10.0, 10.0, 1e-3, nt, v, np.array([src[0]], np.int32),
                          np.array([src[1]], np.int32), np.array([rec[0]], np.int32),
                          np.array([rec[1]], np.int32), w)
        return gpu_model(ctx, s, v)[:, 0]

    assert rel_l2(trace(a, b), trace(b, a)) < 1e-5


def test_ensemble_matches_single_migrations(ctx):
    nx, nz, nt = 180, 70, 350
    base = inputs.layered_faulted(nz, nx, 10.0, 10.0, seed=9, water_depth=100.0)
    ens = inputs.ensemble(base, 10.0, 10.0, 3, water_depth=100.0)
    s = inputs.Survey(nx, nz, 20, 10.0, 10.0, 1e-3, nt, base, np.array([30, 90, 150], np.int32),
                      np.full(3, 1, np.int32), np.arange(nx, dtype=np.int32),
                      np.full(nx, 1, np.int32), inputs.ricker(15.0, 1e-3, nt))
    data = np.stack([ora_model(s, base, k) for k in range(3)])
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, f32(s.wavelet))
    imgs = torch.zeros((3, nz, nx), dtype=torch.float32, device="cuda")
    ctx.migrate_ensemble(rtm.make_grid(*s.grid_tuple()), dev(ens), acq, dev(data),
                         rtm.Opts(2, rtm.SNAP_F32, 1e-6, 1), imgs)
    torch.cuda.synchronize()
    imgs = imgs.cpu().numpy()
    for k in range(3):
        single = gpu_migrate(ctx, s, ens[k], data, isnap=2)
        assert np.array_equal(imgs[k], single)
        assert rel_l2(imgs[k], ora_migrate(s, ens[k], data, isnap=2)) <= IMG_TOL


@pytest.mark.parametrize("n,npix", [(1, 1000), (2, 777), (5, 4099), (64, 12345), (97, 3001),
                                    (300, 517)])
def test_ensemble_stats(ctx, n, npix):
    x = f32(inputs.normal(100 + n, n * npix).reshape(n, npix) * 3.0 + 1.0)
    out = [torch.zeros(npix, dtype=t, device="cuda")
           for t in (torch.float64, torch.float64, torch.float32, torch.float32)]
    ctx.ensemble_stats(torch.from_numpy(x).cuda(), *out)
    torch.cuda.synchronize()
    mean, std, q05, q95 = [o.cpu().numpy() for o in out]
    m, sd, a, b = oracle.ensemble_stats(x)
    assert np.allclose(mean, m, rtol=1e-12, atol=1e-13)
    assert np.allclose(std, sd, rtol=1e-12, atol=1e-13)
    assert np.array_equal(q05, a.astype(np.float32))
    assert np.array_equal(q95, b.astype(np.float32))


def test_ensemble_stats_host_buffers(ctx):
    x = f32(inputs.normal(7, 16 * 999).reshape(16, 999))
    outs = [np.zeros(999, np.float64), np.zeros(999, np.float64), np.zeros(999, np.float32),
            np.zeros(999, np.float32)]
    ctx.ensemble_stats(x, *outs)
    m, sd, a, b = oracle.ensemble_stats(x)
    assert np.allclose(outs[0], m, rtol=1e-12) and np.allclose(outs[1], sd, rtol=1e-12)
    assert np.array_equal(outs[2], a.astype(np.float32))


def test_uncertainty_maps(ctx):
    mean = inputs.normal(1, 5000)
    mean[::7] = 0.0
    std = np.abs(inputs.normal(2, 5000))
    c = torch.zeros(5000, dtype=torch.float64, device="cuda")
    r = torch.zeros(5000, dtype=torch.float64, device="cuda")
    ctx.uncertainty_maps(torch.from_numpy(mean).cuda(), torch.from_numpy(std).cuda(), c, r)
    torch.cuda.synchronize()
    oc, orr = oracle.uncertainty_maps(mean, std)
    assert np.allclose(c.cpu().numpy(), oc, rtol=1e-14, atol=1e-15)
    assert np.allclose(r.cpu().numpy(), orr, rtol=1e-14, atol=0)


def test_errors_are_reported(ctx, flat):
    s, data = flat
    g = rtm.make_grid(*s.grid_tuple())
    keep = rtm._Keep()
    img = torch.zeros((s.nz, s.nx), dtype=torch.float32, device="cuda")
    bad = rtm.make_acq(keep, [s.nx], [2], s.rec_ix, s.rec_iz, f32(s.wavelet))
    with pytest.raises(rtm.RTMError) as e:
        ctx.migrate(g, dev(s.vel), bad, dev(data[None]), rtm.Opts(1, 0, 1e-6, 1), img)
    assert e.value.code == rtm.RTM_ERR_ARG
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, f32(s.wavelet))
    fast = np.full_like(s.vel, 1.01 * rtm.cfl_limit() * 10.0 / 1e-3)
    with pytest.raises(rtm.RTMError) as e:
        ctx.migrate(g, dev(fast), acq, dev(data[None]), rtm.Opts(1, 0, 1e-6, 1), img)
    assert e.value.code == rtm.RTM_ERR_CFL
    with pytest.raises(rtm.RTMError) as e:
        ctx.migrate(g, dev(s.vel), acq, dev(data[None]), rtm.Opts(0, 0, 1e-6, 1), img)
    assert e.value.code == rtm.RTM_ERR_ARG
    small = rtm.Context(0, budget_bytes=1 << 20)
    with pytest.raises(rtm.RTMError) as e:
        small.migrate(g, dev(s.vel), acq, dev(data[None]), rtm.Opts(1, 0, 1e-6, 1), img)
    assert e.value.code == rtm.RTM_ERR_NOMEM
    small.close()


def test_host_buffers_match_device_buffers(ctx, flat):
    s, data = flat
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, f32(s.wavelet))
    g = rtm.make_grid(*s.grid_tuple())
    host_img = np.zeros((s.nz, s.nx), np.float32)
    ctx.migrate(g, f32(s.vel), acq, f32(data[None]), rtm.Opts(2, 0, 1e-6, 1), host_img)
    assert np.array_equal(host_img, gpu_migrate(ctx, s, s.vel, data[None], isnap=2))


def test_legacy_stream_calls_are_ordered(flat):
    # with graphs on, a call given the legacy default stream runs on a
    # context-owned stream joined to it by events: it sees the work enqueued
    # on the legacy stream before it (the velocity, written after a busy
    # wait), and work enqueued after it sees the image
    s, data = flat
    g = _graph_context()
    try:
        keep = rtm._Keep()
        acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, f32(s.wavelet))
        grid = rtm.make_grid(*s.grid_tuple())
        opts = rtm.Opts(2, 0, 1e-6, 1)
        seis = dev(data[None])
        vel_ref = dev(s.vel)
        ref = torch.zeros((s.nz, s.nx), dtype=torch.float32, device="cuda")
        created = torch.cuda.Stream()
        with torch.cuda.stream(created):
            g.migrate(grid, vel_ref, acq, seis, opts, ref)
        created.synchronize()
        legacy = torch.cuda.default_stream()
        assert legacy.cuda_stream == 0
        with torch.cuda.stream(legacy):
            vel = torch.full_like(vel_ref, 1500.0)
            torch.cuda._sleep(50_000_000)  # a bounded busy wait on the legacy stream
            vel.copy_(vel_ref)
            img = torch.zeros_like(ref)
            g.migrate(grid, vel, acq, seis, opts, img)
            out = img * 1.0
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    finally:
        g.close()


def test_full_size_sampled_parity(ctx):
    """The 1701 x 351, 5000-step workload in the bench's launch configuration:
    one shot's seismogram on every 17th receiver and its migrated image
    (FP32 snapshots every 4 steps) against the oracle."""
    s = inputs.full_size(nshot=96)
    shot = 47
    sub = (s.rec_ix[::17], s.rec_iz[::17])
    got = gpu_model(ctx, s, s.vel, shot, rec=sub)
    want = ora_model(s, s.vel, shot, rec=sub)
    e_seis = rel_l2(got, want)
    assert e_seis <= SEIS_TOL
    one = inputs.Survey(s.nx, s.nz, s.nb, s.dx, s.dz, s.dt, s.nt, s.vel, s.src_ix[shot:shot + 1],
                        s.src_iz[shot:shot + 1], s.rec_ix, s.rec_iz, s.wavelet)
    data = f32(ora_model(one, s.vel))[None]
    vm = inputs.smooth(s.vel, s.dx, s.dz, 60.0)
    gi = gpu_migrate(ctx, one, vm, data, isnap=4)
    oi = ora_migrate(one, vm, data, isnap=4)
    e_img = rel_l2(gi, oi)
    print(f"full size: seismograms {e_seis:.2e}, image {e_img:.2e} (relative L2 vs the oracle)")
    assert e_img <= IMG_TOL
    # the bench's launch configuration: 48 shots in flight in one batch, each
    # phase captured as a CUDA graph on a created stream; only shot 47
    # carries data, so the stack is its image
    shots = np.arange(24, 72)
    many = inputs.Survey(s.nx, s.nz, s.nb, s.dx, s.dz, s.dt, s.nt, s.vel, s.src_ix[shots],
                         s.src_iz[shots], s.rec_ix, s.rec_iz, s.wavelet)
    d48 = np.zeros((len(shots), s.nt, s.nrec), np.float32)
    d48[int(np.flatnonzero(shots == shot)[0])] = data[0]
    g = _graph_context()
    try:
        g.set_profiling(True)
        with torch.cuda.stream(torch.cuda.Stream()):
            g48 = gpu_migrate(g, many, vm, d48, isnap=4)
        assert g.stats()["graph_launches"] >= 2  # the forward and backward phases
    finally:
        g.close()
    assert rel_l2(g48, oi) <= IMG_TOL


def _env_context(**env):
    """A context created with the given environment variables set (they pick
    the context's default propagation kernel and tile height)."""
    import os

    old = {k: os.environ.get(k) for k in env}
    os.environ.update({k: str(v) for k, v in env.items()})
    try:
        return rtm.Context(0)
    finally:
        for k, v in old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v


# the two-step kernels: one tile per block (with and without its L2 prefetch
# of later tiles); persistent with 24- and 16-row tiles; one tile per block
# with v^{n+1} over v^n, 24- and 32-row tiles; backward launches that image
# their input field (RTM_IMAGE_INPUT=1) with each kernel; and programmatic
# dependent launches (RTM_PDL=1)
TWO_STEP_KERNELS = [dict(RTM_STEP_KERNEL=2), dict(RTM_STEP_KERNEL=2, RTM_L2_AHEAD=1),
                    dict(RTM_STEP_KERNEL=3), dict(RTM_STEP_KERNEL=3, RTM_TILE_Z=16),
                    dict(RTM_STEP_KERNEL=4), dict(RTM_STEP_KERNEL=4, RTM_TILE_Z=32),
                    dict(RTM_STEP_KERNEL=2, RTM_IMAGE_INPUT=1),
                    dict(RTM_STEP_KERNEL=3, RTM_IMAGE_INPUT=1),
                    dict(RTM_STEP_KERNEL=4, RTM_TILE_Z=32, RTM_IMAGE_INPUT=1),
                    dict(RTM_STEP_KERNEL=4, RTM_TILE_Z=32, RTM_PDL=1)]


@pytest.mark.parametrize("nz", [90, 47])
def test_two_step_kernel_matches_single_step_bitwise(nz):
    """The two-step TMA kernels (one tile per block, with and without the L2
    prefetch; persistent with a copy ring, 24- and 16-row tiles; one tile per
    block with v^{n+1} over v^n, 24- and 32-row tiles) and the single-step
    kernel compute the same
    per-point arithmetic in the same order, so modelling and migration agree
    bit for bit (every snapshot format, even and odd isnap, odd nt, sponge
    widths that are not multiples of 4).  With nz = 47 the padded grid has
    73 rows, so the last row of 24-row tiles holds one row of the grid and
    most of its warps skip both substeps."""
    nx, nt = 250, 301
    v = inputs.layered_faulted(nz, nx, 10.0, 10.0, seed=21, water_depth=80.0)
    s = inputs.Survey(nx, nz, 13, 10.0, 10.0, 1e-3, nt, v, np.array([3, 120, 247], np.int32),
                      np.array([1, 0, 2], np.int32), np.arange(nx, dtype=np.int32),
                      np.full(nx, 1, np.int32), inputs.ricker(20.0, 1e-3, nt))
    data = np.stack([ora_model(s, v, k) for k in range(3)])
    vm = inputs.smooth(v, 10.0, 10.0, 30.0)
    one = _env_context(RTM_STEP_KERNEL=1)
    try:
        ref_model = [gpu_model(one, s, v, shot) for shot in range(3)]
        cases = ((4, rtm.SNAP_F32), (3, rtm.SNAP_F32), (1, rtm.SNAP_F32),
                 (4, rtm.SNAP_F16), (2, rtm.SNAP_BF16), (3, rtm.SNAP_F16))
        ref_img = [gpu_migrate(one, s, vm, data, isnap=i, dtype=m) for i, m in cases]
    finally:
        one.close()
    for env in TWO_STEP_KERNELS:
        two = _env_context(**env)
        try:
            for shot in range(3):
                assert np.array_equal(gpu_model(two, s, v, shot), ref_model[shot]), (env, shot)
            for (isnap, mode), want in zip(cases, ref_img):
                got = gpu_migrate(two, s, vm, data, isnap=isnap, dtype=mode)
                assert np.array_equal(got, want), (env, isnap, mode)
        finally:
            two.close()


def test_persistent_kernel_many_tiles_bitwise():
    """A batch with several times more tiles than the persistent kernel keeps
    resident (24 shots of a 640 x 187 grid: 1152 to 2160 tiles per launch),
    so every block walks several tiles through both stages of its copy ring,
    in both snake directions, and receivers lie in tiles at block boundaries.
    Modelling of all shots side by side and migration in every snapshot
    format must equal the one-tile-per-block kernel bit for bit."""
    nx, nz, nt = 640, 187, 160
    v = inputs.layered_faulted(nz, nx, 10.0, 10.0, seed=77, water_depth=60.0)
    ns = 24
    s = inputs.Survey(nx, nz, 20, 10.0, 10.0, 1e-3, nt, v,
                      np.linspace(5, nx - 6, ns).astype(np.int32), np.full(ns, 2, np.int32),
                      np.arange(0, nx, 2, dtype=np.int32), np.full(nx // 2, 3, np.int32),
                      inputs.ricker(18.0, 1e-3, nt))
    seis = (inputs.normal(9, ns * nt * s.nrec).reshape(ns, nt, s.nrec) * 1e-3).astype(np.float32)
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, f32(s.wavelet))

    def run(c):
        out = torch.zeros((ns, nt, s.nrec), dtype=torch.float32, device="cuda")
        c.model(rtm.make_grid(*s.grid_tuple()), dev(v), acq, -1, out)
        imgs = [gpu_migrate(c, s, v, seis, isnap=i, dtype=m)
                for i, m in ((4, rtm.SNAP_F32), (2, rtm.SNAP_F16), (4, rtm.SNAP_BF16))]
        torch.cuda.synchronize()
        return out.cpu().numpy(), imgs

    ref = None
    for env in TWO_STEP_KERNELS:
        c = _env_context(**env)
        try:
            got = run(c)
        finally:
            c.close()
        if ref is None:
            ref = got
            continue
        assert np.array_equal(got[0], ref[0]), env
        for a, b in zip(got[1], ref[1]):
            assert np.array_equal(a, b), env


def test_full_size_ensemble_sampled_parity(ctx):
    """The 64-sample ensemble at full size (1701 x 351, 5000 steps, GRF
    perturbations of the 60 m-smoothed model) through one migrate_ensemble
    call, one shot: samples 0 and 63 against the oracle's migration, and the
    per-pixel statistics of all 64 images against the oracle's statistics of
    the same images."""
    s = inputs.full_size(nshot=96)
    shot = 30
    one = inputs.Survey(s.nx, s.nz, s.nb, s.dx, s.dz, s.dt, s.nt, s.vel, s.src_ix[shot:shot + 1],
                        s.src_iz[shot:shot + 1], s.rec_ix, s.rec_iz, s.wavelet)
    data = f32(ora_model(one, s.vel))[None]
    vm = inputs.smooth(s.vel, s.dx, s.dz, 60.0)
    ens = f32(inputs.ensemble(vm, s.dx, s.dz, 64))
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, one.src_ix, one.src_iz, one.rec_ix, one.rec_iz, f32(one.wavelet))
    imgs = torch.zeros((64, s.nz, s.nx), dtype=torch.float32, device="cuda")
    ctx.migrate_ensemble(rtm.make_grid(*one.grid_tuple()), dev(ens), acq, dev(data),
                         rtm.Opts(4, rtm.SNAP_F32, 1e-6, 1), imgs)
    npix = s.nz * s.nx
    out = [torch.zeros(npix, dtype=t, device="cuda")
           for t in (torch.float64, torch.float64, torch.float32, torch.float32)]
    ctx.ensemble_stats(imgs, *out)
    torch.cuda.synchronize()
    got = imgs.cpu().numpy()
    for k in (0, 63):
        assert rel_l2(got[k], ora_migrate(one, ens[k], data, isnap=4)) <= IMG_TOL, k
    mean, std, q05, q95 = [o.cpu().numpy() for o in out]
    m, sd, a, b = oracle.ensemble_stats(got.reshape(64, npix))
    assert np.allclose(mean, m, rtol=1e-12, atol=1e-13 * np.abs(m).max())
    assert np.allclose(std, sd, rtol=1e-12, atol=1e-13 * np.abs(sd).max())
    assert np.array_equal(q05, a.astype(np.float32))
    assert np.array_equal(q95, b.astype(np.float32))


def test_velocity_ensemble_uncertainty_maps(ctx):
    """The uncertainty maps of the velocity samples themselves (the paper
    maps the std, confidence index and ratio of its velocity ensemble as
    well as of its images): 64 GRF samples of the full-size model, statistics
    and Eq. 6 / Eq. 7 maps on the GPU against the oracle's on the same samples."""
    s = inputs.full_size(nshot=1)
    ens = f32(inputs.ensemble(inputs.smooth(s.vel, s.dx, s.dz, 60.0), s.dx, s.dz, 64))
    npix = s.nz * s.nx
    x = torch.from_numpy(ens.reshape(64, npix)).cuda()
    out = [torch.zeros(npix, dtype=t, device="cuda")
           for t in (torch.float64, torch.float64, torch.float32, torch.float32)]
    ctx.ensemble_stats(x, *out)
    c = torch.zeros(npix, dtype=torch.float64, device="cuda")
    r = torch.zeros(npix, dtype=torch.float64, device="cuda")
    ctx.uncertainty_maps(out[0], out[1], c, r)
    torch.cuda.synchronize()
    m, sd, a, b = oracle.ensemble_stats(ens.reshape(64, npix))
    assert np.allclose(out[0].cpu().numpy(), m, rtol=1e-12)
    assert np.allclose(out[1].cpu().numpy(), sd, rtol=1e-10, atol=1e-9)
    assert np.array_equal(out[2].cpu().numpy(), a.astype(np.float32))
    assert np.array_equal(out[3].cpu().numpy(), b.astype(np.float32))
    oc, orr = oracle.uncertainty_maps(out[0].cpu().numpy(), out[1].cpu().numpy())
    assert np.allclose(c.cpu().numpy(), oc, rtol=1e-14, atol=1e-15)
    assert np.allclose(r.cpu().numpy(), orr, rtol=1e-14, atol=0)
    # the water layer is not perturbed: zero std, confidence 1 there
    assert np.all(out[1].cpu().numpy().reshape(s.nz, s.nx)[:40] == 0.0)
    assert np.all(c.cpu().numpy().reshape(s.nz, s.nx)[:40] == 1.0)


def _small(nx, nz, nb, nt, sx, sz, rec_iz):
    v = np.full((nz, nx), 2000.0, np.float32)
    s = inputs.Survey(nx, nz, nb, 10.0, 10.0, 1e-3, nt, v, np.array([sx], np.int32),
                      np.array([sz], np.int32), np.arange(nx, dtype=np.int32),
                      np.full(nx, rec_iz, np.int32), inputs.ricker(20.0, 1e-3, nt))
    return s, v


@pytest.mark.parametrize("case", ["no_imaging_step", "one_step", "one_cell", "no_sponge"])
def test_degenerate_migrations(ctx, case):
    """Degenerate cases against the oracle: no imaging step (isnap > nt: the
    image is exactly zero, reading 7's zero denominator), a single time step
    (receivers on the source row), a 1 x 1 grid (its filtered image is zero,
    so the raw image is compared too), and no sponge (nb = 0)."""
    if case == "no_imaging_step":
        s, v = _small(30, 20, 8, 50, 15, 3, 0)
        data = ora_model(s, v)[None]
        got = gpu_migrate(ctx, s, v, data, isnap=64)
        assert np.all(got == 0.0) and np.all(ora_migrate(s, v, data, isnap=64) == 0.0)
        return
    s, v, isnap = {"one_step": _small(30, 20, 8, 1, 15, 3, 3) + (1,),
                   "one_cell": _small(1, 1, 3, 40, 0, 0, 0) + (2,),
                   "no_sponge": _small(40, 24, 0, 120, 20, 2, 0) + (3,)}[case]
    want = ora_model(s, v)
    got = gpu_model(ctx, s, v)
    assert np.abs(want).max() > 0 and rel_l2(got, want) <= SEIS_TOL
    data = f32(want)[None]
    for lap in (True, False):
        gi, oi = gpu_migrate(ctx, s, v, data, isnap=isnap, lap=lap), ora_migrate(s, v, data, isnap,
                                                                                 lap=lap)
        if not np.any(oi):
            assert case == "one_cell" and lap and np.all(gi == 0.0)
        else:
            assert rel_l2(gi, oi) <= IMG_TOL, (case, lap)


def test_empty_acquisitions_are_refused(ctx):
    s, v = _small(30, 20, 8, 50, 15, 3, 0)
    keep = rtm._Keep()
    img = torch.zeros((s.nz, s.nx), dtype=torch.float32, device="cuda")
    seis = torch.zeros((1, s.nt, s.nx), dtype=torch.float32, device="cuda")
    opts = rtm.Opts(1, rtm.SNAP_F32, 1e-6, 1)
    none = np.zeros(0, np.int32)
    for acq, grid in ((rtm.make_acq(keep, none, none, s.rec_ix, s.rec_iz, f32(s.wavelet)),
                       rtm.make_grid(*s.grid_tuple())),
                      (rtm.make_acq(keep, s.src_ix, s.src_iz, none, none, f32(s.wavelet)),
                       rtm.make_grid(*s.grid_tuple())),
                      (rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, f32(s.wavelet)),
                       rtm.make_grid(s.nx, s.nz, s.nb, s.dx, s.dz, s.dt, 0))):
        with pytest.raises(rtm.RTMError) as e:
            ctx.migrate(grid, dev(v), acq, seis, opts, img)
        assert e.value.code == rtm.RTM_ERR_ARG


def test_size_limits(ctx):
    """The statistics kernel at its largest sample count (32768: one pixel per
    block, a 128 KB sort in shared memory) against the oracle, one sample
    more refused; a grid beyond the 2^31-point padded limit refused before
    any array is read."""
    n, npix = 32768, 37
    x = f32(inputs.normal(3, n * npix).reshape(n, npix))
    out = [torch.zeros(npix, dtype=t, device="cuda")
           for t in (torch.float64, torch.float64, torch.float32, torch.float32)]
    ctx.ensemble_stats(torch.from_numpy(x).cuda(), *out)
    torch.cuda.synchronize()
    m, sd, a, b = oracle.ensemble_stats(x)
    assert np.allclose(out[0].cpu().numpy(), m, rtol=1e-12, atol=1e-13)
    assert np.allclose(out[1].cpu().numpy(), sd, rtol=1e-12, atol=1e-13)
    assert np.array_equal(out[2].cpu().numpy(), a.astype(np.float32))
    assert np.array_equal(out[3].cpu().numpy(), b.astype(np.float32))
    with pytest.raises(rtm.RTMError) as e:
        ctx.ensemble_stats(torch.zeros((n + 1, npix), dtype=torch.float32, device="cuda"), *out)
    assert e.value.code == rtm.RTM_ERR_ARG
    s, v = _small(30, 20, 8, 50, 15, 3, 0)
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, f32(s.wavelet))
    huge = rtm.make_grid(50000, 50000, 20, 10.0, 10.0, 1e-3, 50)
    img = torch.zeros((s.nz, s.nx), dtype=torch.float32, device="cuda")
    with pytest.raises(rtm.RTMError) as e:
        ctx.migrate(huge, dev(v), acq, torch.zeros((1, 50, 30), device="cuda"),
                    rtm.Opts(1, rtm.SNAP_F32, 1e-6, 1), img)
    assert e.value.code == rtm.RTM_ERR_ARG
