"""GPU codec (rtm_compress / rtm_decompress) against the codec oracle:
streams byte-identical, decoded arrays bit-identical, on ragged shapes that
span several chunks and tiles, in both modes, through device and host
pointers; at full size (one 5000 x 1701 seismogram at the paper's 1e-4
tolerance, and a batch of images) byte-identical streams too; malformed
streams and non-finite inputs are reported."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2001_06444_gb300 import inputs, rtm

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = rtm.Context(0)
    yield c
    c.close()


def _arrays(seed, count, n0, n1, kind):
    if kind == "normal":
        a = inputs.normal(seed, count * n0 * n1).reshape(count, n0, n1) * 3.0
        a[:, min(1, n0 - 1), :] *= 1e-5
        return a.astype(np.float32)
    if kind == "smooth":
        out = np.stack([inputs.smooth(inputs.layered_faulted(n0, n1, 10.0, 10.0, seed=seed + i),
                                      10, 10, 30.0) for i in range(count)])
        return out.astype(np.float32)
    bits = (inputs.uniform(seed, count * n0 * n1) * 2 ** 32).astype(np.uint64).astype(np.uint32)
    return bits.view(np.float32).reshape(count, n0, n1).copy()


def _check_against_oracle(ctx, x, tol, via_host=False):
    count, n0, n1 = x.shape
    data = x if via_host else torch.from_numpy(x).cuda()
    out, stride, sizes = ctx.compress(data, tol)
    blob = out if via_host else out.cpu().numpy()
    dec = np.zeros_like(x) if via_host else torch.zeros(x.shape, dtype=torch.float32,
                                                         device="cuda")
    ctx.decompress(out, stride, count, n0, n1, dec)
    dec = dec if via_host else dec.cpu().numpy()
    for i in range(count):
        want = oracle.codec_compress(x[i], tol)
        got = blob[i * stride:i * stride + sizes[i]].tobytes()
        assert sizes[i] == len(want), (i, sizes[i], len(want))
        assert got == want, i
        ref = oracle.codec_decompress(want, n0, n1)
        assert np.array_equal(dec[i].view(np.uint32), ref.view(np.uint32)), i
    return sizes


@pytest.mark.parametrize("shape", [(1, 4, 4), (3, 23, 38), (2, 130, 301), (1, 257, 1030),
                                   (2, 1, 1), (1, 1, 37), (3, 130, 1), (1, 5, 3)])
@pytest.mark.parametrize("kind,tols", [("normal", (1e-6, 1e-3, 0.5, 0.0)),
                                       ("smooth", (1e-4, 1e-1, 0.0)),
                                       ("bits", (0.0,))])
def test_streams_identical_to_oracle(ctx, shape, kind, tols):
    x = _arrays(7, *shape, kind)
    for tol in tols:
        _check_against_oracle(ctx, x, tol)


def test_host_pointers(ctx):
    x = _arrays(9, 2, 61, 77, "normal")
    _check_against_oracle(ctx, x, 1e-3, via_host=True)
    _check_against_oracle(ctx, x, 0.0, via_host=True)


def test_full_size_seismogram_and_images(ctx):
    # one shot of the 1701-receiver, 5000-sample survey (§4.2 compresses
    # seismograms at 1e-4) and 8 images of the 1701 x 351 grid
    nt, nrec = 5000, 1701
    seis = inputs.normal(21, nt * nrec).reshape(1, nt, nrec).astype(np.float32)
    t = np.arange(nt)[:, None]
    seis[0] *= np.exp(-t / 1500.0).astype(np.float32) * 1e-3  # decaying traces
    sizes = _check_against_oracle(ctx, seis, 1e-4)
    assert sizes[0] < seis.nbytes
    imgs = _arrays(31, 8, 351, 1701, "smooth")
    _check_against_oracle(ctx, imgs, 1e-1)


def test_error_bound_and_lossless_on_device(ctx):
    x = _arrays(41, 4, 300, 517, "normal")
    for tol in (1e-2, 1e-5):
        d = torch.from_numpy(x).cuda()
        out, stride, sizes = ctx.compress(d, tol)
        y = torch.zeros_like(d)
        ctx.decompress(out, stride, 4, 300, 517, y)
        err = (y - d).abs().cpu().numpy()
        mx = np.abs(x).max()
        assert err.max() <= max(tol, 2.0 ** (np.frexp(mx)[1] - 23))
    bits = _arrays(43, 2, 100, 90, "bits")
    d = torch.from_numpy(bits).cuda()
    out, stride, sizes = ctx.compress(d, 0.0)
    y = torch.zeros_like(d)
    ctx.decompress(out, stride, 2, 100, 90, y)
    assert torch.equal(y.view(torch.int32), d.view(torch.int32))


def test_nonfinite_and_malformed_are_reported(ctx):
    x = _arrays(51, 3, 40, 40, "normal")
    x[1, 7, 9] = np.inf
    d = torch.from_numpy(x).cuda()
    with pytest.raises(rtm.RTMError) as ei:
        ctx.compress(d, 1e-3)
    assert ei.value.code == rtm.RTM_ERR_ARG
    stride = (rtm.compress_bound(40, 40) + 15) // 16 * 16
    out = torch.zeros(3 * stride, dtype=torch.uint8, device="cuda")
    sizes = (C.c_uint64 * 3)()
    rc = rtm.lib().rtm_compress(ctx.h, C.c_void_p(d.data_ptr()), 3, 40, 40, 1e-3,
                                C.c_void_p(out.data_ptr()), stride, sizes, None)
    assert rc == rtm.RTM_ERR_ARG and sizes[1] == 0 and sizes[0] > 0 and sizes[2] > 0
    # the two good streams still decode like the oracle's
    for i in (0, 2):
        got = out[i * stride:i * stride + sizes[i]].cpu().numpy().tobytes()
        assert got == oracle.codec_compress(x[i], 1e-3)
    # damaged streams: wrong shape, bad magic, a cut bit section
    good, stride, sizes = ctx.compress(torch.from_numpy(x[[0, 2]]).cuda(), 1e-3)
    y = torch.zeros((2, 40, 40), dtype=torch.float32, device="cuda")
    with pytest.raises(rtm.RTMError):
        ctx.decompress(good, stride, 2, 40, 41, torch.zeros((2, 40, 41), device="cuda"))
    bad = good.clone()
    bad[stride] ^= 1
    with pytest.raises(rtm.RTMError, match="stream 1"):
        ctx.decompress(bad, stride, 2, 40, 40, y)
    bad = good.clone()
    bad[40:48] = torch.tensor(np.frombuffer(np.uint64(3).tobytes(), np.uint8).copy())
    with pytest.raises(rtm.RTMError, match="stream 0"):
        ctx.decompress(bad, stride, 2, 40, 40, y)
    ctx.decompress(good, stride, 2, 40, 40, y)  # the context is still usable
    assert np.array_equal(y.cpu().numpy()[1], oracle.codec_decompress(
        oracle.codec_compress(x[2], 1e-3), 40, 40))


def test_migration_through_the_codec(ctx):
    """The paper's compression-error experiment (§4.2) on the flat-reflector
    survey: seismograms and velocity passed through the codec, then migrated.
    Lossless round trips give the uncompressed image bit for bit.  At 1e-4
    the image is linear in the data (the illumination denominator depends on
    the velocity alone), so its relative error stays within a small multiple
    of the seismograms' relative error."""
    import oracle
    from conftest import rel_l2

    s = inputs.flat_reflector(nt=600)
    g = oracle.grid(*s.grid_tuple())
    w = s.wavelet.astype(np.float32).astype(np.float64)
    seis = np.stack([oracle.model(g, s.vel.astype(np.float64), s.src_ix[k], s.src_iz[k],
                                  s.rec_ix, s.rec_iz, w) for k in range(len(s.src_ix))])
    seis = torch.from_numpy(seis.astype(np.float32)).cuda()
    vel = torch.from_numpy(s.vel.astype(np.float32)).cuda()[None].contiguous()
    keep = rtm._Keep()
    acq = rtm.make_acq(keep, s.src_ix, s.src_iz, s.rec_ix, s.rec_iz, s.wavelet.astype(np.float32))
    grid = rtm.make_grid(*s.grid_tuple())
    opts = rtm.Opts(2, rtm.SNAP_F32, 1e-6, 1)

    def migrate(sd, vd):
        img = torch.zeros((s.nz, s.nx), dtype=torch.float32, device="cuda")
        ctx.migrate(grid, vd[0], acq, sd, opts, img)
        torch.cuda.synchronize()
        return img.cpu().numpy()

    def round_trip(x, tol):
        count, n0, n1 = x.shape
        stride = (rtm.compress_bound(n0, n1) + 15) // 16 * 16
        out = torch.empty(count * stride, dtype=torch.uint8, device="cuda")
        back = torch.empty_like(x)
        ctx.compress(x, tol, out, stride)
        ctx.decompress(out, stride, count, n0, n1, back)
        return back

    ref = migrate(seis, vel)
    assert np.array_equal(migrate(round_trip(seis, 0.0), round_trip(vel, 0.0)), ref)
    sq = round_trip(seis, 1e-4)
    data_err = rel_l2(sq.cpu().numpy(), seis.cpu().numpy())
    img_err = rel_l2(migrate(sq, round_trip(vel, 1e-4)), ref)
    assert 0 < data_err and img_err <= 10 * data_err, (img_err, data_err)
    print(f"1e-4: seismograms within {data_err:.1e}, image within {img_err:.1e} (relative L2)")


def test_damaged_streams_decode_or_are_rejected(ctx):
    # bytes of valid streams overwritten at seeded positions (header, chunk
    # index, bit section): every call either decodes or reports the stream
    # as malformed, and reads stay inside each stream and its chunks, so the
    # context keeps working
    x = _arrays(61, 2, 133, 517, "normal")
    x[1] *= np.exp(-np.arange(133) / 30.0)[:, None].astype(np.float32)
    count, n0, n1 = x.shape
    for tol in (1e-3, 0.0):
        good, stride, sizes = ctx.compress(torch.from_numpy(x).cuda(), tol)
        ref = torch.zeros(x.shape, dtype=torch.float32, device="cuda")
        ctx.decompress(good, stride, count, n0, n1, ref)
        u = inputs.uniform(71 if tol else 73, 4 * 40)
        nchunk = -(-(-(-n0 // 4) * -(-n1 // 4)) // 32)
        ib = 16 * -(-nchunk // 4)  # the chunk index follows the 64-byte header
        rejected = 0
        for t in range(40):
            bad = good.clone()
            s = int(u[4 * t] * count)
            region = int(u[4 * t + 1] * 3)  # 0 header, 1 index, 2 bit section
            lo, hi = ((0, 64), (64, 64 + ib), (64 + ib, int(sizes[s])))[region]
            pos = s * stride + lo + int(u[4 * t + 2] * (hi - lo))
            bad[pos] ^= 1 + int(u[4 * t + 3] * 255)
            y = torch.zeros_like(ref)
            try:
                ctx.decompress(bad, stride, count, n0, n1, y)
            except rtm.RTMError as e:
                assert e.code == rtm.RTM_ERR_ARG
                assert f"stream {s}" in str(e)
                rejected += 1
            else:
                # accepted: the other stream decodes as before
                o = 1 - s
                assert torch.equal(y[o].view(torch.int32), ref[o].view(torch.int32))
        assert rejected >= 10
        y = torch.zeros_like(ref)
        ctx.decompress(good, stride, count, n0, n1, y)
        assert torch.equal(y.view(torch.int32), ref.view(torch.int32))


def test_mixed_modes_over_several_groups(ctx):
    # 4100 small arrays in one decompression: more blocks than one group of
    # the decoder's lists holds, so it runs in two groups of 2050; quarters
    # coded alternately at 1e-3 and losslessly into one buffer, so each
    # group holds streams of both modes
    count, n0, n1 = 4100, 20, 23
    x = _arrays(81, count, n0, n1, "normal")
    x[::3] *= np.float32(1e-3)  # some arrays with many all-zero blocks at 1e-3
    d = torch.from_numpy(x).cuda()
    stride = (rtm.compress_bound(n0, n1) + 15) // 16 * 16
    out = torch.zeros(count * stride, dtype=torch.uint8, device="cuda")
    edges = [0, 1025, 2050, 3075, count]
    tols = np.zeros(count)
    sizes = []
    for q in range(4):
        lo, hi = edges[q], edges[q + 1]
        tol = 1e-3 if q % 2 == 0 else 0.0
        tols[lo:hi] = tol
        _, _, sz = ctx.compress(d[lo:hi].contiguous(), tol, out[lo * stride:hi * stride], stride)
        sizes += list(sz)
    y = torch.zeros_like(d)
    ctx.decompress(out, stride, count, n0, n1, y)
    got = y.cpu().numpy()
    blob = out.cpu().numpy()
    for i in list(range(0, count, 97)) + [1024, 1025, 2049, 2050, 3074, 3075, count - 1]:
        want = oracle.codec_compress(x[i], tols[i])
        assert blob[i * stride:i * stride + sizes[i]].tobytes() == want, i
        ref = oracle.codec_decompress(want, n0, n1)
        assert np.array_equal(got[i].view(np.uint32), ref.view(np.uint32)), i
    ll = tols == 0.0
    assert np.array_equal(got[ll].view(np.uint32), x[ll].view(np.uint32))
    assert np.abs(got[~ll] - x[~ll]).max() <= 1e-3
