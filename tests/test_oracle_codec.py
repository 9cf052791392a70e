"""Pins of the codec oracle (the fixed-accuracy block codec used between the
workflow's stages, §3 / §4.2):

- the integer transform is exactly reversible and maps a constant block to a
  single coefficient;
- every decoded element lies within max(tol, 2^(e-23)) of its input (e: the
  block exponent), on data of very different scales;
- small integers round-trip exactly;
- the stream length of a constant block and of an all-zero array follow from
  the coding rules by hand;
- the lowest kept plane follows its closed form.
"""
import math
import struct

import numpy as np
import pytest

import oracle
from paper_2001_06444_gb300 import inputs


def _stream_bits(blob):
    return struct.unpack_from("<Q", blob, 32)[0]


def _block_exponents(x):
    n0, n1 = x.shape
    e = np.zeros(x.shape)
    for bi in range(0, n0, 4):
        for bj in range(0, n1, 4):
            blk = x[bi:bi + 4, bj:bj + 4].astype(np.float64)
            # edge blocks repeat their last row/column: same maximum
            m = np.abs(blk).max()
            e[bi:bi + 4, bj:bj + 4] = math.frexp(m)[1] if m > 0 else -200
    return e


def test_transform_is_exactly_reversible():
    u = inputs.uniform(3, 16 * 500)
    for t in range(500):
        q = np.rint((u[16 * t:16 * t + 16] * 2 - 1) * 2 ** 28).astype(np.int32).reshape(4, 4)
        fwd, back = oracle.codec_transform(q)
        assert np.array_equal(back, q)
    fwd, back = oracle.codec_transform(np.full((4, 4), 12345, np.int32))
    want = np.zeros((4, 4), np.int32)
    want[0, 0] = 12345
    assert np.array_equal(fwd, want)
    # a ramp along a row: level-1 differences are the step, the rest follow
    fwd, _ = oracle.codec_transform(np.tile(np.array([0, 10, 20, 30], np.int32), (4, 1)))
    assert fwd[0].tolist() == [15, 20, 10, 10] and np.all(fwd[1:] == 0)


@pytest.mark.parametrize("scale", [1e-30, 1e-3, 1.0, 3e4, 1e30])
@pytest.mark.parametrize("rel_tol", [1e-1, 1e-4, 1e-7])
def test_error_bound(scale, rel_tol):
    n0, n1 = 23, 38  # ragged edge blocks in both directions
    x = (inputs.normal(11, n0 * n1).reshape(n0, n1) * scale).astype(np.float32)
    x[5, :] *= 1e-6  # large dynamic range inside blocks
    x[8:12, 8:12] = 0.0  # an all-zero block
    tol = rel_tol * scale
    y = oracle.codec_decompress(oracle.codec_compress(x, tol), n0, n1)
    bound = np.maximum(tol, np.ldexp(1.0, (_block_exponents(x) - 23).astype(int)))
    assert np.all(np.abs(y.astype(np.float64) - x) <= bound)
    assert np.all(y[8:12, 8:12] == 0.0)


def test_small_integers_round_trip_exactly():
    x = np.rint((inputs.uniform(5, 40 * 40) - 0.5) * 2000).reshape(40, 40).astype(np.float32)
    y = oracle.codec_decompress(oracle.codec_compress(x, 1e-9), 40, 40)
    assert np.array_equal(x, y)


def test_constant_block_stream_length():
    # one block of value 3.0 (e = 2): only coefficient (0, 0) = 3 * 2^26 is
    # nonzero; its top bit is plane 27.  Bits: 1 flag + 9 exponent; planes
    # 30..28: a zero group test each; plane 27: group 1, its bit, its sign,
    # then group 0 for the other 15; planes 26..kmin: its bit and a zero
    # group test.
    tol = 1e-3
    kmin = oracle.codec_kmin(tol, 2)
    assert kmin == 12  # 16 * 2^13 + 21.5 <= 1e-3 * 2^26 < 16 * 2^14 + 21.5
    blob = oracle.codec_compress(np.full((4, 4), 3.0, np.float32), tol)
    assert _stream_bits(blob) == 10 + 3 + 4 + 2 * (27 - kmin)
    y = oracle.codec_decompress(blob, 4, 4)
    assert np.all(np.abs(y - 3.0) <= tol)


def test_zero_array_costs_one_bit_per_block():
    blob = oracle.codec_compress(np.zeros((17, 30), np.float32), 1e-3)
    assert _stream_bits(blob) == 5 * 8
    assert np.all(oracle.codec_decompress(blob, 17, 30) == 0)


def test_kmin_closed_form():
    for tol, e in ((1e-3, 2), (0.5, -5), (1e-12, 10), (1e3, 0), (7.0, 3)):
        T = math.ldexp(tol, 28 - e)
        want = 0
        while want < 30 and 16 * 2 ** (want + 1) + 21.5 <= T:
            want += 1
        assert oracle.codec_kmin(tol, e) == want


def test_ratio_grows_with_tolerance_and_smoothness():
    smooth = inputs.smooth(inputs.layered_faulted(120, 300, 10.0, 10.0, seed=2), 10, 10, 40.0)
    noise = inputs.normal(4, 120 * 300).reshape(120, 300) * smooth.std() + smooth.mean()
    sizes = [len(oracle.codec_compress(smooth, t)) for t in (1e-4, 1e-2, 1.0)]
    assert sizes[0] > sizes[1] > sizes[2]
    assert len(oracle.codec_compress(smooth, 1.0)) < len(oracle.codec_compress(noise, 1.0))
