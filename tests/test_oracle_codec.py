"""Pins of the codec oracle (the transform block codec used between the
workflow's stages, §3 / §4.2, Tables 1-2):

- the integer transform is exactly reversible and maps a constant block to a
  single coefficient;
- fixed accuracy: every decoded element lies within max(tol, 2^(e-23)) of
  its input (e: the block exponent), on data of very different scales,
  including subnormal ones;
- lossless: every float bit pattern (NaN, infinities, -0, subnormals) comes
  back exactly;
- two streams worked out by hand from the coding rules, bit by bit, and the
  stream length of a constant block and of an all-zero array;
- the lowest kept plane follows its closed form;
- malformed streams are rejected.
"""
import math
import struct

import numpy as np
import pytest

import oracle
from paper_2001_06444_gb300 import inputs

HEADER = 64


def _words(blob):
    """(words of the bit section, chunk index, bit-section words)."""
    nwords, nchunk = struct.unpack_from("<QQ", blob, 40)
    start = HEADER + 16 * ((nchunk + 3) // 4)
    index = np.frombuffer(blob, np.uint32, nchunk, HEADER)
    return nwords, index, np.frombuffer(blob, np.uint32, nwords, start)


def _block_exponents(x):
    n0, n1 = x.shape
    e = np.zeros(x.shape)
    for bi in range(0, n0, 4):
        for bj in range(0, n1, 4):
            # edge blocks repeat their last row/column: same maximum
            m = np.abs(x[bi:bi + 4, bj:bj + 4].astype(np.float64)).max()
            e[bi:bi + 4, bj:bj + 4] = math.frexp(m)[1] if m > 0 else -200
    return e


def test_transform_is_exactly_reversible():
    u = inputs.uniform(3, 16 * 500)
    for t in range(500):
        q = np.rint((u[16 * t:16 * t + 16] * 2 - 1) * 2 ** 31).astype(np.int64).reshape(4, 4)
        fwd, back = oracle.codec_transform(q)
        assert np.array_equal(back, q)
        assert np.abs(fwd).max() < 2 ** 33  # lossless coding starts at plane 32
    fwd, back = oracle.codec_transform(np.full((4, 4), 12345))
    want = np.zeros((4, 4), np.int64)
    want[0, 0] = 12345
    assert np.array_equal(fwd, want)
    # a ramp along each row: s = 15 (rounded mean), differences 20, 10, 10
    fwd, _ = oracle.codec_transform(np.tile(np.array([0, 10, 20, 30]), (4, 1)))
    assert fwd[0].tolist() == [15, 20, 10, 10] and np.all(fwd[1:] == 0)


@pytest.mark.parametrize("scale", [1e-40, 1e-30, 1e-3, 1.0, 3e4, 1e30])
@pytest.mark.parametrize("rel_tol", [1e-1, 1e-4, 1e-7])
def test_error_bound(scale, rel_tol):
    n0, n1 = 23, 38  # ragged edge blocks in both directions, two chunks
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


def test_lossless_round_trip_of_every_bit_pattern():
    bits = (inputs.uniform(6, 37 * 61) * 2 ** 32).astype(np.uint64).astype(np.uint32)
    x = bits.view(np.float32).reshape(37, 61).copy()  # includes NaNs and infinities
    special = np.array([np.nan, np.inf, -np.inf, -0.0, 0.0, 1e-45, -1e-45, 3.4e38],
                       np.float32)
    x[0, :8] = special
    x[20:24, 12:16] = 0.0
    blob = oracle.codec_compress(x, 0.0)
    y = oracle.codec_decompress(blob, 37, 61)
    assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
    smooth = inputs.smooth(inputs.layered_faulted(64, 96, 10.0, 10.0, seed=3), 10, 10, 40.0)
    smooth = smooth.astype(np.float32)
    blob = oracle.codec_compress(smooth, 0.0)
    assert len(blob) < smooth.nbytes
    y = oracle.codec_decompress(blob, 64, 96)
    assert np.array_equal(smooth.view(np.uint32), y.view(np.uint32))


def test_hand_coded_lossless_block():
    # 16 copies of the smallest subnormal: ordered integer 1 everywhere, so
    # the transform leaves one coefficient, 1.  Bits: flag 1; planes 32..1:
    # a failed group test each (32 zeros); plane 0: group 1, coefficient 0
    # has the bit (1), group 0 for the other 15; refinement of coefficient 0:
    # no planes below 0, its sign (0).  37 bits: word 0 = 1, word 1 = 0b110.
    x = np.full((4, 4), 1e-45, np.float32)
    assert x.view(np.uint32)[0, 0] == 1
    nwords, index, words = _words(oracle.codec_compress(x, 0.0))
    assert nwords == 2 and index.tolist() == [0] and words.tolist() == [1, 6]


def test_hand_coded_block_with_a_scanned_zero_member():
    # rows [s, s, 0, 0], s the smallest subnormal (ordered integer 1), coded
    # losslessly.  Each row [1, 1, 0, 0] transforms to (ss, dd, d1, d2) =
    # (0, -1, 0, 0): d1 = d2 = 0, s1 = 1, s2 = 0, dd = s2 - s1 = -1, ss = s1 +
    # floor(-1/2) = 0; the columns are then constant, so the one coefficient
    # left is -1 at (0, 1), coding position 1.  Bits: flag 1 (bit 0); planes
    # 32..1 fail (bits 1..32); plane 0: group 1 (33), coefficient 0 lacks the
    # bit (34: 0, a scanned member), coefficient 1 has it (35: 1), group 0
    # for the other 14 (36); refinement, no planes below 0: the scanned
    # member's sign bit, 0 as its kept magnitude is zero (37), the found
    # member's sign, 1 (38).  Word 1 = 2^1 + 2^3 + 2^6 = 74; without a sign
    # bit for the zero member it would be 42.
    s = np.uint32(1).view(np.float32)
    x = np.tile(np.array([s, s, 0.0, 0.0], np.float32), (4, 1))
    f, _ = oracle.codec_transform(x.view(np.uint32).astype(np.int64))
    want = np.zeros((4, 4), np.int64)
    want[0, 1] = -1
    assert np.array_equal(f, want)
    blob = oracle.codec_compress(x, 0.0)
    nwords, index, words = _words(blob)
    assert nwords == 2 and index.tolist() == [0] and words.tolist() == [1, 74]
    y = oracle.codec_decompress(blob, 4, 4)
    assert np.array_equal(y.view(np.uint32), x.view(np.uint32))


def test_hand_coded_fixed_accuracy_block():
    # 16 copies of 0.75 at tol 0.5: e = 0 (0.75 = 0.75 2^0), kmin = 22
    # (16 2^22 + 21.5 <= 2^27 < 16 2^23 + 21.5); q = 3 2^26, one coefficient,
    # top bit on plane 27.  Bits: flag (bit 0); e + 150 = 150 in 9 bits (bits
    # 2, 3, 5, 8); planes 30..28 fail (10..12); plane 27: group 1 (13), the
    # bit (14), group 0 (15); planes 26..22 fail (16..20); refinement planes
    # 22..26 = 0,0,0,0,1 (bit 25); sign 0 (26).
    x = np.full((4, 4), 0.75, np.float32)
    assert oracle.codec_kmin(0.5, 0) == 22
    blob = oracle.codec_compress(x, 0.5)
    nwords, _, words = _words(blob)
    want = sum(1 << b for b in (0, 2, 3, 5, 8, 13, 14, 25))
    assert nwords == 1 and words.tolist() == [want]
    # decoded: (48 2^22 + 2^21) 2^-28, the midpoint of the kept interval
    assert np.all(oracle.codec_decompress(blob, 4, 4) == np.float32(0.75 + 2 ** -7))


def test_constant_block_stream_length():
    # one block of value 3.0 (e = 2): one coefficient, 3 2^26, top plane 27.
    # 10 (flag, exponent) + significance 3 + 2 + 1 + (27 - kmin) +
    # refinement (27 - kmin) + 1 sign.
    tol = 1e-3
    kmin = oracle.codec_kmin(tol, 2)
    assert kmin == 12  # 16 2^12 + 21.5 <= 1e-3 2^26 < 16 2^13 + 21.5
    nwords, _, words = _words(oracle.codec_compress(np.full((4, 4), 3.0, np.float32), tol))
    nbits = 10 + 6 + 2 * (27 - kmin) + 1
    assert nwords == (nbits + 31) // 32
    assert int(words[-1]) >> ((nbits - 1) % 32) <= 1  # nothing beyond the last bit
    assert (int(words[nbits // 32]) >> ((nbits - 2) % 32)) & 1 == 1  # refinement top bit


def test_zero_array_costs_one_bit_per_block():
    # 5 x 8 blocks = a chunk of 32 (one word) and a chunk of 8 (one word)
    blob = oracle.codec_compress(np.zeros((17, 30), np.float32), 1e-3)
    nwords, index, words = _words(blob)
    assert nwords == 2 and index.tolist() == [0, 1] and words.tolist() == [0, 0]
    assert np.all(oracle.codec_decompress(blob, 17, 30) == 0)


def test_kmin_closed_form():
    for tol, e in ((1e-3, 2), (0.5, -5), (1e-12, 10), (1e3, 0), (7.0, 3), (1e30, -100)):
        T = math.ldexp(tol, 28 - e)
        want = 0
        while want < 30 and 16 * 2 ** (want + 1) + 21.5 <= T:
            want += 1
        assert oracle.codec_kmin(tol, e) == want


def test_ratio_grows_with_tolerance_and_smoothness():
    smooth = inputs.smooth(inputs.layered_faulted(120, 300, 10.0, 10.0, seed=2), 10, 10, 40.0)
    noise = inputs.normal(4, 120 * 300).reshape(120, 300) * smooth.std() + smooth.mean()
    sizes = [len(oracle.codec_compress(smooth, t)) for t in (0.0, 1e-4, 1e-2, 1.0)]
    # velocities of 1500-4500 m/s: 1e-4 is below float precision there, so
    # fixed accuracy keeps every plane and lossless is as small (the paper's
    # velocity column of Table 1 shows the same)
    assert sizes[0] < smooth.nbytes and sizes[0] <= sizes[1] > sizes[2] > sizes[3]
    assert len(oracle.codec_compress(smooth, 1.0)) < len(oracle.codec_compress(noise, 1.0))
    assert len(oracle.codec_compress(noise, 1.0)) <= oracle.codec_bound(120, 300)


def test_malformed_streams_are_rejected():
    x = inputs.normal(8, 30 * 30).reshape(30, 30).astype(np.float32)
    blob = bytearray(oracle.codec_compress(x, 1e-3))
    with pytest.raises(ValueError):
        oracle.codec_decompress(bytes(blob), 30, 31)  # wrong shape
    with pytest.raises(ValueError):
        oracle.codec_decompress(bytes(blob[:len(blob) - 8]), 30, 30)  # truncated
    bad = bytearray(blob)
    bad[0] ^= 1
    with pytest.raises(ValueError):
        oracle.codec_decompress(bytes(bad), 30, 30)  # magic
    with pytest.raises(ValueError):
        oracle.codec_compress(np.full((4, 4), np.nan, np.float32), 1e-3)


@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (130, 1), (5, 3)])
def test_degenerate_shapes(shape):
    x = inputs.normal(13, shape[0] * shape[1]).reshape(shape).astype(np.float32)
    y = oracle.codec_decompress(oracle.codec_compress(x, 1e-3), *shape)
    assert np.all(np.abs(y.astype(np.float64) - x) <= 1e-3)
    y = oracle.codec_decompress(oracle.codec_compress(x, 0.0), *shape)
    assert np.array_equal(x.view(np.uint32), y.view(np.uint32))
