"""Pins of the oracle's snapshot rounding and ensemble statistics.

- FP16 / BF16 rounding (round to nearest, ties to even) against numpy's
  float16 conversion and against an integer bit-level BF16 rounding of
  float32 values; per-snapshot scaling keeps the element error within the
  unit roundoff of the format (2^-11 FP16 normal range, 2^-8 BF16).
- Mean / standard deviation (divisor N-1) against closed forms; the 5% and
  95% quantiles against a brute-force sort and numpy's 'linear' method
  (Hyndman-Fan type 7); Eq. 6 and Eq. 7 maps against hand values (§2.3).
"""
import numpy as np
import pytest

import oracle
from paper_2001_06444_gb300 import inputs


def _bf16_rne_bits(x32: np.ndarray) -> np.ndarray:
    b = x32.view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def test_fp16_rounding_matches_numpy():
    y = inputs.normal(5, 4000) * np.exp(inputs.normal(6, 4000) * 4.0)
    y = np.concatenate([y, [6.103515625e-05, 2.0 ** -24, 3 * 2.0 ** -25, 1.0 + 2.0 ** -11,
                            1.0 + 3 * 2.0 ** -11, 2.0 ** -20 * 1.5]])
    y = y[np.abs(y) < 60000]
    mine = np.array([oracle.round_format(v, 11, -14) for v in y])
    ref = y.astype(np.float16).astype(np.float64)
    assert np.array_equal(mine, ref)


def test_bf16_rounding_matches_bit_rounding():
    y32 = (inputs.normal(7, 4000) * np.exp(inputs.normal(8, 4000) * 6.0)).astype(np.float32)
    ties = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(2.0 + 2.0 ** -7)], np.float32)
    y32 = np.concatenate([y32, ties])
    mine = np.array([oracle.round_format(float(v), 8, -126) for v in y32])
    assert np.array_equal(mine, _bf16_rne_bits(y32))


@pytest.mark.parametrize("mode,bound", [(2, 2.0 ** -11), (1, 2.0 ** -8)])
def test_snapshot_quantisation_error_bound(mode, bound):
    S = inputs.normal(9, 5000) * 3.7e-3
    q = oracle.quantize_snapshot(S, mode)
    mx = np.abs(S).max()
    assert np.abs(q).max() == pytest.approx(mx, rel=bound)
    if mode == 2:
        s = mx / 32768.0
        normal = np.abs(S / s) >= 2.0 ** -14
        assert np.all(np.abs(q - S)[normal] <= bound * np.abs(S)[normal])
        assert np.all(np.abs(q - S)[~normal] <= 2.0 ** -25 * s)
    else:
        assert np.all(np.abs(q - S) <= bound * np.abs(S))
    assert np.array_equal(oracle.quantize_snapshot(S, 0), S)
    assert np.array_equal(oracle.quantize_snapshot(np.zeros(10), mode), np.zeros(10))


def test_stats_closed_forms():
    # pixel p holds the values a_p + b_p * k for k = 0..N-1
    N, P = 21, 7
    k = np.arange(N)[:, None]
    a = np.linspace(-3, 3, P)[None, :]
    b = np.linspace(0.5, 2, P)[None, :]
    x = a + b * k
    mean, std, q05, q95 = oracle.ensemble_stats(x)
    assert np.allclose(mean, a[0] + b[0] * (N - 1) / 2)
    assert np.allclose(std, b[0] * np.sqrt(N * (N + 1) / 12.0))
    # h = (N-1) p = 1.0 and 19.0 exactly -> order statistics 1 and 19
    assert np.allclose(q05, a[0] + b[0] * 1.0)
    assert np.allclose(q95, a[0] + b[0] * 19.0)


@pytest.mark.parametrize("n", [1, 2, 5, 64, 97])
def test_quantiles_brute_force_and_numpy(n):
    x = inputs.normal(40 + n, n * 33).reshape(n, 33).astype(np.float32)
    mean, std, q05, q95 = oracle.ensemble_stats(x)
    xd = x.astype(np.float64)
    for p, q in ((0.05, q05), (0.95, q95)):
        assert np.allclose(q, np.quantile(xd, p, axis=0, method="linear"), rtol=0, atol=1e-12)
        for j in range(33):
            col = sorted(xd[:, j])
            h = (n - 1) * p
            lo = int(np.floor(h))
            hi = min(lo + 1, n - 1)
            assert q[j] == pytest.approx(col[lo] + (h - lo) * (col[hi] - col[lo]), abs=1e-12)
    if n > 1:
        assert np.allclose(std, xd.std(axis=0, ddof=1), rtol=1e-12)
    else:
        assert np.all(std == 0)


def test_uncertainty_maps_hand_values():
    mean = np.array([1.0, 2.0, 0.0, -4.0])
    std = np.array([0.5, 1.0, 2.0, 1.5])
    conf, ratio = oracle.uncertainty_maps(mean, std)
    assert np.allclose(conf, [1.0, 2 / 3, 0.0, 1 / 3])
    assert np.allclose(ratio, [0.5, 0.5, 0.0, -0.375])
    conf, _ = oracle.uncertainty_maps(mean, np.full(4, 0.3))
    assert np.all(conf == 1.0)
