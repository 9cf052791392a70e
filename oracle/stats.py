"""FP64 oracle of the ensemble statistics — TEST INFRASTRUCTURE ONLY.

Stage 3 of the workflow (§3) summarises the image ensemble per pixel (§2.3):
mean, standard deviation, the 5% / 95% quantiles, the confidence index of
Eq. 6 and the std/mean ratio of Eq. 7.  Plain numpy in float64.
"""
from __future__ import annotations

import numpy as np


def _quantile_type7(sorted_x: np.ndarray, p: float) -> np.ndarray:
    """Linear interpolation between order statistics at h = (N-1) p
    (Hyndman & Fan type 7).  sorted_x is sorted along axis 0."""
    n = sorted_x.shape[0]
    h = (n - 1) * p
    lo = int(np.floor(h))
    hi = min(lo + 1, n - 1)
    frac = h - lo
    return sorted_x[lo] + frac * (sorted_x[hi] - sorted_x[lo])


def ensemble_stats(images: np.ndarray):
    """images [N][...] -> (mean, std, q05, q95), all float64, per pixel.

    mean = sum(x) / N; std = sqrt(sum((x - mean)^2) / (N - 1)) (0 for N = 1).
    """
    x = np.asarray(images, dtype=np.float64)
    n = x.shape[0]
    mean = x.sum(axis=0) / n
    if n > 1:
        std = np.sqrt(((x - mean) ** 2).sum(axis=0) / (n - 1))
    else:
        std = np.zeros_like(mean)
    srt = np.sort(x, axis=0)
    return mean, std, _quantile_type7(srt, 0.05), _quantile_type7(srt, 0.95)


def uncertainty_maps(mean: np.ndarray, std: np.ndarray):
    """Confidence index c = (s_max - s) / (s_max - s_min) (Eq. 6), with the
    extremes taken over the whole map (1 everywhere when s_max == s_min), and
    the ratio r = s / mean (Eq. 7), 0 where mean == 0."""
    std = np.asarray(std, np.float64)
    mean = np.asarray(mean, np.float64)
    smax, smin = std.max(), std.min()
    if smax > smin:
        conf = (smax - std) / (smax - smin)
    else:
        conf = np.ones_like(std)
    ratio = np.zeros_like(std)
    nz = mean != 0
    ratio[nz] = std[nz] / mean[nz]
    return conf, ratio
