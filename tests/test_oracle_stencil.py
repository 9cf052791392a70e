"""Pins of the oracle's spatial operators against closed forms.

- The 8th-order Laplacian (§3: "eighth order in space") must be exact on
  polynomials of degree <= 9 and not on degree 10, and its symbol at the
  Nyquist wavenumber must be -2048/315 per axis.
- The stability limit of leapfrog with that stencil is
  v dt / h <= 2 / sqrt(2 * 2048/315) for square cells; the oracle's scheme must
  stay bounded just below it and blow up just above it.
- The Laplacian image filter of §3 (-(D_zz + D_xx), 3-point, replicated
  border) is checked on quadratics and on a linear ramp at the border.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2001_06444_gb300 import inputs


def _poly_field(nz, nx, dz, dx, kz, kx):
    z = (np.arange(nz) - nz // 2) * dz
    x = (np.arange(nx) - nx // 2) * dx
    return z[:, None] ** kz * np.ones((1, nx)) + np.ones((nz, 1)) * x[None, :] ** kx, z, x


@pytest.mark.parametrize("k", range(0, 10))
def test_laplacian8_exact_on_polynomials(k):
    nz, nx, dz, dx = 21, 25, 0.5, 0.25
    a, z, x = _poly_field(nz, nx, dz, dx, k, k)
    lap = oracle.laplacian8(a, dz, dx)
    exact = np.zeros_like(a)
    if k >= 2:
        exact = k * (k - 1) * (z[:, None] ** (k - 2) + x[None, :] ** (k - 2))
    inner = (slice(4, nz - 4), slice(4, nx - 4))
    scale = max(1.0, np.abs(exact[inner]).max())
    assert np.abs(lap[inner] - exact[inner]).max() <= 1e-9 * scale


def test_laplacian8_not_exact_on_degree_10():
    nz, nx, dz, dx = 21, 21, 0.5, 0.5
    a, z, x = _poly_field(nz, nx, dz, dx, 10, 0)
    lap = oracle.laplacian8(a, dz, dx)
    exact = 90.0 * z[:, None] ** 8 * np.ones((1, nx))
    inner = (slice(4, nz - 4), slice(4, nx - 4))
    err = np.abs(lap[inner] - exact[inner])
    # leading error term of an 8th-order second difference: -h^8 f^(10) / 3150
    expected = dz ** 8 * math.factorial(10) / 3150.0
    assert np.allclose(err, expected, rtol=1e-6)


def test_laplacian8_symbol_at_nyquist():
    nz, nx, dz, dx = 16, 18, 2.0, 3.0
    i = np.arange(nz)[:, None]
    j = np.arange(nx)[None, :]
    a = (-1.0) ** (i + j)
    lap = oracle.laplacian8(a, dz, dx)
    inner = (slice(4, nz - 4), slice(4, nx - 4))
    want = -2048.0 / 315.0 * (1 / dz ** 2 + 1 / dx ** 2) * a
    assert np.allclose(lap[inner], want[inner], rtol=1e-13, atol=0)


def test_cfl_closed_form():
    limit = 2.0 / math.sqrt(2.0 * 2048.0 / 315.0)
    assert abs(limit - 0.55463) < 1e-5
    # courant number 1 exactly at the closed-form limit, square cells
    assert oracle.courant(limit, 1.0, 1.0, 1.0) == pytest.approx(1.0, rel=1e-14)
    # rectangular cells: v dt sqrt((1/dx^2 + 1/dz^2) 2048/315) / 2
    c = oracle.courant(3000.0, 1e-3, 10.0, 7.0)
    assert c == pytest.approx(3.0 * math.sqrt((1 / 100 + 1 / 49) * 2048 / 315) / 2, rel=1e-14)


def _impulse_run(courant_number, nt):
    nz = nx = 24
    g = oracle.grid(nx, nz, 4, 10.0, 10.0, 1e-3, nt)
    limit = 2.0 / math.sqrt(2.0 * 2048.0 / 315.0)
    v = np.full((nz, nx), courant_number * limit * 10.0 / 1e-3)
    w = np.zeros(nt)
    w[0] = 1.0
    rx = np.arange(nx, dtype=np.int32)
    rz = np.full(nx, nz // 2, np.int32)
    return oracle.model(g, v, nx // 2, nz // 2, rx, rz, w)


def test_stability_limit_is_the_schemes():
    """Just below the limit the oracle's recurrence stays bounded; just above
    it grows without bound (CPU only)."""
    below = _impulse_run(0.995, 4000)
    above = _impulse_run(1.02, 400)
    assert np.all(np.isfinite(below))
    assert np.abs(below[-500:]).max() <= 10 * np.abs(below[:50]).max()
    assert np.all(np.isfinite(above))
    assert np.abs(above[-50:]).max() >= 1e20 * np.abs(above[:20]).max()


def test_image_filter_on_quadratic_and_border():
    nz, nx, dz, dx = 12, 15, 10.0, 5.0
    z = np.arange(nz)[:, None] * dz
    x = np.arange(nx)[None, :] * dx
    img = 3.0 * z ** 2 - 2.0 * x ** 2 + 0.5 * x * z + 7.0
    out = oracle.image_filter(img, dz, dx)
    # -(d2/dz2 + d2/dx2) = -(6 - 4) = -2 away from the border
    assert np.allclose(out[1:-1, 1:-1], -2.0, rtol=0, atol=1e-9)
    ramp = np.ones((nz, 1)) * (np.arange(nx)[None, :] * dx)
    out = oracle.image_filter(ramp, dz, dx)
    assert np.allclose(out[:, 1:-1], 0.0, atol=1e-12)
    # replicated border: first column sees (I_1 - I_0) / dx^2 -> -1/dx
    assert np.allclose(out[:, 0], -1.0 / dx, atol=1e-12)
    assert np.allclose(out[:, -1], 1.0 / dx, atol=1e-12)


def test_sponge_profile_shape():
    g = oracle.grid(30, 20, 10, 10.0, 10.0, 1e-3, 1)
    s = oracle.sponge(g)
    NZ, NX = 40, 50
    assert s.shape == (NZ, NX)
    assert np.all(s[10:30, 10:40] == 1.0)
    assert s[0, 25] == pytest.approx(math.exp(-(0.015 * 10) ** 2))
    assert s[0, 0] == pytest.approx(math.exp(-(0.015 * 10) ** 2) ** 2)
    assert np.allclose(s, s[::-1, :]) and np.allclose(s, s[:, ::-1])
    # monotone towards the outer edge
    assert np.all(np.diff(s[25, :10]) > 0)
