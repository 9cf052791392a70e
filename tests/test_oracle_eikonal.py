"""Pins of the traveltime oracle (first-arrival eikonal solver of the
tomography stage, §2.1 Eq. 1 and §3; first-order upwind scheme solved by fast
marching):

- the local update solves its defining equation, and its two branches give
  the hand-derived values (one-sided: u + s h; two-sided on a square cell:
  (1 + 1/sqrt 2) h s next to a source);
- constant velocity: exact times along the grid axes, and the scheme's
  bounds r/v <= T <= (|di| dz + |dj| dx)/v;
- a plane wave from a line source through a layered model: T is the running
  sum of dz s, exactly;
- tiny grids: equal to Gauss-Seidel sweeping iterated to its fixed point,
  with each local quadratic solved by bisection on its defining equation;
- refinement: the error at a fixed point falls as the grid is refined.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2001_06444_gb300 import inputs


def _solve_local_bisect(a, b, s, dz, dx):
    """The root T >= min(a, b) of ((T-a)^+/dz)^2 + ((T-b)^+/dx)^2 = s^2."""
    if math.isinf(a) and math.isinf(b):
        return math.inf
    lo = min(a, b)
    hi = lo + s * max(dz, dx) + 1.0
    f = lambda t: (max(t - a, 0.0) / dz) ** 2 + (max(t - b, 0.0) / dx) ** 2 - s * s
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def test_local_update_solves_its_equation():
    u = inputs.uniform(12, 4000)
    for k in range(1000):
        a, b = u[4 * k] * 3.0, u[4 * k + 1] * 3.0
        s = 0.2 + u[4 * k + 2]
        dz, dx = 1.0 + u[4 * k + 3], 1.0 + 0.5 * u[4 * k + 2]
        t = oracle.eikonal_update(a, b, s, dz, dx)
        assert t >= min(a, b)
        res = (max(t - a, 0) / dz) ** 2 + (max(t - b, 0) / dx) ** 2 - s * s
        assert abs(res) <= 1e-12 * s * s
        assert t == pytest.approx(_solve_local_bisect(a, b, s, dz, dx), rel=1e-12, abs=1e-12)
    assert oracle.eikonal_update(2.0, math.inf, 0.5, 10.0, 3.0) == 2.0 + 5.0  # one-sided
    assert oracle.eikonal_update(math.inf, math.inf, 0.5, 1.0, 1.0) == math.inf
    # next to a source on a square cell: both neighbours at h s
    h, s = 10.0, 1.0 / 2000.0
    t = oracle.eikonal_update(h * s, h * s, s, h, h)
    assert t == pytest.approx((1 + 1 / math.sqrt(2)) * h * s, rel=1e-15)


def test_constant_velocity_axes_and_bounds():
    v, dz, dx = 2500.0, 10.0, 15.0
    nz, nx, iz, ix = 31, 40, 7, 25
    T = oracle.eikonal(np.full((nz, nx), v), dz, dx, iz, ix)
    zz, xx = np.meshgrid((np.arange(nz) - iz) * dz, (np.arange(nx) - ix) * dx, indexing="ij")
    # along an axis every update is one-sided: the running sum of h s, exactly
    sx, sz = np.cumsum(np.full(nx, dx * (1.0 / v))), np.cumsum(np.full(nz, dz * (1.0 / v)))
    assert np.array_equal(T[iz, ix + 1:], sx[:nx - ix - 1])
    assert np.array_equal(T[iz, ix - 1::-1], sx[:ix])
    assert np.array_equal(T[iz + 1:, ix], sz[:nz - iz - 1])
    assert np.array_equal(T[iz - 1::-1, ix], sz[:iz])
    assert np.allclose(T[iz, :], np.abs(xx[iz, :]) / v, rtol=1e-14, atol=0)
    r = np.hypot(zz, xx) / v
    assert np.all(T >= r * (1 - 1e-14))
    assert np.all(T <= (np.abs(zz) + np.abs(xx)) / v * (1 + 1e-14))
    assert T[iz, ix] == 0.0


def test_plane_wave_through_layers_is_a_running_sum():
    nz, nx, dz, dx = 40, 23, 12.0, 9.0
    vz = 1500.0 + 3000.0 * inputs.uniform(5, nz)
    vel = np.repeat(vz[:, None], nx, axis=1)
    T = oracle.eikonal(vel, dz, dx, np.zeros(nx, np.int32), np.arange(nx, dtype=np.int32))
    s = 1.0 / vz
    want = np.concatenate([[0.0], np.cumsum(dz * s[1:])])
    assert np.array_equal(T, np.repeat(want[:, None], nx, axis=1))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_tiny_grids_equal_sweeping_to_the_fixed_point(seed):
    nz, nx = 7, 9
    u = inputs.uniform(seed, nz * nx + 2)
    vel = (1500.0 + 3000.0 * u[:nz * nx]).reshape(nz, nx)
    dz, dx = 10.0, 10.0 + 5.0 * seed
    iz, ix = int(u[-2] * nz), int(u[-1] * nx)
    T = oracle.eikonal(vel, dz, dx, iz, ix)
    s = 1.0 / vel
    W = np.full((nz, nx), math.inf)
    W[iz, ix] = 0.0
    orders = [(range(nz), range(nx)), (range(nz - 1, -1, -1), range(nx)),
              (range(nz - 1, -1, -1), range(nx - 1, -1, -1)), (range(nz), range(nx - 1, -1, -1))]
    for _ in range(50):
        changed = False
        for rows, cols in orders:
            for i in rows:
                for j in cols:
                    if (i, j) == (iz, ix):
                        continue
                    a = min(W[i - 1, j] if i > 0 else math.inf, W[i + 1, j] if i < nz - 1 else math.inf)
                    b = min(W[i, j - 1] if j > 0 else math.inf, W[i, j + 1] if j < nx - 1 else math.inf)
                    t = _solve_local_bisect(a, b, s[i, j], dz, dx)
                    if t < W[i, j] * (1 - 1e-13):
                        W[i, j] = t
                        changed = True
        if not changed:
            break
    assert not changed
    assert np.allclose(T, W, rtol=1e-11, atol=0)


def test_error_falls_under_refinement():
    v = 3000.0
    errs = []
    for h in (40.0, 20.0, 10.0, 5.0):
        n = int(round(800.0 / h)) + 1
        T = oracle.eikonal(np.full((n, n), v), h, h, 0, 0)
        i = int(round(600.0 / h))
        j = int(round(400.0 / h))
        errs.append(T[i, j] - math.hypot(600.0, 400.0) / v)
    assert all(e > 0 for e in errs)
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 0.6 * errs[1]
