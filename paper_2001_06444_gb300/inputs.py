"""Seeded synthetic inputs for the RTM path: velocity models, velocity
ensembles, wavelets, acquisition geometries and request streams.

This module holds no step of the method itself; it only makes input arrays.
The tests feed the same arrays to the CUDA library and to the FP64 oracle.
Every random draw comes from SplitMix64 (Steele, Lea & Flood 2014) used as a
counter-based generator, so a (seed, index) pair fixes each number on any
machine and numpy version.

The workloads stand in for those of the paper's experiments (§4.1 two-layer
model; §4.2 / §4.4 Marmousi2, which is not reproduced here): a flat two-layer
reflector, and a layered, faulted, dipping model with a water layer and a
high-velocity body, perturbed by smooth Gaussian random fields to form the
velocity ensemble that stage 1 of the workflow (§3) would provide.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MODEL_SEED = 2001064
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+n-1 of SplitMix64 started at state `seed`."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1): the top 53 bits of each SplitMix64 output."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normal deviates by Box-Muller on consecutive uniform pairs."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))  # 1 - u1 in (0, 1]
    th = 2.0 * np.pi * u2
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(th)
    z[1::2] = r * np.sin(th)
    return z[:n]


def ricker(f: float, dt: float, nt: int, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet of peak frequency f sampled at t = n dt, n = 0..nt-1,
    delayed by t0 = 1/f, unit peak amplitude."""
    t0 = 1.0 / f if t0 is None else t0
    t = np.arange(nt) * dt - t0
    a = (np.pi * f * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def two_layer(nz: int, nx: int, dz: float, z_interface: float, v_top: float,
              v_bottom: float) -> np.ndarray:
    """Flat reflector: v_top for z < z_interface, v_bottom below (z = iz dz)."""
    z = np.arange(nz) * dz
    v = np.where(z < z_interface - 1e-9, v_top, v_bottom)
    return np.repeat(v[:, None], nx, axis=1).astype(np.float64)


def layered_faulted(nz: int, nx: int, dx: float, dz: float, seed: int = MODEL_SEED,
                    water_depth: float = 450.0, n_layers: int = 12,
                    v_layers=(1600.0, 3500.0), v_basement: float = 4700.0,
                    n_faults: int = 3, throw=(50.0, 200.0), max_dip_deg: float = 15.0,
                    v_body: float = 4500.0) -> np.ndarray:
    """Layered, faulted sedimentary model under a water layer.

    Water (1500 m/s) above `water_depth`; n_layers dipping layers with
    velocities increasing linearly over v_layers; a basement half-space of
    v_basement below the last interface; n_faults normal faults with random
    throws in `throw` (m) that drop the hanging wall; an elliptical body of
    v_body.  Velocity never decreases with depth inside the layered part
    because the layer index at a point counts the interfaces above it.
    """
    u = iter(uniform(seed, 64))
    zz = (np.arange(nz) * dz)[:, None] * np.ones((1, nx))
    xx = np.ones((nz, 1)) * (np.arange(nx) * dx)[None, :]
    width, depth = (nx - 1) * dx, (nz - 1) * dz
    xc = 0.5 * width
    # normal faults: plane x_f(z) = x0 + (z - water) / tan(phi); hanging wall
    # (x beyond the plane) is dropped by the throw, so structure there is read
    # from z - throw.
    shift = np.zeros_like(zz)
    for _ in range(n_faults):
        x0 = (0.15 + 0.7 * next(u)) * width
        phi = math.radians(55.0 + 15.0 * next(u))
        t = throw[0] + (throw[1] - throw[0]) * next(u)
        plane = x0 + (zz - water_depth) / math.tan(phi)
        shift += np.where(xx > plane, t, 0.0)
    zs = zz - shift
    # dipping interfaces, evenly spaced at the centre column
    z_base = water_depth + 0.85 * (depth - water_depth)
    count = np.zeros((nz, nx), np.int32)
    for k in range(1, n_layers + 1):
        z0 = water_depth + k * (z_base - water_depth) / n_layers
        dip = math.radians(max_dip_deg * (2.0 * next(u) - 1.0))
        zk = z0 + math.tan(dip) * (xx - xc)
        zk = np.clip(zk, water_depth + dz, depth)
        count += (zs >= zk).astype(np.int32)
    vl = np.linspace(v_layers[0], v_layers[1], n_layers)
    v = np.where(count >= n_layers, v_basement, vl[np.minimum(count, n_layers - 1)])
    # elliptical high-velocity body in the middle of the section
    bx = (0.3 + 0.4 * next(u)) * width
    bz = water_depth + (0.35 + 0.3 * next(u)) * (depth - water_depth)
    ax = 600.0 + 600.0 * next(u)
    az = 150.0 + 150.0 * next(u)
    body = ((xx - bx) / ax) ** 2 + ((zz - bz) / az) ** 2 <= 1.0
    v = np.where(body, v_body, v)
    v = np.where(zz < water_depth - 1e-9, 1500.0, v)
    return v.astype(np.float64)


def gaussian_random_field(nz: int, nx: int, dx: float, dz: float, seed: int,
                          corr_len: float = 300.0) -> np.ndarray:
    """White N(0,1) smoothed by a Gaussian kernel of std corr_len / 2, which
    gives a correlation exp(-r^2 / corr_len^2).  Unit-free, unnormalised."""
    from scipy.ndimage import gaussian_filter

    white = normal(seed, nz * nx).reshape(nz, nx)
    sig = 0.5 * corr_len
    return gaussian_filter(white, sigma=(sig / dz, sig / dx), mode="reflect", truncate=4.0)


def perturb(v: np.ndarray, dx: float, dz: float, seed: int, corr_len: float = 300.0,
            rel_std: float = 0.04, water_depth: float = 450.0,
            v_clip: float = 5400.0) -> np.ndarray:
    """One velocity sample: v (1 + field), the field scaled to an empirical
    std of rel_std over the cells below the water layer, the water fixed and
    the result clipped to v_clip (keeps every sample inside the CFL bound)."""
    nz, nx = v.shape
    fld = gaussian_random_field(nz, nx, dx, dz, seed, corr_len)
    wet = (np.arange(nz) * dz < water_depth - 1e-9)[:, None] * np.ones((1, nx), bool)
    dry = ~wet
    f = fld - fld[dry].mean()
    f *= rel_std / f[dry].std()
    out = np.where(dry, v * (1.0 + f), v)
    return np.minimum(out, v_clip)


def ensemble(v: np.ndarray, dx: float, dz: float, n: int, base_seed: int = MODEL_SEED,
             **kw) -> np.ndarray:
    """n velocity samples; sample i uses seed base_seed + 1000 + i."""
    return np.stack([perturb(v, dx, dz, base_seed + 1000 + i, **kw) for i in range(n)])


def smooth(v: np.ndarray, dx: float, dz: float, length: float) -> np.ndarray:
    """Gaussian-smoothed copy of v (std `length` metres), e.g. a migration
    velocity as in §4.1."""
    from scipy.ndimage import gaussian_filter

    return gaussian_filter(v, sigma=(length / dz, length / dx), mode="nearest")


def metres_to_index(x: float, d: float) -> int:
    """Nearest grid index of a position: floor(x / d + 0.5)."""
    return int(math.floor(x / d + 0.5))


@dataclass
class Survey:
    """A complete synthetic problem: grid, velocity, acquisition, wavelet."""

    nx: int
    nz: int
    nb: int
    dx: float
    dz: float
    dt: float
    nt: int
    vel: np.ndarray
    src_ix: np.ndarray
    src_iz: np.ndarray
    rec_ix: np.ndarray
    rec_iz: np.ndarray
    wavelet: np.ndarray
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def nshot(self) -> int:
        return int(self.src_ix.size)

    @property
    def nrec(self) -> int:
        return int(self.rec_ix.size)

    def grid_tuple(self):
        return (self.nx, self.nz, self.nb, self.dx, self.dz, self.dt, self.nt)


def flat_reflector(nt: int = 1000) -> Survey:
    """201 x 101 cells at 10 m; 1500 m/s above a flat reflector at 500 m,
    2500 m/s below; 20-cell sponge; 15 Hz Ricker at (1000 m, 20 m); 201
    receivers at 20 m depth; dt = 1 ms."""
    nx, nz, d = 201, 101, 10.0
    v = two_layer(nz, nx, d, 500.0, 1500.0, 2500.0)
    return Survey(nx, nz, 20, d, d, 1e-3, nt, v,
                  np.array([metres_to_index(1000.0, d)], np.int32),
                  np.array([metres_to_index(20.0, d)], np.int32),
                  np.arange(nx, dtype=np.int32),
                  np.full(nx, metres_to_index(20.0, d), np.int32),
                  ricker(15.0, 1e-3, nt), name="flat_reflector_201x101")


def full_size(nshot: int = 96, nt: int = 5000, seed: int = MODEL_SEED) -> Survey:
    """1701 x 351 cells at 10 m, layered/faulted model, 96 shots every 170 m
    from 430 m at 10 m depth, 1701 receivers at 10 m depth, 10 Hz Ricker,
    dt = 1 ms, 5000 steps."""
    nx, nz, d = 1701, 351, 10.0
    v = layered_faulted(nz, nx, d, d, seed)
    xs = 430.0 + 170.0 * np.arange(nshot)
    return Survey(nx, nz, 20, d, d, 1e-3, nt, v,
                  np.array([metres_to_index(x, d) for x in xs], np.int32),
                  np.full(nshot, metres_to_index(10.0, d), np.int32),
                  np.arange(nx, dtype=np.int32),
                  np.full(nx, metres_to_index(10.0, d), np.int32),
                  ricker(10.0, 1e-3, nt), name="layered_faulted_1701x351")


def scaled_survey(nx: int, nz: int, nshot: int, nt: int, f: float, seed: int,
                  d: float = 10.0, nb: int = 20, dt: float = 1e-3) -> Survey:
    """A layered/faulted survey of any size: shots spread evenly over the
    surface at 10 m depth, receivers at every cell at 10 m depth."""
    v = layered_faulted(nz, nx, d, d, seed)
    if nshot == 1:
        xs = np.array([0.5 * (nx - 1) * d])
    else:
        xs = np.linspace(0.05, 0.95, nshot) * (nx - 1) * d
    return Survey(nx, nz, nb, d, d, dt, nt, v,
                  np.array([metres_to_index(x, d) for x in xs], np.int32),
                  np.full(nshot, 1, np.int32),
                  np.arange(nx, dtype=np.int32),
                  np.full(nx, 1, np.int32),
                  ricker(f, dt, nt), name=f"layered_{nx}x{nz}")


MIXED_GRIDS = ((201, 101), (851, 176), (1701, 351), (2401, 601))


def request_stream(n: int = 256, rate_hz: float = 1.0, seed: int = 7,
                   grids=MIXED_GRIDS, shots=(1, 32), freqs=(10.0, 15.0),
                   steps=(2000, 6000)):
    """Poisson arrivals of migration requests: each entry is a dict with the
    arrival time (s), grid (nx, nz), shot count, Ricker frequency and nt,
    drawn uniformly from the given ranges."""
    u = uniform(seed, 5 * n).reshape(n, 5)
    t = np.cumsum(-np.log1p(-u[:, 0]) / rate_hz)
    out = []
    for i in range(n):
        g = grids[min(int(u[i, 1] * len(grids)), len(grids) - 1)]
        out.append(dict(t=float(t[i]), nx=g[0], nz=g[1],
                        nshot=shots[0] + min(int(u[i, 2] * (shots[1] - shots[0] + 1)),
                                             shots[1] - shots[0]),
                        f=freqs[0] + (freqs[1] - freqs[0]) * float(u[i, 3]),
                        nt=steps[0] + int(u[i, 4] * (steps[1] - steps[0])),
                        seed=MODEL_SEED + 5000 + i))
    return out
