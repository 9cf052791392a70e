"""FP64 CPU oracle of the RTM path — TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the CPU-baseline / reference leg of the
benchmark use this package.  The library never imports it and it imports
nothing from the library: both sides receive the same generated input arrays
(numpy, float64 here; the CUDA side gets them rounded to float32 by the
caller).

The wave-propagation part is plain C (``rtm_oracle.c``), compiled with gcc on
first use (``build()``); the statistics part is numpy (``stats.py``).  Paper
references: "A workflow for seismic imaging with quantified uncertainty"
(arXiv 2001.06444) — §2.2 (Eqs. 4, 5), §2.3 (Eqs. 6, 7), §3.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

from .stats import ensemble_stats, uncertainty_maps  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "rtm_oracle.c"), os.path.join(_HERE, "codec_oracle.c"),
         os.path.join(_HERE, "eikonal_oracle.c")]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


class Grid(C.Structure):
    """Mirror of the oracle's grid struct: physical nx, nz; sponge nb;
    spacings dx, dz (m); time step dt (s); number of updates nt."""

    _fields_ = [("nx", C.c_int), ("nz", C.c_int), ("nb", C.c_int),
                ("dx", C.c_double), ("dz", C.c_double), ("dt", C.c_double),
                ("nt", C.c_int)]


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/_build/liboracle.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-fno-fast-math", "-ffp-contract=off", *_SRCS, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            g = C.POINTER(Grid)
            L.oracle_model.argtypes = [g, dp, C.c_int, C.c_int, C.c_int, ip, ip, dp, dp]
            L.oracle_adjoint_at_source.argtypes = [g, dp, C.c_int, C.c_int, C.c_int, ip, ip, dp, dp]
            L.oracle_migrate.argtypes = [g, dp, C.c_int, ip, ip, C.c_int, ip, ip, dp, dp,
                                         C.c_int, C.c_int, C.c_double, C.c_int, dp, dp, dp]
            L.oracle_born.argtypes = [g, dp, C.c_int, C.c_int, C.c_int, ip, ip, dp, C.c_int, dp, dp]
            L.oracle_laplacian8.argtypes = [dp, C.c_int, C.c_int, C.c_double, C.c_double, dp]
            L.oracle_laplacian8.restype = None
            L.oracle_image_filter.argtypes = [dp, C.c_int, C.c_int, C.c_double, C.c_double, dp]
            L.oracle_image_filter.restype = None
            L.oracle_round_format.argtypes = [C.c_double, C.c_int, C.c_int]
            L.oracle_round_format.restype = C.c_double
            L.oracle_quantize_snapshot.argtypes = [dp, C.c_long, C.c_int, dp]
            L.oracle_quantize_snapshot.restype = None
            L.oracle_courant.argtypes = [C.c_double] * 4
            L.oracle_courant.restype = C.c_double
            L.oracle_sponge.argtypes = [g, dp]
            L.oracle_threads.restype = C.c_int
            L.oracle_codec_kmin.argtypes = [C.c_double, C.c_int]
            L.oracle_codec_transform.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            L.oracle_codec_transform.restype = None
            L.oracle_codec_bound.argtypes = [C.c_int64, C.c_int64]
            L.oracle_codec_bound.restype = C.c_uint64
            L.oracle_codec_compress.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_double,
                                                C.c_void_p, C.c_uint64]
            L.oracle_codec_compress.restype = C.c_uint64
            L.oracle_codec_decompress.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p, C.c_int64,
                                                  C.c_int64]
            L.oracle_set_threads.argtypes = [C.c_int]
            L.oracle_set_threads.restype = None
            L.oracle_eikonal_update.argtypes = [C.c_double] * 5
            L.oracle_eikonal_update.restype = C.c_double
            L.oracle_eikonal.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_void_p,
                                         C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
            _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int))


def grid(nx, nz, nb, dx, dz, dt, nt) -> Grid:
    return Grid(int(nx), int(nz), int(nb), float(dx), float(dz), float(dt), int(nt))


def model(g: Grid, vel, src_ix, src_iz, rec_ix, rec_iz, wavelet):
    """Seismogram [nt][nrec] of one shot: d[n][r] = u^{n+1}(receiver r)."""
    vel, pv = _d(vel)
    rx, prx = _i(rec_ix)
    rz, prz = _i(rec_iz)
    w, pw = _d(wavelet)
    out = np.zeros((g.nt, rx.size), np.float64)
    rc = lib().oracle_model(C.byref(g), pv, int(src_ix), int(src_iz), rx.size, prx, prz, pw,
                            out.ctypes.data_as(C.POINTER(C.c_double)))
    if rc:
        raise MemoryError("oracle_model failed")
    return out


def adjoint_at_source(g: Grid, vel, src_ix, src_iz, rec_ix, rec_iz, seis):
    """Transpose of ``model`` with respect to the wavelet samples."""
    vel, pv = _d(vel)
    rx, prx = _i(rec_ix)
    rz, prz = _i(rec_iz)
    s, ps = _d(seis)
    out = np.zeros(g.nt, np.float64)
    rc = lib().oracle_adjoint_at_source(C.byref(g), pv, int(src_ix), int(src_iz), rx.size,
                                        prx, prz, ps, out.ctypes.data_as(C.POINTER(C.c_double)))
    if rc:
        raise MemoryError("oracle_adjoint_at_source failed")
    return out


def migrate(g: Grid, vel, src_ix, src_iz, rec_ix, rec_iz, wavelet, seis, isnap=1,
            snap_mode=0, eps=1e-6, laplacian=True, return_parts=False):
    """RTM image [nz][nx] of all shots; optionally also per-shot num, den."""
    vel, pv = _d(vel)
    sx, psx = _i(np.atleast_1d(src_ix))
    sz, psz = _i(np.atleast_1d(src_iz))
    rx, prx = _i(rec_ix)
    rz, prz = _i(rec_iz)
    w, pw = _d(wavelet)
    s, ps = _d(seis)
    ns = sx.size
    assert s.size == ns * g.nt * rx.size
    img = np.zeros((g.nz, g.nx), np.float64)
    dpn = C.POINTER(C.c_double)
    num = den = None
    pn = pd = None
    if return_parts:
        num = np.zeros((ns, g.nz, g.nx), np.float64)
        den = np.zeros((ns, g.nz, g.nx), np.float64)
        pn = num.ctypes.data_as(dpn)
        pd = den.ctypes.data_as(dpn)
    rc = lib().oracle_migrate(C.byref(g), pv, ns, psx, psz, rx.size, prx, prz, pw, ps,
                              int(isnap), int(snap_mode), float(eps), int(bool(laplacian)),
                              img.ctypes.data_as(dpn), pn, pd)
    if rc:
        raise MemoryError(f"oracle_migrate failed ({rc})")
    return (img, num, den) if return_parts else img


def born(g: Grid, vel, src_ix, src_iz, rec_ix, rec_iz, wavelet, isnap, refl):
    """Linearised data of reflectivity ``refl`` [nz][nx] for one shot."""
    vel, pv = _d(vel)
    rx, prx = _i(rec_ix)
    rz, prz = _i(rec_iz)
    w, pw = _d(wavelet)
    m, pm = _d(refl)
    out = np.zeros((g.nt, rx.size), np.float64)
    rc = lib().oracle_born(C.byref(g), pv, int(src_ix), int(src_iz), rx.size, prx, prz, pw,
                           int(isnap), pm, out.ctypes.data_as(C.POINTER(C.c_double)))
    if rc:
        raise MemoryError("oracle_born failed")
    return out


def laplacian8(a, dz, dx):
    a, pa = _d(a)
    out = np.zeros_like(a)
    lib().oracle_laplacian8(pa, a.shape[0], a.shape[1], float(dz), float(dx),
                            out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def image_filter(img, dz, dx):
    img, pi = _d(img)
    out = np.zeros_like(img)
    lib().oracle_image_filter(pi, img.shape[0], img.shape[1], float(dz), float(dx),
                              out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def round_format(y, p, emin):
    return lib().oracle_round_format(float(y), int(p), int(emin))


def quantize_snapshot(S, mode):
    S, ps = _d(S)
    out = np.zeros_like(S)
    lib().oracle_quantize_snapshot(ps, S.size, int(mode), out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def courant(vmax, dt, dx, dz):
    return lib().oracle_courant(float(vmax), float(dt), float(dx), float(dz))


def sponge(g: Grid):
    out = np.zeros((g.nz + 2 * g.nb, g.nx + 2 * g.nb), np.float64)
    lib().oracle_sponge(C.byref(g), out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def threads() -> int:
    """Threads the oracle's OpenMP loops use."""
    return int(lib().oracle_threads())


def set_threads(n: int) -> None:
    """Set the threads of the oracle's OpenMP loops."""
    lib().oracle_set_threads(int(n))


# ---------------------------------------------------------------- codec --

def codec_kmin(tol, e) -> int:
    """Lowest bit plane the codec keeps for tolerance tol, block exponent e."""
    return int(lib().oracle_codec_kmin(float(tol), int(e)))


def codec_transform(block):
    """(forward, forward-then-inverse) integer transform of a 4 x 4 integer block."""
    q = np.ascontiguousarray(np.asarray(block, np.int64).reshape(16))
    f = np.zeros(16, np.int64)
    b = np.zeros(16, np.int64)
    lib().oracle_codec_transform(q.ctypes.data, f.ctypes.data, b.ctypes.data)
    return f.reshape(4, 4), b.reshape(4, 4)


def codec_bound(n0, n1) -> int:
    """Upper bound of the stream size in bytes of an n0 x n1 array."""
    return int(lib().oracle_codec_bound(int(n0), int(n1)))


def codec_compress(data, tol) -> bytes:
    """Compressed stream of a 2D float32 array: absolute tolerance tol > 0,
    or lossless with tol == 0."""
    a = np.ascontiguousarray(np.asarray(data, np.float32))
    n0, n1 = a.shape
    cap = int(lib().oracle_codec_bound(n0, n1))
    out = np.zeros(cap, np.uint8)
    n = int(lib().oracle_codec_compress(a.ctypes.data, n0, n1, float(tol), out.ctypes.data, cap))
    if n == 0:
        raise ValueError("bad codec arguments (or a non-finite value with tol > 0)")
    return out[:n].tobytes()


def codec_decompress(blob: bytes, n0, n1):
    buf = np.frombuffer(blob, np.uint8).copy()
    out = np.zeros((n0, n1), np.float32)
    rc = lib().oracle_codec_decompress(buf.ctypes.data, buf.size, out.ctypes.data, int(n0), int(n1))
    if rc:
        raise ValueError(f"corrupt stream ({rc})")
    return out


# -------------------------------------------------------------- eikonal --

def eikonal_update(a, b, s, dz, dx) -> float:
    """Upwind update of one node from its smaller vertical (a) and horizontal
    (b) neighbour times."""
    return float(lib().oracle_eikonal_update(float(a), float(b), float(s), float(dz), float(dx)))


def eikonal(vel, dz, dx, src_iz, src_ix):
    """First-arrival traveltimes [nz][nx] (FP64, fast marching) for velocity
    vel [nz][nx] from the source nodes (src_iz[k], src_ix[k]), all at T = 0."""
    v = np.ascontiguousarray(np.asarray(vel, np.float64))
    nz, nx = v.shape
    s = np.ascontiguousarray(1.0 / v)
    iz, _ = _i(np.atleast_1d(src_iz))
    ix, _ = _i(np.atleast_1d(src_ix))
    T = np.empty((nz, nx))
    rc = lib().oracle_eikonal(nz, nx, float(dz), float(dx), s.ctypes.data, iz.size,
                              iz.ctypes.data, ix.ctypes.data, T.ctypes.data)
    if rc:
        raise ValueError("bad eikonal arguments")
    return T
