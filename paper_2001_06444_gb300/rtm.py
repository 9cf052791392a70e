"""Thin ctypes binding of the C ABI in ``include/rtm.h``.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays; CUDA
tensors are passed in place on the current torch stream, host arrays are
staged by the library.  If the library is missing it is built with nvcc; if
that is impossible the call raises — there is no other implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

RTM_OK, RTM_ERR_ARG, RTM_ERR_CFL, RTM_ERR_NOMEM = 0, 1, 2, 3
RTM_ERR_BUSY, RTM_ERR_TIMEOUT, RTM_ERR_CUDA, RTM_ERR_STATE = 4, 5, 6, 7
EIK_OFFCHIP, EIK_SHARED = 1, 2
SNAP_F32, SNAP_BF16, SNAP_F16 = 0, 1, 2
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3
_NAMES = {0: "RTM_OK", 1: "RTM_ERR_ARG", 2: "RTM_ERR_CFL", 3: "RTM_ERR_NOMEM",
          4: "RTM_ERR_BUSY", 5: "RTM_ERR_TIMEOUT", 6: "RTM_ERR_CUDA", 7: "RTM_ERR_STATE"}

# every entry point the header declares
EXPORTS = ("rtm_ctx_create", "rtm_ctx_destroy", "rtm_ctx_set_batch", "rtm_ctx_set_profiling",
           "rtm_ctx_stats", "rtm_plan_bytes", "rtm_autotune", "rtm_model", "rtm_migrate",
           "rtm_migrate_ensemble", "rtm_born", "rtm_migrate_adjoint", "rtm_lsrtm",
           "rtm_ensemble_stats",
           "rtm_uncertainty_maps",
           "rtm_submit", "rtm_poll", "rtm_model_noalloc", "rtm_selftest_wait",
           "rtm_ctx_inject_wait_timeout", "rtm_compress_bound",
           "rtm_compress", "rtm_decompress", "rtm_eikonal", "rtm_last_error", "rtm_cfl_limit")


class RTMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("nz", C.c_int), ("nb", C.c_int), ("dx", C.c_double),
                ("dz", C.c_double), ("dt", C.c_double), ("nt", C.c_int)]


class Acq(C.Structure):
    _fields_ = [("nshot", C.c_int), ("src_ix", C.POINTER(C.c_int)), ("src_iz", C.POINTER(C.c_int)),
                ("nrec", C.c_int), ("rec_ix", C.POINTER(C.c_int)), ("rec_iz", C.POINTER(C.c_int)),
                ("wavelet", C.POINTER(C.c_float))]


class Opts(C.Structure):
    """isnap, snap_dtype, eps, laplacian, checkpoint (0 = keep every snapshot,
    C > 0 = keep the state every C steps and recompute, -1 = least memory)."""

    _fields_ = [("isnap", C.c_int), ("snap_dtype", C.c_int), ("eps", C.c_double),
                ("laplacian", C.c_int), ("checkpoint", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("step_launches", C.c_longlong), ("step_ms", C.c_double),
                ("step_bytes", C.c_double), ("point_updates", C.c_double),
                ("launches", C.c_longlong), ("migrations", C.c_longlong),
                ("codec_launches", C.c_longlong), ("codec_ms", C.c_double),
                ("codec_bytes", C.c_double), ("eik_launches", C.c_longlong),
                ("eik_ms", C.c_double), ("eik_updates", C.c_double),
                ("graph_launches", C.c_longlong), ("requests_peak_running", C.c_longlong),
                ("requests_backfilled", C.c_longlong)]


class Request(C.Structure):
    _fields_ = [("grid", Grid), ("vel", C.c_void_p), ("acq", Acq), ("seis", C.c_void_p),
                ("opts", Opts), ("image", C.c_void_p)]


_lib = None
_lock = threading.Lock()


def lib():
    """The loaded CUDA library (built on first use).  With RTM_DEBUG=1 in the
    environment, the bounds-checked build instead."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build(debug=os.environ.get("RTM_DEBUG") == "1")
            L = C.CDLL(path)
            vp, ip = C.c_void_p, C.c_int
            L.rtm_ctx_create.argtypes = [C.POINTER(vp), ip, C.c_size_t]
            L.rtm_ctx_destroy.argtypes = [vp]
            L.rtm_ctx_set_batch.argtypes = [vp, ip]
            L.rtm_ctx_set_profiling.argtypes = [vp, ip]
            L.rtm_ctx_stats.argtypes = [vp, C.POINTER(Stats), ip]
            L.rtm_model.argtypes = [vp, C.POINTER(Grid), vp, C.POINTER(Acq), ip, vp, vp]
            L.rtm_migrate.argtypes = [vp, C.POINTER(Grid), vp, C.POINTER(Acq), vp, C.POINTER(Opts),
                                      vp, vp]
            L.rtm_migrate_ensemble.argtypes = [vp, C.POINTER(Grid), ip, vp, C.POINTER(Acq), vp,
                                               C.POINTER(Opts), vp, vp]
            L.rtm_born.argtypes = [vp, C.POINTER(Grid), vp, C.POINTER(Acq), vp, C.POINTER(Opts), vp,
                                   vp]
            L.rtm_migrate_adjoint.argtypes = [vp, C.POINTER(Grid), vp, C.POINTER(Acq), vp,
                                              C.POINTER(Opts), vp, vp]
            L.rtm_lsrtm.argtypes = [vp, C.POINTER(Grid), vp, C.POINTER(Acq), vp, C.POINTER(Opts),
                                    ip, vp, C.POINTER(C.c_double), vp]
            L.rtm_ensemble_stats.argtypes = [vp, vp, ip, C.c_long, vp, vp, vp, vp, vp]
            L.rtm_uncertainty_maps.argtypes = [vp, vp, vp, C.c_long, vp, vp, vp]
            L.rtm_submit.argtypes = [vp, C.POINTER(Request), C.POINTER(C.c_uint64)]
            L.rtm_poll.argtypes = [vp, C.c_uint64, C.POINTER(ip), ip]
            L.rtm_last_error.argtypes = [vp]
            L.rtm_last_error.restype = C.c_char_p
            L.rtm_cfl_limit.restype = C.c_double
            L.rtm_autotune.argtypes = [vp, C.POINTER(Grid), C.POINTER(Acq), C.POINTER(Opts), ip,
                                       C.POINTER(C.c_int), vp]
            L.rtm_selftest_wait.argtypes = [vp, ip, C.POINTER(ip), vp]
            L.rtm_ctx_inject_wait_timeout.argtypes = [vp, ip]
            L.rtm_model_noalloc.argtypes = [C.POINTER(Grid), vp, C.POINTER(Acq), ip, vp, vp]
            ll, u64 = C.c_longlong, C.c_uint64
            L.rtm_compress_bound.argtypes = [ll, ll]
            L.rtm_compress_bound.restype = u64
            L.rtm_compress.argtypes = [vp, vp, ll, ll, ll, C.c_double, vp, u64,
                                       C.POINTER(u64), vp]
            L.rtm_decompress.argtypes = [vp, vp, u64, ll, ll, ll, vp, vp]
            L.rtm_eikonal.argtypes = [vp, ip, ip, C.c_double, C.c_double, ip, vp, ip, vp, vp, ip,
                                      vp, vp, ip, ip, vp, vp, vp, vp]
            L.rtm_plan_bytes.argtypes = [C.POINTER(Grid), C.POINTER(Acq), C.POINTER(Opts), ip,
                                         C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
            _lib = L
    return _lib


def cfl_limit() -> float:
    return lib().rtm_cfl_limit()


def plan_bytes(grid: Grid, acq: Acq, opts: Opts, nsample: int = 1):
    """(bytes per call, bytes per migration in flight) of a migration."""
    a, b = C.c_size_t(), C.c_size_t()
    rc = lib().rtm_plan_bytes(C.byref(grid), C.byref(acq), C.byref(opts), int(nsample),
                              C.byref(a), C.byref(b))
    if rc:
        raise RTMError(rc, "rtm_plan_bytes: bad arguments")
    return a.value, b.value


def make_grid(nx, nz, nb, dx, dz, dt, nt) -> Grid:
    return Grid(int(nx), int(nz), int(nb), float(dx), float(dz), float(dt), int(nt))


class _Keep:
    """Holds host copies alive for the duration of a call."""

    def __init__(self):
        self.items = []

    def i32(self, a):
        a = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
        self.items.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_int))

    def f32(self, a):
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
        self.items.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_float))


def make_acq(keep: _Keep, src_ix, src_iz, rec_ix, rec_iz, wavelet) -> Acq:
    src_ix = np.atleast_1d(src_ix)
    return Acq(int(src_ix.size), keep.i32(src_ix), keep.i32(np.atleast_1d(src_iz)),
               int(np.size(rec_ix)), keep.i32(rec_ix), keep.i32(rec_iz), keep.f32(wavelet))


def _ptr(a):
    """(pointer, is_cuda) of a torch tensor or numpy array (contiguous)."""
    try:
        import torch

        if isinstance(a, torch.Tensor):
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return a.data_ptr(), a.is_cuda
    except ImportError:  # pragma: no cover
        pass
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, False
    raise TypeError(f"unsupported array type {type(a)}")


def _check_dtype(a, want):
    dt = str(a.dtype).replace("torch.", "")
    if dt != want:
        raise TypeError(f"expected {want} array, got {dt}")


def _stream(*arrays):
    for a in arrays:
        if getattr(a, "is_cuda", False):
            import torch

            return C.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)
    return C.c_void_p(0)


def compress_bound(n0: int, n1: int) -> int:
    """Bytes one compressed n0 x n1 stream can take at most."""
    b = int(lib().rtm_compress_bound(int(n0), int(n1)))
    if not b:
        raise ValueError(f"unsupported shape {n0} x {n1}")
    return b


class Context:
    """An rtm_ctx on one CUDA device."""

    def __init__(self, device: int = 0, budget_bytes: int = 0):
        h = C.c_void_p()
        rc = lib().rtm_ctx_create(C.byref(h), int(device), C.c_size_t(int(budget_bytes)))
        if rc:
            raise RTMError(rc, f"rtm_ctx_create(device={device}) failed")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            lib().rtm_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc):
        if rc:
            raise RTMError(rc, lib().rtm_last_error(self.h).decode())

    def last_error(self) -> str:
        return lib().rtm_last_error(self.h).decode()

    def set_batch(self, max_items: int):
        self._check(lib().rtm_ctx_set_batch(self.h, int(max_items)))

    def set_profiling(self, on: bool):
        self._check(lib().rtm_ctx_set_profiling(self.h, int(bool(on))))

    def stats(self, reset: bool = False) -> dict:
        st = Stats()
        self._check(lib().rtm_ctx_stats(self.h, C.byref(st), int(bool(reset))))
        return {k: getattr(st, k) for k, _ in Stats._fields_}

    def autotune(self, grid: Grid, acq: Acq, opts: Opts, trial_steps: int = 64) -> dict:
        """Time the launch configurations on short synthetic trials and keep
        the fastest for this shape; returns it."""
        ch = (C.c_int * 5)()
        self._check(lib().rtm_autotune(self.h, C.byref(grid), C.byref(acq), C.byref(opts),
                                       int(trial_steps), ch, C.c_void_p(0)))
        return {"step_kernel": ch[0], "max_items": ch[1], "graph": ch[2], "tile_z": ch[3],
                "l2_ahead": ch[4]}

    def inject_wait_timeout(self, count: int = 1):
        """The next `count` migration or modelling calls start with their
        wait-timeout flag raised (test hook of the failure reporting)."""
        self._check(lib().rtm_ctx_inject_wait_timeout(self.h, int(count)))

    def selftest_wait(self, wait_ms: int = 200) -> bool:
        """Run the bounded device-side wait on a barrier nothing completes;
        True if its error flag reached the host."""
        r = C.c_int(0)
        self._check(lib().rtm_selftest_wait(self.h, int(wait_ms), C.byref(r), C.c_void_p(0)))
        return bool(r.value)

    def model(self, grid: Grid, vel, acq: Acq, shot: int, seis):
        _check_dtype(vel, "float32")
        _check_dtype(seis, "float32")
        pv, _ = _ptr(vel)
        ps, _ = _ptr(seis)
        self._check(lib().rtm_model(self.h, C.byref(grid), C.c_void_p(pv), C.byref(acq), int(shot),
                                    C.c_void_p(ps), _stream(vel, seis)))
        return seis

    def migrate(self, grid: Grid, vel, acq: Acq, seis, opts: Opts, image):
        for a in (vel, seis, image):
            _check_dtype(a, "float32")
        pv, _ = _ptr(vel)
        ps, _ = _ptr(seis)
        pi, _ = _ptr(image)
        self._check(lib().rtm_migrate(self.h, C.byref(grid), C.c_void_p(pv), C.byref(acq),
                                      C.c_void_p(ps), C.byref(opts), C.c_void_p(pi),
                                      _stream(vel, seis, image)))
        return image

    def migrate_ensemble(self, grid: Grid, vels, acq: Acq, seis, opts: Opts, images):
        for a in (vels, seis, images):
            _check_dtype(a, "float32")
        ns = int(vels.shape[0])
        pv, _ = _ptr(vels)
        ps, _ = _ptr(seis)
        pi, _ = _ptr(images)
        self._check(lib().rtm_migrate_ensemble(self.h, C.byref(grid), ns, C.c_void_p(pv),
                                               C.byref(acq), C.c_void_p(ps), C.byref(opts),
                                               C.c_void_p(pi), _stream(vels, seis, images)))
        return images

    def born(self, grid: Grid, vel, acq: Acq, refl, opts: Opts, seis):
        """Born modelling of every shot of acq: reflectivity refl [nz][nx] ->
        seis [nshot][nt][nrec] (float32, host or device)."""
        for a in (vel, refl, seis):
            _check_dtype(a, "float32")
        ptrs = [C.c_void_p(_ptr(a)[0]) for a in (vel, refl, seis)]
        self._check(lib().rtm_born(self.h, C.byref(grid), ptrs[0], C.byref(acq), ptrs[1],
                                   C.byref(opts), ptrs[2], _stream(vel, refl, seis)))
        return seis

    def migrate_adjoint(self, grid: Grid, vel, acq: Acq, seis, opts: Opts, image):
        """The adjoint of born: the stacked imaging numerator of seis
        [nshot][nt][nrec] into image [nz][nx] (float32, host or device)."""
        for a in (vel, seis, image):
            _check_dtype(a, "float32")
        ptrs = [C.c_void_p(_ptr(a)[0]) for a in (vel, seis, image)]
        self._check(lib().rtm_migrate_adjoint(self.h, C.byref(grid), ptrs[0], C.byref(acq), ptrs[1],
                                              C.byref(opts), ptrs[2], _stream(vel, seis, image)))
        return image

    def lsrtm(self, grid: Grid, vel, acq: Acq, seis, opts: Opts, niter: int, refl):
        """Least-squares migration (CGLS over born / migrate_adjoint): the
        reflectivity into refl [nz][nx]; returns the misfits
        ||d - B m_k||^2, k = 0..niter."""
        for a in (vel, seis, refl):
            _check_dtype(a, "float32")
        mis = (C.c_double * (int(niter) + 1))()
        ptrs = [C.c_void_p(_ptr(a)[0]) for a in (vel, seis, refl)]
        self._check(lib().rtm_lsrtm(self.h, C.byref(grid), ptrs[0], C.byref(acq), ptrs[1],
                                    C.byref(opts), int(niter), ptrs[2], mis,
                                    _stream(vel, seis, refl)))
        return list(mis)

    def ensemble_stats(self, images, mean, std, q05, q95):
        _check_dtype(images, "float32")
        n = int(images.shape[0])
        npix = int(np.prod(images.shape[1:]))
        ptrs = [C.c_void_p(_ptr(a)[0]) for a in (images, mean, std, q05, q95)]
        self._check(lib().rtm_ensemble_stats(self.h, ptrs[0], n, npix, *ptrs[1:],
                                             _stream(images, mean, std, q05, q95)))
        return mean, std, q05, q95

    def compress(self, data, tol: float, out=None, stride: int = 0):
        """Compress data [count][n0][n1] (or [n0][n1]) float32, host or
        device: absolute tolerance tol > 0, lossless with tol == 0.  Streams
        go to out (uint8, host or device, count * stride bytes; allocated on
        data's device when None) at a stride of compress_bound(n0, n1)
        rounded up to 16 unless given.  Returns (out, stride, byte counts)."""
        _check_dtype(data, "float32")
        shape = tuple(int(v) for v in data.shape)
        count, n0, n1 = (1, *shape) if len(shape) == 2 else shape
        if not stride:
            stride = (compress_bound(n0, n1) + 15) // 16 * 16
        if out is None:
            if getattr(data, "is_cuda", False):
                import torch

                out = torch.empty(count * stride, dtype=torch.uint8, device=data.device)
            else:
                out = np.empty(count * stride, np.uint8)
        sizes = (C.c_uint64 * count)()
        self._check(lib().rtm_compress(self.h, C.c_void_p(_ptr(data)[0]), count, n0, n1,
                                       float(tol), C.c_void_p(_ptr(out)[0]), int(stride), sizes,
                                       _stream(data, out)))
        return out, stride, [int(v) for v in sizes]

    def decompress(self, streams, stride: int, count: int, n0: int, n1: int, out):
        """Decompress count streams (uint8, host or device, at the given
        stride) into out [count][n0][n1] float32 (host or device)."""
        _check_dtype(out, "float32")
        self._check(lib().rtm_decompress(self.h, C.c_void_p(_ptr(streams)[0]), int(stride),
                                         int(count), int(n0), int(n1),
                                         C.c_void_p(_ptr(out)[0]), _stream(streams, out)))
        return out

    def eikonal(self, vel, dz: float, dx: float, src_iz, src_ix, rec_iz=None, rec_ix=None,
                times=None, fields=None, max_iter: int = 0, storage: str = "auto"):
        """First-arrival traveltimes for vel [nsample][nz][nx] (or [nz][nx])
        float32, host or device, from each source node; times [nsample][nsrc]
        [nrec] at the receivers and/or fields [nsample][nsrc][nz][nx].
        storage: "auto", "shared" or "offchip" (where the work fields live).
        Returns the iterations each problem took (list)."""
        flags = {"auto": 0, "offchip": EIK_OFFCHIP, "shared": EIK_SHARED}[storage]
        _check_dtype(vel, "float32")
        shape = tuple(int(v) for v in vel.shape)
        ns, nz, nx = (1, *shape) if len(shape) == 2 else shape
        siz = np.ascontiguousarray(np.atleast_1d(src_iz), np.int32)
        six = np.ascontiguousarray(np.atleast_1d(src_ix), np.int32)
        nrec = 0 if rec_iz is None else len(rec_iz)
        riz = np.ascontiguousarray(rec_iz if nrec else np.zeros(1), np.int32)
        rix = np.ascontiguousarray(rec_ix if nrec else np.zeros(1), np.int32)
        it = (C.c_int * (ns * siz.size))()
        tp = C.c_void_p(_ptr(times)[0]) if times is not None else None
        fp = C.c_void_p(_ptr(fields)[0]) if fields is not None else None
        arrays = [a for a in (vel, times, fields) if a is not None]
        self._check(lib().rtm_eikonal(self.h, nz, nx, float(dz), float(dx), ns,
                                      C.c_void_p(_ptr(vel)[0]), siz.size, siz.ctypes.data,
                                      six.ctypes.data, nrec, riz.ctypes.data, rix.ctypes.data,
                                      int(max_iter), flags, tp, fp, it,
                                      _stream(*arrays)))
        return list(it)

    def uncertainty_maps(self, mean, std, conf, ratio):
        npix = int(np.prod(mean.shape))
        ptrs = [C.c_void_p(_ptr(a)[0]) for a in (mean, std, conf, ratio)]
        self._check(lib().rtm_uncertainty_maps(self.h, ptrs[0], ptrs[1], npix, ptrs[2], ptrs[3],
                                               _stream(mean, std, conf, ratio)))
        return conf, ratio

    def submit(self, req: Request) -> int:
        t = C.c_uint64()
        self._check(lib().rtm_submit(self.h, C.byref(req), C.byref(t)))
        return t.value

    def poll(self, ticket: int, timeout_ms: int = 0):
        """(state, rc): rc is RTM_OK when the request reached DONE/FAILED."""
        st = C.c_int(-1)
        rc = lib().rtm_poll(self.h, C.c_uint64(ticket), C.byref(st), int(timeout_ms))
        if rc not in (RTM_OK, RTM_ERR_TIMEOUT):
            self._check(rc)
        return st.value, rc
