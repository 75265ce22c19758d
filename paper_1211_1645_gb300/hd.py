"""Thin ctypes binding of the C ABI in include/hd.h (argument marshalling only).

Every function here forwards to the CUDA library ``_build/libhd.so``; there is
no computational fallback.  If the library is missing or cannot be loaded the
import of a function raises ``HDError``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

HD_OK, HD_ERR_ARG, HD_ERR_CUDA, HD_ERR_OVERFLOW, HD_ERR_TIMEOUT, HD_ERR_REACH, HD_ERR_STATE = range(7)
HD_FP64, HD_FIXED32 = 0, 1
HD_LATTICE_SQUARE, HD_LATTICE_TRIANGULAR = 0, 1

PRECISIONS = {"fp64": HD_FP64, "fixed": HD_FIXED32}
LATTICES = {"square": HD_LATTICE_SQUARE, "triangular": HD_LATTICE_TRIANGULAR}


class HDError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status) if _lib_or_none() else status} (status {status})")


class hd_opts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("lattice", ctypes.c_int32),
        ("trials_per_cell", ctypes.c_int32),
        ("hist_bins", ctypes.c_int32),
        ("hist_dr", ctypes.c_double),
        ("cell_min", ctypes.c_double),
        ("block_threads", ctypes.c_int32),
        ("sweep_kernel", ctypes.c_int32),
        ("threads_per_cell", ctypes.c_int32),
        ("cell_min_per_replica", ctypes.c_void_p),
        ("strips", ctypes.c_int32),
        ("replica_branches", ctypes.c_int32),
    ]


class hd_geometry(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int64),
        ("m", ctypes.c_int32),
        ("capacity", ctypes.c_int32),
        ("trials_per_cell", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("hist_bins", ctypes.c_int32),
        ("graph_branches", ctypes.c_int32),
        ("L", ctypes.c_double),
        ("w", ctypes.c_double),
        ("delta", ctypes.c_double),
        ("eta", ctypes.c_double),
        ("hist_dr", ctypes.c_double),
        ("sweeps", ctypes.c_int64),
    ]


_lock = threading.Lock()
_lib = None


def _lib_or_none():
    return _lib


def load(path: str | None = None):
    """Load libhd.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        so = path or _build.build()
        if not os.path.exists(so):
            raise HDError(HD_ERR_CUDA, f"libhd.so not found at {so}")
        lib = ctypes.CDLL(so)
        c = ctypes
        P = c.c_void_p
        S = c.c_int
        sig = {
            "hd_default_opts": (None, [c.POINTER(hd_opts)]),
            "hd_status_string": (c.c_char_p, [S]),
            "hd_init": (S, [c.POINTER(P), c.c_int64, c.c_double, c.c_double, c.c_double, c.c_uint64,
                            c.POINTER(hd_opts)]),
            "hd_batch_init": (S, [c.POINTER(P), c.c_int32, P, P, c.c_double, P, P, c.POINTER(hd_opts)]),
            "hd_destroy": (S, [P]),
            "hd_set_stream": (S, [P, P]),
            "hd_sweep": (S, [P, c.c_int64]),
            "hd_pressure": (S, [P, P, P, P]),
            "hd_psi6": (S, [P, P, P, P]),
            "hd_positions": (S, [P, P]),
            "hd_positions_device": (S, [P, P]),
            "hd_psi6_local_device": (S, [P, P]),
            "hd_set_positions": (S, [P, P]),
            "hd_stats": (S, [P, P, P]),
            "hd_get_geometry": (S, [P, c.c_int32, c.POINTER(hd_geometry)]),
            "hd_replicas": (c.c_int32, [P]),
            "hd_profile": (S, [P, c.c_int32]),
            "hd_run": (S, [P, c.c_int64, c.c_int32, c.c_int32]),
            "hd_series_reserve": (S, [P, c.c_int64]),
            "hd_series": (S, [P, P, P, c.c_int64]),
            "hd_series_clear": (S, [P]),
            "hd_psi6_mean_noalloc": (S, [P, c.c_int64, P, P]),
            "hd_checkpoint_size": (S, [P, c.POINTER(c.c_size_t)]),
            "hd_set_delta": (S, [P, P]),
            "hd_tune_delta": (S, [P, c.c_double, c.c_int32, c.c_int32, P]),
            "hd_checkpoint": (S, [P, P, c.c_size_t]),
            "hd_restore": (S, [P, P, c.c_size_t]),
            "hd_kernel_times": (S, [P, P, P]),
            "hd_psi6_acf": (S, [P, c.c_int64, P]),
            "hd_psi6_tau": (S, [P, c.c_int64, c.c_int64, P]),
            "hd_psi6_field": (S, [P, c.c_int32, P]),
            "hd_structure_factor": (S, [P, c.c_int32, P, P]),
            "hd_positional_q0": (S, [P, c.c_int32, P, P]),
            "hd_positional_field": (S, [P, P, c.c_int32, P]),
            "hd_positional_corr": (S, [P, P, c.c_int32, c.c_double, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def status_string(s: int) -> str:
    return load().hd_status_string(int(s)).decode()


def _check(st: int, where: str):
    if st != HD_OK:
        raise HDError(st, where)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def hd_default_opts() -> hd_opts:
    o = hd_opts()
    load().hd_default_opts(ctypes.byref(o))
    return o


SWEEP_KERNELS = {"split": 0, "fused": 1, "tma": 2, "persistent": 3}


def make_opts(precision="fp64", lattice="square", trials_per_cell=0, hist_bins=50, hist_dr=1e-3,
              cell_min=2.0, block_threads=128, sweep_kernel="split", threads_per_cell=1, strips=0,
              replica_branches=0) -> hd_opts:
    """hd_opts from keyword values.  cell_min may be one value or one per
    replica (a sequence); the per-replica array is kept alive on the returned
    struct until it is dropped (the library reads it only at creation).
    strips: 0 automatic, 1 none, K >= 2 strips; replica_branches: 0
    automatic, 1 off (see hd.h)."""
    o = hd_default_opts()
    o.precision = PRECISIONS.get(precision, precision)
    o.lattice = LATTICES.get(lattice, lattice)
    o.trials_per_cell = int(trials_per_cell)
    o.hist_bins = int(hist_bins)
    o.hist_dr = float(hist_dr)
    if np.ndim(cell_min) == 0:
        o.cell_min = float(cell_min)
    else:
        per = np.ascontiguousarray(cell_min, dtype=np.float64)
        o.cell_min = float(per.min())
        o._cell_min_keep = per
        o.cell_min_per_replica = per.ctypes.data_as(ctypes.c_void_p)
    o.block_threads = int(block_threads)
    o.sweep_kernel = SWEEP_KERNELS.get(sweep_kernel, sweep_kernel)
    o.threads_per_cell = int(threads_per_cell)
    o.strips = int(strips)
    o.replica_branches = int(replica_branches)
    return o


def hd_init(N, eta, sigma, delta, seed, opts: hd_opts | None = None):
    h = ctypes.c_void_p()
    st = load().hd_init(ctypes.byref(h), int(N), float(eta), float(sigma), float(delta), int(seed),
                        ctypes.byref(opts) if opts is not None else None)
    _check(st, "hd_init")
    return h


def hd_batch_init(N, eta, sigma, delta, seed, opts: hd_opts | None = None):
    N = np.ascontiguousarray(N, np.int64)
    eta = np.ascontiguousarray(eta, np.float64)
    delta = np.ascontiguousarray(delta, np.float64)
    seed = np.ascontiguousarray(seed, np.uint64)
    R = len(N)
    if not (len(eta) == len(delta) == len(seed) == R):
        raise ValueError("per-replica arrays must have equal length")
    h = ctypes.c_void_p()
    st = load().hd_batch_init(ctypes.byref(h), R, _ptr(N), _ptr(eta), float(sigma), _ptr(delta), _ptr(seed),
                              ctypes.byref(opts) if opts is not None else None)
    _check(st, "hd_batch_init")
    return h


def hd_destroy(h):
    _check(load().hd_destroy(h), "hd_destroy")


def hd_set_stream(h, stream_ptr: int | None):
    _check(load().hd_set_stream(h, ctypes.c_void_p(stream_ptr or 0)), "hd_set_stream")


def hd_sweep(h, n: int):
    _check(load().hd_sweep(h, int(n)), "hd_sweep")


def hd_replicas(h) -> int:
    return int(load().hd_replicas(h))


def hd_get_geometry(h, r: int = 0) -> dict:
    g = hd_geometry()
    _check(load().hd_get_geometry(h, int(r), ctypes.byref(g)), "hd_get_geometry")
    return {name: getattr(g, name) for name, _ in hd_geometry._fields_}


def _ntot(h) -> int:
    return sum(hd_get_geometry(h, r)["N"] for r in range(hd_replicas(h)))


def hd_pressure(h, want_hist: bool = True):
    R = hd_replicas(h)
    bp = np.zeros(R, np.float64)
    g0 = np.zeros(R, np.float64)
    K = hd_get_geometry(h, 0)["hist_bins"]
    hist = np.zeros((R, K), np.uint64) if want_hist else None
    _check(load().hd_pressure(h, _ptr(bp), _ptr(g0), _ptr(hist)), "hd_pressure")
    return bp, g0, hist


def hd_psi6(h, want_local: bool = True):
    R = hd_replicas(h)
    re = np.zeros(R, np.float64)
    im = np.zeros(R, np.float64)
    loc = np.zeros((_ntot(h), 2), np.float64) if want_local else None
    _check(load().hd_psi6(h, _ptr(re), _ptr(im), _ptr(loc)), "hd_psi6")
    return re + 1j * im, (None if loc is None else loc[:, 0] + 1j * loc[:, 1])


def hd_positions(h) -> np.ndarray:
    out = np.empty((_ntot(h), 2), np.float64)
    _check(load().hd_positions(h, _ptr(out)), "hd_positions")
    return out


def hd_positions_device(h, dev_ptr: int):
    _check(load().hd_positions_device(h, ctypes.c_void_p(dev_ptr)), "hd_positions_device")


def hd_psi6_local_device(h, dev_ptr: int):
    _check(load().hd_psi6_local_device(h, ctypes.c_void_p(dev_ptr)), "hd_psi6_local_device")


def hd_set_positions(h, xy):
    a = np.ascontiguousarray(xy, np.float64).reshape(-1, 2)
    if a.shape[0] != _ntot(h):
        raise ValueError("positions must have one row per disk")
    _check(load().hd_set_positions(h, _ptr(a)), "hd_set_positions")


def hd_stats(h):
    R = hd_replicas(h)
    a = np.zeros(R, np.uint64)
    b = np.zeros(R, np.uint64)
    _check(load().hd_stats(h, _ptr(a), _ptr(b)), "hd_stats")
    return a, b


def hd_run(h, steps: int, sweeps_per_step: int, measure: int = 1):
    _check(load().hd_run(h, int(steps), int(sweeps_per_step), int(measure)), "hd_run")


def hd_series_reserve(h, steps: int):
    _check(load().hd_series_reserve(h, int(steps)), "hd_series_reserve")


def hd_series(h, max_steps: int = 1 << 20):
    """Recorded steps as an array [n, R, 4]: beta P / rho, g(2 sigma+), Re, Im Psi_6."""
    R = hd_replicas(h)
    n = np.zeros(1, np.int64)
    cap = int(max_steps)
    probe = ctypes.c_int64(0)
    _check(load().hd_series(h, ctypes.byref(probe), None, cap), "hd_series")
    out = np.zeros((max(1, int(probe.value)), R, 4), np.float64)
    _check(load().hd_series(h, _ptr(n), _ptr(out), int(probe.value)), "hd_series")
    return out[: int(n[0])]


def hd_checkpoint(h) -> bytes:
    """The full chain state as bytes (restore with hd_restore)."""
    n = ctypes.c_size_t(0)
    _check(load().hd_checkpoint_size(h, ctypes.byref(n)), "hd_checkpoint_size")
    buf = ctypes.create_string_buffer(n.value)
    _check(load().hd_checkpoint(h, buf, n.value), "hd_checkpoint")
    return buf.raw


def hd_restore(h, blob: bytes):
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(load().hd_restore(h, buf, len(blob)), "hd_restore")


def hd_set_delta(h, delta):
    d = np.ascontiguousarray(np.broadcast_to(np.asarray(delta, np.float64), (hd_replicas(h),)))
    _check(load().hd_set_delta(h, _ptr(d)), "hd_set_delta")


def hd_tune_delta(h, target: float = 0.3, sweeps_per_probe: int = 20, probes: int = 10) -> np.ndarray:
    out = np.zeros(hd_replicas(h), np.float64)
    _check(load().hd_tune_delta(h, float(target), int(sweeps_per_probe), int(probes), _ptr(out)), "hd_tune_delta")
    return out


def hd_series_clear(h):
    _check(load().hd_series_clear(h), "hd_series_clear")


KERNEL_CLASSES = ["draws", "rebuild", "pass", "hist", "fit", "psi6", "psi6_reduce", "positions", "sweep",
                  "analysis"]


def hd_profile(h, enable: bool):
    _check(load().hd_profile(h, int(bool(enable))), "hd_profile")


def hd_psi6_acf(h, max_lag: int):
    """Eq. 9 autocorrelation of the recorded Psi_6 series: complex [R, max_lag + 1]."""
    R = hd_replicas(h)
    out = np.zeros((R, int(max_lag) + 1, 2), np.float64)
    _check(load().hd_psi6_acf(h, int(max_lag), _ptr(out)), "hd_psi6_acf")
    return out[..., 0] + 1j * out[..., 1]


def hd_psi6_tau(h, lag_lo: int, lag_hi: int):
    """Correlation time (in recorded steps) from the exponential part of C: [R]."""
    R = hd_replicas(h)
    out = np.zeros(R, np.float64)
    _check(load().hd_psi6_tau(h, int(lag_lo), int(lag_hi), _ptr(out)), "hd_psi6_tau")
    return out


def hd_psi6_field(h, bins: int):
    """Coarse-grained psi_6 over bins x bins sampling areas: complex [R, bins, bins] ([r, iy, ix])."""
    R = hd_replicas(h)
    out = np.zeros((R, int(bins), int(bins), 2), np.float64)
    _check(load().hd_psi6_field(h, int(bins), _ptr(out)), "hd_psi6_field")
    return out[..., 0] + 1j * out[..., 1]


def hd_structure_factor(h, hk):
    """Eq. 10 at the wave vectors 2 pi (h, k) / L: hk [R, nq, 2] (or [nq, 2] for every replica) -> S [R, nq]."""
    R = hd_replicas(h)
    hk = np.asarray(hk, np.int32)
    if hk.ndim == 2:
        hk = np.broadcast_to(hk, (R,) + hk.shape)
    hk = np.ascontiguousarray(hk, np.int32)
    out = np.zeros((R, hk.shape[1]), np.float64)
    _check(load().hd_structure_factor(h, int(hk.shape[1]), _ptr(hk), _ptr(out)), "hd_structure_factor")
    return out


def hd_positional_q0(h, half_width: int = 3):
    """q_0 = (h, k) of largest S around the first reciprocal shell: ([R, 2] ints, S0 [R])."""
    R = hd_replicas(h)
    hk0 = np.zeros((R, 2), np.int32)
    S0 = np.zeros(R, np.float64)
    _check(load().hd_positional_q0(h, int(half_width), _ptr(hk0), _ptr(S0)), "hd_positional_q0")
    return hk0, S0


def hd_positional_field(h, hk0, bins: int):
    """Mean of chi_j = exp(i q_0 . x_j) over bins x bins areas: complex [R, bins, bins]."""
    R = hd_replicas(h)
    hk0 = np.ascontiguousarray(np.broadcast_to(np.asarray(hk0, np.int32), (R, 2)), np.int32)
    out = np.zeros((R, int(bins), int(bins), 2), np.float64)
    _check(load().hd_positional_field(h, _ptr(hk0), int(bins), _ptr(out)), "hd_positional_field")
    return out[..., 0] + 1j * out[..., 1]


def hd_positional_corr(h, hk0, nr: int, dr: float):
    """Eq. 12 at r_k = (k + 1) dr: complex [R, nr]."""
    R = hd_replicas(h)
    hk0 = np.ascontiguousarray(np.broadcast_to(np.asarray(hk0, np.int32), (R, 2)), np.int32)
    out = np.zeros((R, int(nr), 2), np.float64)
    _check(load().hd_positional_corr(h, _ptr(hk0), int(nr), float(dr), _ptr(out)), "hd_positional_corr")
    return out[..., 0] + 1j * out[..., 1]


def hd_kernel_times(h):
    """{class: (total device ms or 0 when not profiled, launches)}."""
    ms = np.zeros(len(KERNEL_CLASSES), np.float64)
    n = np.zeros(len(KERNEL_CLASSES), np.int64)
    _check(load().hd_kernel_times(h, _ptr(ms), _ptr(n)), "hd_kernel_times")
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNEL_CLASSES)}


class HardDisks:
    """Convenience owner of one context (R >= 1 replicas)."""

    def __init__(self, N, eta, delta, seed, sigma=1.0, precision="fp64", lattice="square", trials_per_cell=0,
                 hist_bins=50, hist_dr=1e-3, cell_min=2.0, block_threads=128, sweep_kernel="split",
                 threads_per_cell=1, strips=0, replica_branches=0):
        opts = make_opts(precision, lattice, trials_per_cell, hist_bins, hist_dr, cell_min, block_threads,
                         sweep_kernel, threads_per_cell, strips, replica_branches)
        if np.ndim(N) == 0:
            self.h = hd_init(N, eta, sigma, delta, seed, opts)
        else:
            self.h = hd_batch_init(N, eta, sigma, delta, seed, opts)
        self.R = hd_replicas(self.h)
        self.precision = precision

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            hd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n=1):
        hd_sweep(self.h, n)

    def positions(self):
        return hd_positions(self.h)

    def set_positions(self, xy):
        hd_set_positions(self.h, xy)

    def stats(self):
        return hd_stats(self.h)

    def pressure(self, want_hist=True):
        return hd_pressure(self.h, want_hist)

    def psi6(self, want_local=True):
        return hd_psi6(self.h, want_local)

    def geometry(self, r=0):
        return hd_get_geometry(self.h, r)

    def set_stream(self, stream_ptr):
        hd_set_stream(self.h, stream_ptr)

    def run(self, steps, sweeps_per_step, measure=True):
        """measure: False/0 sweeps only; True/1 pressure and Psi_6 per step;
        2 also keeps each measurement's local psi_j field on the device."""
        hd_run(self.h, steps, sweeps_per_step, int(measure))

    def psi6_local_device(self, dev_ptr):
        hd_psi6_local_device(self.h, dev_ptr)

    def series(self):
        return hd_series(self.h)

    def set_delta(self, delta):
        hd_set_delta(self.h, delta)

    def tune_delta(self, target=0.3, sweeps_per_probe=20, probes=10):
        return hd_tune_delta(self.h, target, sweeps_per_probe, probes)

    def checkpoint(self):
        return hd_checkpoint(self.h)

    def restore(self, blob):
        hd_restore(self.h, blob)

    def series_reserve(self, steps):
        hd_series_reserve(self.h, steps)

    def series_clear(self):
        hd_series_clear(self.h)

    def profile(self, enable=True):
        hd_profile(self.h, enable)

    def kernel_times(self):
        return hd_kernel_times(self.h)

    def psi6_acf(self, max_lag):
        return hd_psi6_acf(self.h, max_lag)

    def psi6_tau(self, lag_lo, lag_hi):
        return hd_psi6_tau(self.h, lag_lo, lag_hi)

    def psi6_field(self, bins):
        return hd_psi6_field(self.h, bins)

    def structure_factor(self, hk):
        return hd_structure_factor(self.h, hk)

    def positional_q0(self, half_width=3):
        return hd_positional_q0(self.h, half_width)

    def positional_field(self, hk0, bins):
        return hd_positional_field(self.h, hk0, bins)

    def positional_corr(self, hk0, nr, dr):
        return hd_positional_corr(self.h, hk0, nr, dr)
