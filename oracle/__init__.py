"""CPU oracle for massively parallel local Monte Carlo of hard disks.

TEST INFRASTRUCTURE ONLY.  This package is the slow, sequential, obviously
correct statement of what the GPU library computes:

* ``hd_oracle.c`` - the checkerboard MPMC chain of Engel et al.,
  arXiv:1211.1645, Sec. II.B (four colours, random colour order, random grid
  shift after each sweep, shuffled serial trials inside a cell, moves that
  leave the cell rejected), in plain FP64 and in cell-relative fixed point;
  the contact-shell pair histogram (numerator of Eq. 2) and the local /
  global bond order psi_6 (Eq. 8).
* this module - ctypes access to it, plus the g(r) normalisation (Eq. 2),
  the quartic contact extrapolation (Sec. II.C.1) and the contact-value
  pressure (Eq. 4) in numpy; the autocorrelation of the global psi_6 series
  and its correlation time (Sec. III, Eq. 9, Table II); the coarse-grained
  psi_6 field over square sampling areas (Sec. IV, Figs. 5-6); the structure
  factor, the positional order chi_j and the positional correlation function
  (Sec. IV.C, Eqs. 10-12).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library.

Pins (tests/test_oracle_*.py): Philox known-answer vectors; never-overlap
invariant; exact two-disk separation law and two-disk pressure; hard-disk
virial series at low density; ideal-gas g(r) = (N-1)/N; exact synthetic
quartic recovery; frame-change invariance; psi_6 of hand-built hexagonal
shells and its rotation / reflection covariance; brute-force neighbour and
pair enumeration; the autocorrelation of constant and uniformly rotating
series (exact), of a complex AR(1) process (rho^dt) and an exact exponential
(tau); the coarse field of uniform psi_j, of one sampling area (= Psi_6),
of disks on sampling-area edges, and against a per-area loop; the global
Psi_6 against exact rational arithmetic and under reordering of the disks.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hd_oracle.c")
_SO = os.path.join(_HERE, "_build", "libhd_oracle.so")
_lock = threading.Lock()
_lib = None

FP64 = 0
FIXED = 1
FORMS = {"fp64": FP64, "fixed": FIXED}
LATTICES = {"square": 0, "triangular": 1}

# 2^24 fixed-point units per sigma
FX_SCALE = 16777216.0


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, IEEE order kept)."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm",
        ])
        os.replace(tmp, _SO)
    return _SO


_OMP_SRC = os.path.join(_HERE, "hd_oracle_omp.c")
_OMP_SO = os.path.join(_HERE, "_build", "libhd_oracle_omp.so")
_omp_lib = None


def build_omp(force: bool = False) -> str | None:
    """Compile the OpenMP sweep (hd_oracle_omp.c, which includes the oracle's
    own source) with gcc -fopenmp; None when the compiler has no OpenMP."""
    os.makedirs(os.path.dirname(_OMP_SO), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_OMP_SRC))
    if force or not os.path.exists(_OMP_SO) or os.path.getmtime(_OMP_SO) < newest:
        tmp = _OMP_SO + f".tmp{os.getpid()}"
        r = subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                            "-fopenmp", "-Wall", "-o", tmp, _OMP_SRC, "-lm"], capture_output=True)
        if r.returncode != 0:
            return None
        os.replace(tmp, _OMP_SO)
    return _OMP_SO


def _load_omp():
    """The OpenMP library, or None.  It shares the state layout of the oracle
    (the same source), so it advances the oracle's own chains."""
    global _omp_lib
    with _lock:
        if _omp_lib is None:
            so = build_omp()
            if so is None:
                return None
            lib = ctypes.CDLL(so)
            lib.hdo_sweep_omp.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]
            _omp_lib = lib
        return _omp_lib


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        c = ctypes
        P = c.c_void_p
        lib.hdo_create.restype = P
        lib.hdo_create.argtypes = [c.c_int64, c.c_double, c.c_double, c.c_uint64, c.c_int,
                                   c.c_int, c.c_int, c.c_double, c.POINTER(c.c_int)]
        lib.hdo_destroy.argtypes = [P]
        lib.hdo_sweep.argtypes = [P, c.c_int64]
        lib.hdo_positions.argtypes = [P, P]
        lib.hdo_set_positions.argtypes = [P, P]
        lib.hdo_set_positions.restype = c.c_int
        lib.hdo_stats.argtypes = [P, P, P]
        lib.hdo_geometry.argtypes = [P, P]
        lib.hdo_frame.argtypes = [P, P, P, P]
        lib.hdo_histogram.argtypes = [P, c.c_int, c.c_double, c.c_int, P]
        lib.hdo_histogram.restype = c.c_int
        lib.hdo_psi6.argtypes = [P, c.c_int, P]
        lib.hdo_psi6.restype = c.c_int
        lib.hdo_philox4x32_10.argtypes = [P, P, P]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block: four 32-bit counter words, two key words."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.hdo_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


class OracleChain:
    """One MPMC chain: N disks of radius sigma = 1 at packing fraction eta.

    form      "fp64" or "fixed" (cell-relative 2^-24 sigma integers)
    lattice   "square" or "triangular" (odd rows offset by half a spacing)
    nt        trial moves per occupied active cell per pass (0: ceil(N/m^2))
    cell_min  minimum cell side (>= 2 sigma)
    """

    def __init__(self, N: int, eta: float, delta: float, seed: int, form: str = "fp64",
                 lattice: str = "square", nt: int = 0, cell_min: float = 2.0):
        lib = _load()
        st = ctypes.c_int(0)
        self._h = lib.hdo_create(int(N), float(eta), float(delta), int(seed), FORMS[form],
                                 LATTICES[lattice], int(nt), float(cell_min), ctypes.byref(st))
        if not self._h:
            raise ValueError(f"oracle rejected N={N} eta={eta} delta={delta} form={form} (status {st.value})")
        self.N = int(N)
        self.form = form
        self.eta_requested = float(eta)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _load().hdo_destroy(h)
            self._h = None

    def sweep(self, n: int = 1) -> None:
        _load().hdo_sweep(self._h, int(n))

    def sweep_omp(self, n: int = 1, threads: int = 0) -> bool:
        """The same n sweeps with each colour's cells shared out between
        `threads` host threads (0: all); False when OpenMP is unavailable."""
        lib = _load_omp()
        if lib is None:
            return False
        lib.hdo_sweep_omp(self._h, int(n), int(threads))
        return True

    def positions(self) -> np.ndarray:
        out = np.empty((self.N, 2), dtype=np.float64)
        _load().hdo_positions(self._h, _ptr(out))
        return out

    def set_positions(self, xy) -> None:
        a = np.ascontiguousarray(xy, dtype=np.float64).reshape(self.N, 2)
        _load().hdo_set_positions(self._h, _ptr(a))

    def stats(self):
        a = np.zeros(1, np.uint64)
        b = np.zeros(1, np.uint64)
        _load().hdo_stats(self._h, _ptr(a), _ptr(b))
        return int(a[0]), int(b[0])

    def geometry(self) -> dict:
        g = np.zeros(10, np.float64)
        _load().hdo_geometry(self._h, _ptr(g))
        L = g[0]
        return {"L": L, "w": g[1], "delta": g[2], "m": int(g[3]), "W": int(g[4]), "LF": int(g[5]),
                "D": int(g[6]), "nt": int(g[7]), "max_occupancy": int(g[8]), "sweeps": int(g[9]),
                "eta": self.N * np.pi / (L * L)}

    def frame(self):
        cells = np.empty((self.N, 2), np.int32)
        offs = np.empty((self.N, 2), np.float64)
        shift = np.empty(2, np.float64)
        _load().hdo_frame(self._h, _ptr(cells), _ptr(offs), _ptr(shift))
        return cells, offs, shift

    def histogram(self, K: int, dr: float, brute: bool = False) -> np.ndarray:
        out = np.zeros(int(K), np.uint64)
        rc = _load().hdo_histogram(self._h, int(K), float(dr), int(bool(brute)), _ptr(out))
        if rc != 0:
            raise ValueError(f"histogram reach exceeds the box (status {rc})")
        return out

    def psi6(self, brute: bool = False):
        """Local psi_j (Eq. 8) by disk id, and the global Psi_6 = (1/N) sum_j
        psi_j: each part's sum over the disks exactly rounded to double
        (math.fsum), then divided by N."""
        loc = np.empty((self.N, 2), np.float64)
        rc = _load().hdo_psi6(self._h, int(bool(brute)), _ptr(loc))
        if rc != 0:
            raise ValueError(f"psi6 neighbour search failed (status {rc})")
        return loc[:, 0] + 1j * loc[:, 1], psi6_mean(loc[:, 0] + 1j * loc[:, 1])

    def realised_dr(self, dr: float) -> float:
        """Bin width actually used: dr itself (FP64) or dr on the 2^-24 grid."""
        if self.form == "fixed":
            return float(np.round(dr * FX_SCALE)) / FX_SCALE
        return float(dr)


def psi6_mean(psi_local) -> complex:
    """Global Psi_6 = (1/N) sum_j psi_j (Eq. 8).  The sum of each part is
    exactly rounded to double (math.fsum: independent of summation order),
    then divided by N once."""
    z = np.asarray(psi_local, dtype=np.complex128).ravel()
    n = float(z.size)
    return complex(math.fsum(z.real.tolist()) / n, math.fsum(z.imag.tolist()) / n)


def g_of_r(counts, N: int, L: float, dr: float):
    """Eq. 2: g(r_k) = (n_k / p) / (2 pi r_k dr / V) at bin centres r_k.

    p = N^2 / 2, the reading under which Eq. 4 is exact at finite N (for two
    disks it reproduces beta P = 1/V + 1/(V - 4 pi sigma^2) exactly)."""
    n = np.asarray(counts, dtype=np.float64)
    K = n.shape[-1]
    r = 2.0 + (np.arange(K, dtype=np.float64) + 0.5) * dr
    V = L * L
    p = 0.5 * float(N) * float(N)
    return r, (n / p) / (2.0 * np.pi * r * dr / V)


def contact_fit(r, g, degree: int = 4) -> float:
    """Sec. II.C.1: least-squares polynomial of the given degree (fourth
    order in the paper) in x = r - 2 sigma, extrapolated to x = 0."""
    x = np.asarray(r, dtype=np.float64) - 2.0
    A = np.vander(x, degree + 1, increasing=True)
    coef, *_ = np.linalg.lstsq(A, np.asarray(g, dtype=np.float64), rcond=None)
    return float(coef[0])


def contact_pressure(counts, N: int, L: float, dr: float, degree: int = 4) -> dict:
    """Eq. 4: beta P / rho = 1 + 2 eta g(2 sigma+), with eta = N pi / L^2.
    P* = beta P (2 sigma)^2 (Eq. 1)."""
    r, g = g_of_r(counts, N, L, dr)
    g0 = contact_fit(r, g, degree)
    eta = N * np.pi / (L * L)
    bp_rho = 1.0 + 2.0 * eta * g0
    return {"g0": g0, "betaP_over_rho": bp_rho, "Pstar": bp_rho * 4.0 * N / (L * L), "eta": eta,
            "g": g, "r": r}


def psi6_acf(psi, max_lag: int) -> np.ndarray:
    """Eq. 9: C(dt) = <Psi_6(t) Psi_6*(t + dt)>_t / <|Psi_6|^2> of a series
    Psi_6(t), t = 0 .. T-1, one entry per measurement.  The numerator averages
    over the T - dt pairs the series holds, the denominator over all T
    entries, so C(0) = 1.  Returns complex C(0 .. max_lag)."""
    z = np.asarray(psi, dtype=np.complex128)
    T = len(z)
    if max_lag < 0 or max_lag >= T:
        raise ValueError("need 0 <= max_lag < len(series)")
    den = np.mean(z.real * z.real + z.imag * z.imag)
    return np.array([np.mean(z[:T - d] * np.conj(z[d:])) / den for d in range(max_lag + 1)])


def acf_tau(C, lag_lo: int, lag_hi: int) -> float:
    """Correlation time from the purely exponential part C(dt) ~ exp(-dt / tau)
    (Sec. III): the least-squares line through (dt, ln Re C(dt)) over
    lag_lo <= dt <= lag_hi where Re C > 0; tau = -1 / slope, in the units of
    dt.  NaN with fewer than two such lags or a slope >= 0."""
    c = np.real(np.asarray(C))
    d = np.arange(lag_lo, lag_hi + 1)
    d = d[(d < len(c)) & (c[np.minimum(d, len(c) - 1)] > 0)]
    if len(d) < 2:
        return float("nan")
    slope = np.polyfit(d.astype(np.float64), np.log(c[d]), 1)[0]
    return float(-1.0 / slope) if slope < 0 else float("nan")


def psi6_field(xy, psi_local, L: float, bins: int, LF: int | None = None) -> np.ndarray:
    """Coarse-grained psi_6 (the sampling-area averages of Figs. 5-6): the
    mean of psi_j over the disks whose centres lie in each of bins x bins
    half-open squares of side L / bins, NaN where a square is empty.  Square
    index floor(x bins / L) per axis; in the fixed-point form (LF = box side
    in 2^-24 sigma units) the index is floor(X bins / LF) of the exact integer
    coordinate X.  Returns complex [bins, bins] indexed [iy, ix]."""
    xy = np.asarray(xy, dtype=np.float64)
    psi = np.asarray(psi_local, dtype=np.complex128)
    if LF is None:
        ix = np.floor(xy[:, 0] * bins / L).astype(np.int64)
        iy = np.floor(xy[:, 1] * bins / L).astype(np.int64)
    else:
        X = np.round(xy * FX_SCALE).astype(np.int64)
        ix = (X[:, 0] * bins) // int(LF)
        iy = (X[:, 1] * bins) // int(LF)
    ix = np.minimum(ix, bins - 1)
    iy = np.minimum(iy, bins - 1)
    flat = iy * bins + ix
    cnt = np.bincount(flat, minlength=bins * bins).astype(np.float64)
    re = np.bincount(flat, weights=psi.real, minlength=bins * bins)
    im = np.bincount(flat, weights=psi.imag, minlength=bins * bins)
    with np.errstate(invalid="ignore", divide="ignore"):
        out = (re + 1j * im) / cnt
    out[cnt == 0] = np.nan + 1j * np.nan
    return out.reshape(bins, bins)


def structure_factor(xy, hk, L: float) -> np.ndarray:
    """Eq. 10: S(q) = (1/N) sum_{n,m} exp(i q (x_n - x_m)) = |sum_n exp(i q x_n)|^2 / N
    at the box-periodic wave vectors q = 2 pi (h, k) / L, hk [nq, 2] integers."""
    xy = np.asarray(xy, dtype=np.float64)
    q = 2.0 * np.pi * np.asarray(hk, dtype=np.float64) / L
    amp = np.exp(1j * (xy @ q.T)).sum(axis=0)
    return (amp.real ** 2 + amp.imag ** 2) / len(xy)


def q0_window(psi6_global: complex, eta: float, L: float, half_width: int) -> np.ndarray:
    """Candidate wave vectors for q_0 (Sec. IV.C): the box's reciprocal grid
    points within +-half_width of the first-shell reciprocal vector of a
    triangular lattice of the same density (|q| = 4 pi / (a sqrt 3), area per
    disk sqrt(3) a^2 / 2) whose bonds follow the global orientation
    (angle arg(Psi_6) / 6), i.e. at that angle + 30 degrees.  The paper leaves
    q_0 to the maximum of S near this point because vacancies and other
    defects stretch the effective lattice constant.  Returns hk [nq, 2]."""
    rho = eta / np.pi
    a = np.sqrt(2.0 / (np.sqrt(3.0) * rho))
    qmag = 4.0 * np.pi / (a * np.sqrt(3.0))
    th = np.angle(psi6_global) / 6.0 + np.pi / 6.0
    hc = int(np.rint(qmag * np.cos(th) * L / (2.0 * np.pi)))
    kc = int(np.rint(qmag * np.sin(th) * L / (2.0 * np.pi)))
    d = np.arange(-half_width, half_width + 1)
    H, K = np.meshgrid(hc + d, kc + d, indexing="ij")
    return np.stack([H.ravel(), K.ravel()], axis=1)


def positional_q0(xy, hk_window, L: float):
    """q_0 = the candidate of largest S (first in window order on ties)."""
    S = structure_factor(xy, hk_window, L)
    i = int(np.argmax(S))
    return np.asarray(hk_window[i]), float(S[i])


def positional_chi(xy, hk0, L: float) -> np.ndarray:
    """Eq. 11: chi_j = exp(i q_0 . x_j), q_0 = 2 pi hk0 / L."""
    q = 2.0 * np.pi * np.asarray(hk0, dtype=np.float64) / L
    return np.exp(1j * (np.asarray(xy, dtype=np.float64) @ q))


def positional_corr(xy, hk0, L: float, r):
    """Eq. 12: C(r) = < exp(i q_0 (x_n - x_m)) > over the ordered pairs n != m
    whose minimum-image separation lies in [r - sigma, r + sigma] (sigma = 1),
    for every r of `r`; NaN where no pair qualifies.  Brute force.  The
    window test is lo^2 <= d^2 <= (r + 1)^2 with lo = max(r - 1, 0) and
    d^2 = dx dx + dy dy of the minimum-image difference d = x_m - x_n -
    L rint((x_m - x_n) / L) of the global positions, in that operation order."""
    xy = np.asarray(xy, dtype=np.float64)
    chi = positional_chi(xy, hk0, L)
    d = xy[None, :, :] - xy[:, None, :]  # [n, m] = x_m - x_n
    d = d - L * np.rint(d / L)
    d2 = d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]
    prod = chi[:, None] * np.conj(chi[None, :])
    np.fill_diagonal(d2, -10.0)
    out = np.empty(len(r), complex)
    for i, rr in enumerate(r):
        lo = max(rr - 1.0, 0.0)
        sel = (d2 >= lo * lo) & (d2 <= (rr + 1.0) * (rr + 1.0))
        out[i] = prod[sel].mean() if sel.any() else np.nan + 1j * np.nan
    return out
