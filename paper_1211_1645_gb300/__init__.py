"""GB300-native massively parallel local Monte Carlo for hard disks.

Implements the hot path of Engel et al., "Hard-disk equation of state"
(arXiv:1211.1645): the four-colour checkerboard sweep with random grid
shifts (Sec. II.B), the contact-value pressure (Sec. II.C.1, Eqs. 2 and 4)
and the psi_6 orientational order (Sec. III, Eq. 8), as CUDA kernels for
sm_103a behind the C ABI of include/hd.h, with the autocorrelation and
correlation time of Psi_6 (Eq. 9, Table II) and its coarse-grained field.  This package is the ctypes
binding of that library (``hd``) and its build step (``build``).
"""
from . import build
from .hd import (HD_FIXED32, HD_FP64, HDError, HardDisks, hd_batch_init, hd_checkpoint, hd_destroy,
                 hd_get_geometry, hd_init, hd_kernel_times, hd_positions, hd_positions_device, hd_pressure, hd_profile,
                 hd_positional_corr, hd_positional_field, hd_positional_q0, hd_psi6, hd_psi6_acf, hd_psi6_field, hd_psi6_tau, hd_replicas, hd_restore, hd_run, hd_series,
                 hd_series_clear, hd_series_reserve, hd_set_delta, hd_set_positions, hd_set_stream, hd_stats,
                 hd_structure_factor, hd_sweep, hd_tune_delta, load, make_opts)

__all__ = [
    "build", "load", "make_opts", "HardDisks", "HDError", "HD_FP64", "HD_FIXED32", "hd_init", "hd_batch_init",
    "hd_destroy", "hd_sweep", "hd_pressure", "hd_psi6", "hd_positions", "hd_positions_device",
    "hd_set_positions", "hd_stats", "hd_get_geometry", "hd_replicas", "hd_set_stream", "hd_run", "hd_series",
    "hd_series_reserve", "hd_series_clear", "hd_profile", "hd_kernel_times", "hd_checkpoint", "hd_restore",
    "hd_set_delta", "hd_tune_delta", "hd_psi6_acf", "hd_psi6_tau", "hd_psi6_field", "hd_structure_factor",
    "hd_positional_q0", "hd_positional_field", "hd_positional_corr",
]
