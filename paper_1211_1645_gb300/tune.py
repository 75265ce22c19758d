"""Performance autotuner for the sweep.

Chooses, for one workload, the minimum cell side (any side >= 2 sigma is a
valid MPMC cell system, Sec. II.B; larger cells hold more disks and make
more trials per cell), the sweep kernel (split launches or one fused
shared-memory launch per sweep) and the threads per block of the split
kernels, by timing graph-captured steps of the library on the current GPU.
Every candidate runs the same chain definition, so only speed is compared;
the trial count per step is read back from the library, so a candidate that
makes cheaper (e.g. more often rejected) trials is not favoured unduly --
only attempted trial moves per second count.
"""
from __future__ import annotations

import itertools

from .hd import HardDisks


def time_config(N, eta, delta, seed, precision, cell_min, sweep_kernel, block_threads, sweeps=50, steps=3):
    """Attempted trial moves per second of `steps` graph-captured steps of
    `sweeps` sweeps (after one untimed step), timed with CUDA events."""
    import torch
    g = HardDisks(N, eta, delta, seed, precision=precision, cell_min=cell_min, sweep_kernel=sweep_kernel,
                  block_threads=block_threads)
    stream = torch.cuda.current_stream()
    g.set_stream(stream.cuda_stream)
    g.run(1, sweeps, measure=False)
    torch.cuda.synchronize()
    a0 = int(g.stats()[0].sum())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.run(steps, sweeps, measure=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    attempts = int(g.stats()[0].sum()) - a0
    geo = g.geometry()
    g.close()
    return {"cell_min": cell_min, "sweep_kernel": sweep_kernel, "block_threads": block_threads,
            "cells_per_side": geo["m"], "trials_per_cell": geo["trials_per_cell"],
            "trial_moves_per_s": attempts / (ms / 1e3)}


def autotune(N, eta, delta, seed=1, precision="fixed", cell_mins=(2.0, 2.2, 2.4), kernels=("split", "fused"),
             block_threads=(64, 128, 256), sweeps=50, steps=3):
    """Time every candidate and return (best, all results sorted by speed).
    Candidates whose geometry is invalid for the workload are skipped."""
    results = []
    for cm, kern, bt in itertools.product(cell_mins, kernels, block_threads):
        if kern == "fused" and bt != block_threads[0]:
            continue  # the fused kernel has a fixed block size
        try:
            results.append(time_config(N, eta, delta, seed, precision, cm, kern, bt, sweeps, steps))
        except Exception:  # an invalid candidate (e.g. a cell too wide for the box)
            continue
    results.sort(key=lambda r: -r["trial_moves_per_s"])
    return (results[0] if results else None), results
