"""Performance autotuner for the sweep.

Any cell side of at least 2 sigma is a valid MPMC cell system (Sec. II.B):
larger cells hold more disks and make more trials per occupied cell, smaller
ones are cheaper per trial.  The autotuner chooses, by timing graph-captured
steps of the library on the current GPU:

* for one workload (``autotune``): the minimum cell side, the sweep kernel
  (split launches, one fused shared-memory launch per sweep, or one
  persistent launch for many sweeps), the threads
  per block of the split kernels, the threads per active cell of the
  split colour pass (1, or a group of 2, 4 or 8 lanes that split the overlap
  tests and combine them with a warp ballot), and for the split one-thread
  pass the strips of the step graph's wavefront (hd_opts.strips);
* for a batch of replicas at different state points, such as the
  equation-of-state scan of Sec. IV.A (``autotune_replicas``): first each
  replica's own cell side, timed on that replica alone, then the threads per
  block and per cell of the whole batch with those cell sides.

The objective is attempted trial moves per second, read back from the
library, so a candidate that makes cheaper (e.g. more often rejected) trials
is not favoured unduly.  A larger cell side is a valid cell system with the
same equilibrium, but with n_t = ceil(N / m^2) trials per occupied cell it
can make two serial trials per cell, which raise the trial rate without
decorrelating the configuration as fast; compare such choices by the Psi_6
correlation time per second (hd_psi6_tau), not by trial moves alone.  The step size delta is tuned
separately, toward an acceptance target (hd_tune_delta), because it changes
the chain's dynamics rather than its speed.
"""
from __future__ import annotations

import itertools

import numpy as np

from .hd import HardDisks


def _time(g, sweeps, steps):
    import torch
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
    return (int(g.stats()[0].sum()) - a0) / (ms / 1e3)


def time_config(N, eta, delta, seed, precision, cell_min, sweep_kernel, block_threads, sweeps=50, steps=3,
                threads_per_cell=1, strips=0):
    """Attempted trial moves per second of `steps` graph-captured steps of
    `sweeps` sweeps (after one untimed step), timed with CUDA events.  N, eta,
    delta, seed and cell_min may be per-replica lists (one batched context).
    strips: hd_opts.strips (0 automatic, 1 none, K)."""
    g = HardDisks(N, eta, delta, seed, precision=precision, cell_min=cell_min, sweep_kernel=sweep_kernel,
                  block_threads=block_threads, threads_per_cell=threads_per_cell, strips=strips)
    rate = _time(g, sweeps, steps)
    geo = g.geometry()
    g.close()
    return {"cell_min": cell_min, "sweep_kernel": sweep_kernel, "block_threads": block_threads,
            "threads_per_cell": threads_per_cell, "strips": strips, "graph_branches": geo["graph_branches"],
            "cells_per_side": geo["m"], "trials_per_cell": geo["trials_per_cell"], "trial_moves_per_s": rate}


def autotune(N, eta, delta, seed=1, precision="fixed", cell_mins=(2.0, 2.2, 2.4), kernels=("split", "fused"),
             block_threads=(64, 128, 256), threads_per_cell=(1,), strips=(1,), sweeps=50, steps=3):
    """Time every candidate and return (best, all results sorted by speed).
    Candidates whose geometry or launch shape is invalid for the workload are
    skipped (the library rejects them at creation).  strips applies to the
    split kernel with one thread per cell (others run without strips)."""
    results = []
    for cm, kern, bt, g, k in itertools.product(cell_mins, kernels, block_threads, threads_per_cell, strips):
        if kern == "fused" and (bt != block_threads[0] or g != 1):
            continue  # the fused kernel has a fixed block size and one thread per cell
        if kern in ("tma", "persistent") and g != 1:
            continue
        wave = kern == "split" and g == 1
        if not wave and k != strips[0]:
            continue  # strips apply to the split one-thread pass: the others are timed once, without
        try:
            results.append(time_config(N, eta, delta, seed, precision, cm, kern, bt, sweeps, steps, g,
                                       k if wave else 1))
        except Exception:  # an invalid candidate (e.g. a cell too wide for the box)
            continue
    results.sort(key=lambda r: -r["trial_moves_per_s"])
    return (results[0] if results else None), results


def autotune_replicas(Ns, etas, delta, seed=1, precision="fixed", cell_mins=(2.0, 2.2, 2.4),
                      block_threads=(128, 256), threads_per_cell=(1, 2), sweeps=20, steps=2):
    """Per-replica cell sides for a batch, then the batch's launch shape.

    Stage 1: for each distinct state point (N, eta) of the batch, every cell
    side in `cell_mins` is timed on a single-replica context (split kernel,
    128 threads); the fastest is that replica's cell side.  Stage 2: the whole
    batch is timed with those cell sides, and with the first cell side for
    every replica (a batch runs one kernel specialisation, and a replica whose
    cells make two trials each takes the whole batch off the one-trial one),
    for every (block_threads, threads_per_cell) candidate.  Returns (choice,
    table) where choice holds the per-replica "cell_min" list,
    "block_threads", "threads_per_cell" and the batch's "trial_moves_per_s",
    and table the stage-2 results."""
    R = len(Ns)
    deltas = list(delta) if np.ndim(delta) else [float(delta)] * R
    per_point = {}
    for n, e in sorted(set(zip(Ns, etas))):
        best, best_rate = None, -1.0
        for cm in cell_mins:
            try:
                r = time_config(n, e, deltas[0], seed, precision, cm, "split", 128, sweeps, steps)
            except Exception:
                continue
            if r["trial_moves_per_s"] > best_rate:
                best, best_rate = cm, r["trial_moves_per_s"]
        per_point[(n, e)] = best if best is not None else 2.0
    # the batch runs one kernel specialisation for all replicas: cell sides
    # that give some replica two trials per occupied cell can slow the whole
    # batch, so the uniform first cell side is a candidate too
    layouts = [[per_point[(n, e)] for n, e in zip(Ns, etas)]]
    if any(c != cell_mins[0] for c in layouts[0]):
        layouts.append([cell_mins[0]] * R)
    seeds = [seed + r for r in range(R)]
    table = []
    for cms, bt, g in itertools.product(layouts, block_threads, threads_per_cell):
        try:
            t = time_config(list(Ns), list(etas), deltas, seeds, precision, cms, "split", bt, sweeps, steps, g)
        except Exception:
            continue
        table.append({"cell_min": cms, "block_threads": bt, "threads_per_cell": g,
                      "trial_moves_per_s": t["trial_moves_per_s"]})
    table.sort(key=lambda r: -r["trial_moves_per_s"])
    if not table:
        return None, table
    return dict(table[0]), table
