#!/usr/bin/env python
"""Benchmark: hard-disk trial moves per second at N = 1024^2, eta = 0.716.

One step = S checkerboard sweeps (each: cell rebuild on a freshly shifted
grid + four colour passes) followed by one measurement (contact-histogram
pressure and global psi_6), i.e. one pass of the whole hot path.  The
headline form is the cell-relative fixed-point chain; the plain FP64 chain
runs the same seed schedule and is reported beside it.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events
on the library's stream; L2 is flushed (a 256 MB write) before every timed
step, outside the events.  Under torchrun each rank runs its own replica
(seed + rank, weak scaling) and rank 0 reports the max time over ranks.
Each step is one graph launch of the library (hd_run).

Secondary keys of the same line (same step and timing): `sweeps_only` (the
same S sweeps without the measurement), `fp64` (the plain FP64 chain),
`replicas4` (four replicas of the headline system in one context), `scan31`
(the 31-replica equation-of-state scan), `autotuned` (the headline system
at the cell side and block size the autotuner picks) and `config5` (N =
2048^2 at eta = 0.720, a state larger than L2, 250 sweeps and a measurement
with the local psi_j field per step).

Roofline: after the timed steps two more steps replay as profiled graphs
(a timing event around every kernel node); each kernel class is charged its
share of those event times x the graph-timed ms_per_step, and the dominant
class's time per launch gives its achieved rates against three roofs (HBM
copy bandwidth, L2-resident copy bandwidth, warp-instruction issue).  The
binding roof is picked from the committed ncu counters of that kernel, which
`roofline.ncu` repeats while the kernel's sources are unchanged.

--impl reference times the CPU oracle (one core) on a bounded sample of the
same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "disk trial moves/s at N=1M, η=0.716: fixed-point batched vs plain FP64"
UNIT = "trial moves/s"
L2_FLUSH_BYTES = 256 << 20


def parse_args(argv=None):
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--sweeps-per-step", type=int, default=100)
    p.add_argument("--N", type=int, default=1024 * 1024)
    p.add_argument("--eta", type=float, default=0.716)
    p.add_argument("--delta", type=float, default=0.1)
    p.add_argument("--cell-min", type=float, default=2.0, help="minimum cell side in sigma (>= 2)")
    p.add_argument("--seed", type=int, default=1)
    p.add_argument("--form", choices=["fixed", "fp64"], default="fixed")
    p.add_argument("--lattice", choices=["square", "triangular"], default="square",
                   help="start lattice (triangular: odd rows shifted by half a spacing)")
    p.add_argument("--sweep-kernel", choices=["split", "tma", "fused"], default="split")
    p.add_argument("--strips", type=int, default=0,
                   help="graph wavefront strips of a one-replica step (0: the library's choice, 1: none)")
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison leg")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extras", action="store_true", help="skip the replica, scan and autotuned lines")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--cpu-seconds", type=float, default=10.0, help="CPU oracle sample budget")
    return p.parse_args(argv)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# distributed helpers (one process per GPU, independent replicas)
# ---------------------------------------------------------------------------
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max_sum(world, tmax: float, tsum: float, device):
    """Max of tmax and sum of tsum over ranks."""
    if world == 1:
        return tmax, tsum
    import torch
    import torch.distributed as dist
    a = torch.tensor([tmax], dtype=torch.float64, device=device)
    b = torch.tensor([tsum], dtype=torch.float64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(a.item()), float(b.item())


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def time_form(args, form, rank, world, steps, warmup, sampler=None, N=None, eta=None, cell_min=None,
              block_threads=128, sweep_kernel=None, measure=1, lattice="square", sweeps=None, threads_per_cell=1,
              keep_positions=False, strips=None):
    """Device-resident timing of `steps` steps of one form; returns a dict.
    N and eta may be per-replica lists (one batched context); attempts are
    summed over replicas.  measure: 0 sweeps only, 1 pressure and Psi_6 per
    step, 2 also the local psi_j field kept on the device.  Afterwards two
    more steps are replayed as profiled graphs (a timing event before and
    after every kernel node) for the per-kernel device times."""
    import numpy as np
    import torch

    import paper_1211_1645_gb300 as hd

    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    N = args.N if N is None else N
    eta = args.eta if eta is None else eta
    if np.ndim(N) == 0:
        sysg = hd.HardDisks(N, eta, args.delta, args.seed + rank, precision=form,
                            sweep_kernel=sweep_kernel or args.sweep_kernel, lattice=lattice,
                            cell_min=cell_min or args.cell_min, block_threads=block_threads,
                            threads_per_cell=threads_per_cell, strips=args.strips if strips is None else strips)
    else:
        R = len(N)
        seeds = [args.seed + rank * R + r for r in range(R)]
        sysg = hd.HardDisks(list(N), list(eta), [args.delta] * R, seeds, precision=form,
                            sweep_kernel=sweep_kernel or args.sweep_kernel,
                            cell_min=cell_min or args.cell_min, block_threads=block_threads,
                            threads_per_cell=threads_per_cell)
    sysg.set_stream(stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    S = sweeps or args.sweeps_per_step

    # one step = one graph launch: S sweeps + pressure and Psi_6 recorded on the device
    # (measure=0: the S sweeps alone)
    sysg.series_reserve(warmup + steps + 8)

    def step():
        sysg.run(1, S, measure)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    att0 = int(sysg.stats()[0].sum())
    l0 = sysg.kernel_times()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    barrier(world)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    barrier(world)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    att1, acc1 = sysg.stats()
    attempts = int(att1.sum()) - att0
    acceptance = float(acc1.sum()) / float(att1.sum()) if int(att1.sum()) else None
    l1 = sysg.kernel_times()
    launches = sum(l1[k][1] - l0[k][1] for k in l1)

    # profiled replays: per-kernel device time inside the step graph
    sysg.profile(True)
    for _ in range(PROFILED_STEPS):
        flush.zero_()
        step()
    kt = sysg.kernel_times()
    sysg.profile(False)
    geo = sysg.geometry()
    series = sysg.series()
    final_xy = sysg.positions() if keep_positions else None
    sysg.close()
    return {"ms": ms, "steps": steps, "attempts": attempts, "launches": launches, "clocks": clocks,
            "kernel_times": kt, "geometry": geo, "last_measurement": series[-1, 0].tolist() if len(series) else None,
            "acceptance": acceptance, "final_xy": final_xy}


PROFILED_STEPS = 2


def in_step_times(run, ms_per_step):
    """Per-step device time (ms) and launches of each kernel class from the
    profiled graph replays, and the factor that charges each class its share
    of the graph-timed step: in-step time of a class = its share of the
    summed event times x ms_per_step.  The event nodes add a launch latency
    to every kernel and serialise kernels that overlap in the timed graph, so
    the event times themselves are not in-step durations (their sum is
    typically 1.5x ms_per_step); the shares agree with the ncu launch list.
    Any gap between kernels of the timed step is charged to the kernels,
    which can only lower an achieved rate derived from these times."""
    kt = run["kernel_times"]
    per = {k: v[0] / PROFILED_STEPS for k, v in kt.items() if v[1]}
    n = {k: v[1] / PROFILED_STEPS for k, v in kt.items() if v[1]}
    total = sum(per.values())
    scale = ms_per_step / total if total > 0 else 1.0
    return per, n, total, scale


# The equation-of-state scan: replica r has N = SCAN_N[r mod 5], eta = 0.700 + 0.001 r.
SCAN_N = [128 ** 2, 192 ** 2, 256 ** 2, 384 ** 2, 512 ** 2]


def time_extras(args, rank, world, dev):
    """Secondary lines, same step definition and timing as the headline:
    four replicas of the headline system in one context, the 31-replica
    equation-of-state scan, and the headline system at the cell side, sweep
    kernel and block size the autotuner picks (sweeps only, then re-timed
    with measurement and L2 flush)."""
    from paper_1211_1645_gb300.tune import autotune, autotune_replicas
    out = {}
    steps, warm = max(1, args.steps // 2), 2
    r4 = time_form(args, args.form, rank, world, steps, warm, N=[args.N] * 4, eta=[args.eta] * 4)
    t, a = reduce_max_sum(world, r4["ms"], float(r4["attempts"]), dev)
    out["replicas4"] = {"value": a / (t / 1e3), "unit": UNIT, "ms_per_step": t / steps,
                        "config": f"4 replicas x N={args.N}, eta={args.eta}, one context"}
    R = 31
    Ns = [SCAN_N[r % 5] for r in range(R)]
    etas = [0.700 + 0.001 * r for r in range(R)]
    rs = time_form(args, args.form, rank, world, steps, warm, N=Ns, eta=etas)
    t, a = reduce_max_sum(world, rs["ms"], float(rs["attempts"]), dev)
    out["scan31"] = {"value": a / (t / 1e3), "unit": UNIT, "ms_per_step": t / steps,
                     "config": f"31 replicas, N = {{128^2 .. 512^2}} round-robin ({sum(Ns)} disks), "
                               "eta = 0.700 + 0.001 r, one context"}
    # the scan with a cell side per replica and the batch's launch shape chosen by the autotuner
    choice, stable = autotune_replicas(Ns, etas, args.delta, args.seed + rank * R, precision=args.form,
                                       cell_mins=(2.0, 2.2, 2.4), block_threads=(128, 256),
                                       threads_per_cell=(1, 2, 4))
    if choice:
        ra = time_form(args, args.form, rank, world, steps, warm, N=Ns, eta=etas, cell_min=choice["cell_min"],
                       block_threads=choice["block_threads"], threads_per_cell=choice["threads_per_cell"])
        t, a = reduce_max_sum(world, ra["ms"], float(ra["attempts"]), dev)
        out["scan31_autotuned"] = {
            "value": a / (t / 1e3), "unit": UNIT, "ms_per_step": t / steps,
            "vs_default": (a / (t / 1e3)) / out["scan31"]["value"],
            "choice": {"cell_min_per_replica": choice["cell_min"], "block_threads": choice["block_threads"],
                       "threads_per_cell": choice["threads_per_cell"]},
            "candidates": [{"cell_min_per_replica": c["cell_min"] if len(set(c["cell_min"])) > 1 else c["cell_min"][0],
                            "block_threads": c["block_threads"], "threads_per_cell": c["threads_per_cell"],
                            "trial_moves_per_s": c["trial_moves_per_s"]} for c in stable]}
    best, table = autotune(args.N, args.eta, args.delta, args.seed + rank, precision=args.form,
                           cell_mins=(2.0, 2.2, 2.4), kernels=("split", "persistent"), block_threads=(128, 256),
                           threads_per_cell=(1, 2), strips=(1, 8, 16, 24), sweeps=args.sweeps_per_step, steps=2)
    if best:
        rt = time_form(args, args.form, rank, world, steps, warm, cell_min=best["cell_min"],
                       block_threads=best["block_threads"], sweep_kernel=best["sweep_kernel"],
                       threads_per_cell=best["threads_per_cell"], strips=best["strips"])
        t, a = reduce_max_sum(world, rt["ms"], float(rt["attempts"]), dev)
        keys = ("cell_min", "sweep_kernel", "block_threads", "threads_per_cell", "strips")
        out["autotuned"] = {"value": a / (t / 1e3), "unit": UNIT, "ms_per_step": t / steps,
                            "choice": {k: best[k] for k in keys + ("cells_per_side", "trials_per_cell")},
                            "candidates": [{k: c[k] for k in keys + ("trial_moves_per_s",)} for c in table]}
    return out


def time_e2e(args, form, rank, steps, xy0):
    """Same metric through the public API with host buffers: each step uploads
    the step's input configuration from pinned host memory (hd_set_positions:
    copy and binning on the device), runs the step (hd_run: one graph launch
    of the sweeps and the device-side pressure and Psi_6 measurement) and
    reads the step's result back (hd_series: the recorded count, then the
    step's beta P / rho, g(2 sigma+) and Psi_6; the series is then cleared).
    The input is xy0, the configuration the device-timed leg ended in, so
    that both legs time the same state (trial moves per sweep are the
    occupied cells, which a fresh lattice has more of than a relaxed
    configuration)."""
    import torch

    import paper_1211_1645_gb300 as hd

    sysg = hd.HardDisks(args.N, args.eta, args.delta, args.seed + rank, precision=form, cell_min=args.cell_min,
                        strips=args.strips)
    pinned = torch.empty((xy0.shape[0], 2), dtype=torch.float64, pin_memory=True)
    xy = pinned.numpy()
    xy[:] = xy0
    S = args.sweeps_per_step
    sysg.series_reserve(4)

    def step():
        sysg.set_positions(xy)
        sysg.run(1, S, True)
        result = sysg.series()[-1]
        sysg.series_clear()
        return result

    for _ in range(2):  # capture the step graphs of both buffer parities (hd_set_positions swaps them) untimed
        step()
    torch.cuda.synchronize()
    att0 = int(sysg.stats()[0][0])
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    attempts = int(sysg.stats()[0][0]) - att0
    sysg.close()
    return {"value": attempts / dt, "unit": UNIT, "h2d_bytes_per_step": int(xy.nbytes),
            "d2h_bytes_per_step": 8 + 8 + 4 * 8, "input": "the device-timed leg's final configuration, every step"}


def algorithmic_bytes(kernel, N, m, form):
    """Minimum memory traffic of one launch of `kernel`.

    sweep (fused): the state (coordinates, id, cell occupancy) read once and
    written once.  pass: every occupancy byte and every coordinate pair read
    once, the active quarter of the coordinates written back.  rebuild: the
    state read once and written once."""
    coord = 8 if form == "fixed" else 16
    state = N * (coord + 4) + m * m
    if kernel in ("sweep", "rebuild"):
        return 2 * state
    if kernel == "pass":
        return m * m + N * coord + (N // 4) * coord
    return None


def cpu_oracle(args, form, budget_s, threads=1):
    """The CPU oracle on a bounded sample of the workload: sequential (one
    thread), or with each colour's cells shared out between `threads` host
    threads (the OpenMP build of the same oracle, bit-identical chain).
    None when threads > 1 and the compiler has no OpenMP."""
    import oracle
    oracle.build()
    o = oracle.OracleChain(args.N, args.eta, args.delta, args.seed, form=form, cell_min=args.cell_min)
    if threads > 1 and not o.sweep_omp(0, threads):
        return None
    step = (lambda: o.sweep(1)) if threads == 1 else (lambda: o.sweep_omp(1, threads))
    a0, _ = o.stats()
    t0 = time.perf_counter()
    sweeps = 0
    while sweeps < 2 or time.perf_counter() - t0 < budget_s:
        step()
        sweeps += 1
    dt = time.perf_counter() - t0
    a1, _ = o.stats()
    how = "single thread" if threads == 1 else f"OpenMP over each colour's cells, {threads} threads"
    return {"value": (a1 - a0) / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{sweeps} sweeps of the {form} oracle chain at N={args.N}, eta={args.eta}, seed {args.seed} "
                      f"({how}, {dt:.1f} s)"}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# CUDA sources each kernel class is compiled from (a recorded ncu traffic
# figure stays valid while these are unchanged)
KERNEL_SOURCES = {
    "pass": ["hd_sweep.cu", "hd_sweep_cell.cuh", "hd_cell.cuh", "hd_device.cuh", "hd_kernels.h", "hd_exact.cuh"],
    "rebuild": ["hd_sweep.cu", "hd_sweep_cell.cuh", "hd_cell.cuh", "hd_device.cuh", "hd_kernels.h", "hd_exact.cuh"],
    "draws": ["hd_sweep.cu", "hd_device.cuh", "hd_kernels.h", "hd_exact.cuh"],
    "hist": ["hd_measure.cu", "hd_device.cuh", "hd_kernels.h", "hd_exact.cuh"],
    "psi6": ["hd_measure.cu", "hd_device.cuh", "hd_kernels.h", "hd_exact.cuh"],
}


def kernel_sources_hash(kernel=None):
    """First 16 hex digits of the sha256 of the CUDA sources a kernel class is
    built from (all of them when the class is unknown or None), as recorded
    beside ncu counters."""
    import glob
    import hashlib
    d = os.path.join(ROOT, "paper_1211_1645_gb300", "csrc")
    if kernel in KERNEL_SOURCES:
        files = [os.path.join(d, f) for f in KERNEL_SOURCES[kernel]]
    else:
        files = (sorted(glob.glob(os.path.join(d, "*.cu"))) + sorted(glob.glob(os.path.join(d, "*.cuh")))
                 + sorted(glob.glob(os.path.join(d, "*.h"))))
    h = hashlib.sha256()
    for f in files:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def _recorded(kind, kernel, workload):
    """Key=value figures of a `kind` line ("traffic" or "counters") for
    `kernel` on `workload` ("<N>_<form>") in the committed ncu summaries,
    taken on the current kernel sources; None when there is none."""
    import glob
    import re
    want = kernel_sources_hash(kernel)
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            mt = re.match(rf"\s*{kind} (\S+) (.*) workload=(\S+) sources=(\w+)\s*$", line)
            if mt and mt.group(1) == f"k_{kernel}" and mt.group(3) == workload and mt.group(4) == want:
                return {k: float(v) for k, v in (kv.split("=") for kv in mt.group(2).split())}
    return None


def recorded_counters(kernel, workload):
    """Other ncu figures of one launch of `kernel` (L2 and pipe utilisation,
    issue activity, occupancy) from the committed summaries, or None."""
    return _recorded("counters", kernel, workload)


def recorded_traffic(kernel, workload):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu
    summaries, or None."""
    d = _recorded("traffic", kernel, workload)
    return int(d["bytes_per_launch"]) if d else None


_L2_GBS = None


def l2_copy_gbs():
    """Copy bandwidth of data resident in L2, measured here: buffers of 4, 8,
    16 and 24 MB copied into a second buffer of the same size (at most 48 MB
    in all, well inside the 129 MB L2) 200 times after a warm-up; read +
    write bytes over the CUDA-event time, the best of the sizes.  The
    denominator of the L2 roof."""
    global _L2_GBS
    if _L2_GBS is None:
        import torch
        best = 0.0
        for mb in (4, 8, 16, 24):
            n = mb << 20
            a = torch.ones(n, dtype=torch.uint8, device="cuda")
            b = torch.empty_like(a)
            for _ in range(20):
                b.copy_(a)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(200):
                b.copy_(a)
            e1.record()
            torch.cuda.synchronize()
            best = max(best, 2 * n * 200 / (e0.elapsed_time(e1) / 1e3) / 1e9)
            del a, b
        _L2_GBS = best
    return _L2_GBS


def roofline(per, nl, scale, ms_step, N, m, form, clocks, workload):
    """Roofline of the dominant kernel class of a step.

    Its in-step time per launch t is the profiled in-graph time, scaled by
    `scale` (in_step_times).  Three roofs:
      hbm    algorithmic bytes per launch / t against the measured HBM copy
             bandwidth (MEASURED_PEAKS.json);
      l2     the same bytes / t against the L2-resident copy bandwidth
             measured by l2_copy_gbs;
      issue  warp instructions per launch (committed ncu counters) / t
             against one warp instruction per cycle per scheduler:
             SMs x 4 x the median SM clock sampled during the timed steps.
    The binding roof ("bound") is the one the committed ncu counters of the
    kernel show closest to saturation (DRAM %, L2 %, issue-active %); the
    top-level achieved / peak / frac are that roof's."""
    import torch
    top = max(per, key=lambda k: per[k])
    t_s = per[top] * scale / max(1.0, nl[top]) / 1e3
    alg = algorithmic_bytes(top, N, m, form)
    hbm_peak, peak_kind = peaks()
    out = {"kernel": top, "launches_per_step": nl[top], "in_step_us": t_s * 1e6, "time_scale": scale,
           "algorithmic_bytes_per_launch": alg, "peak_kind": peak_kind,
           "traffic": recorded_traffic(top, workload), "ncu": recorded_counters(top, workload)}
    hbm = l2 = issue = None
    if alg and t_s > 0:
        a = alg / t_s / 1e9
        hbm = {"achieved": a, "peak": hbm_peak, "unit": "GB/s", "frac": a / hbm_peak, "peak_kind": peak_kind}
        lp = l2_copy_gbs()
        l2 = {"achieved": a, "peak": lp, "unit": "GB/s", "frac": a / lp, "peak_kind": "measured L2 copy"}
    cnt = out["ncu"]
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz")
    if cnt and cnt.get("warp_instructions") and mhz and t_s > 0:
        a = cnt["warp_instructions"] / t_s / 1e9
        p = sms * 4 * mhz * 1e6 / 1e9
        issue = {"achieved": a, "peak": p, "unit": "G warp-instructions/s", "frac": a / p,
                 "peak_kind": f"{sms} SMs x 4 schedulers x {mhz:.0f} MHz (sampled)"}
    bound = "hbm"
    if cnt:
        cands = {"hbm": cnt.get("dram_pct", 0.0), "l2": cnt.get("l2_pct", 0.0), "alu": cnt.get("issue_active_pct", 0.0)}
        bound = max(cands, key=cands.get)
        if bound == "alu" and issue is None:
            bound = "hbm"
    prim = {"hbm": hbm, "l2": l2, "alu": issue}[bound] or hbm
    out.update({"bound": bound, "achieved": prim and prim["achieved"], "peak": prim and prim["peak"],
                "unit": prim and prim["unit"], "frac": prim and prim["frac"], "hbm": hbm, "l2": l2, "issue": issue})
    return out


def time_config5(args, rank, world, dev):
    """The state larger than L2: N = 2048^2 at eta = 0.720 from the
    shifted-row lattice, fixed point, one step = 250 sweeps + the pressure,
    the global Psi_6 and the local psi_j field kept on the device; its own
    roofline (HBM is the binding roof once the state exceeds L2)."""
    N, eta, S = 2048 * 2048, 0.720, 250
    steps = max(2, args.steps // 20)
    import torch
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    r = time_form(args, "fixed", rank, world, steps, 2, sampler, N=N, eta=eta, lattice="triangular", sweeps=S,
                  measure=2)
    t, a = reduce_max_sum(world, r["ms"], float(r["attempts"]), dev)
    ms_step = t / steps
    per, nl, ksum, scale = in_step_times(r, ms_step)
    geo = r["geometry"]
    return {"value": a / (t / 1e3), "unit": UNIT, "ms_per_step": ms_step, "steps": steps, "warmup": 2,
            "config": f"N={N}, eta={eta}, shifted-row start, fixed form, {S} sweeps + pressure, Psi_6 and the "
                      "local psi_j field per step; L2 flushed before each step",
            "cells_per_side": geo["m"], "kernel_ms_per_step": {k: v * scale for k, v in per.items()},
            "kernel_event_ms_per_step": per,
            "clocks": r["clocks"],
            "roofline": roofline(per, nl, scale, ms_step, N, geo["m"], "fixed", r["clocks"], f"{N}_fixed")}


def run_ours(args):
    import torch
    rank, world, local = dist_setup(args)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU; use --impl reference for the CPU oracle")
    import paper_1211_1645_gb300 as hd
    hd.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    main = time_form(args, args.form, rank, world, args.steps, args.warmup, sampler, lattice=args.lattice,
                     keep_positions=not args.no_e2e)
    tmax, att_sum = reduce_max_sum(world, main["ms"], float(main["attempts"]), dev)
    value = att_sum / (tmax / 1e3)
    fp64 = None
    if not args.no_fp64 and args.form != "fp64":
        s64 = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
        steps64 = max(1, args.steps // 2)
        r = time_form(args, "fp64", rank, world, steps64, max(3, args.warmup), s64, lattice=args.lattice)
        t64, a64 = reduce_max_sum(world, r["ms"], float(r["attempts"]), dev)
        p64, n64, _, sc64 = in_step_times(r, t64 / steps64)
        fp64 = {"value": a64 / (t64 / 1e3), "ms_per_step": t64 / steps64, "steps": steps64,
                "kernel_ms_per_step": {k: v * sc64 for k, v in p64.items()}, "clocks": r["clocks"],
                "roofline": roofline(p64, n64, sc64, t64 / steps64, args.N, r["geometry"]["m"], "fp64", r["clocks"],
                                     f"{args.N}_fp64")}
    # the sweep loop alone (rebuild + four colour passes per sweep), same timing
    so = time_form(args, args.form, rank, world, max(1, args.steps // 2), 2, measure=0)
    tso, aso = reduce_max_sum(world, so["ms"], float(so["attempts"]), dev)
    sweeps_only = {"value": aso / (tso / 1e3), "unit": UNIT, "ms_per_step": tso / max(1, args.steps // 2),
                   "config": f"{args.sweeps_per_step} sweeps per step, no measurement"}
    e2e = None
    if not args.no_e2e:
        e2e = time_e2e(args, args.form, rank, max(1, args.steps // 2), main["final_xy"])
    extras = None if args.no_extras else time_extras(args, rank, world, dev)
    c5 = None if args.no_extras else time_config5(args, rank, world, dev)
    if rank != 0:
        return
    geo = main["geometry"]
    ms_step = tmax / args.steps
    per, nl, ksum, scale = in_step_times(main, ms_step)
    assert abs(ksum * scale - ms_step) <= 1e-9 * ms_step  # the classes' in-step times fill the step exactly
    roof = roofline(per, nl, scale, ms_step, args.N, geo["m"], args.form, main["clocks"], f"{args.N}_{args.form}")
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": tmax / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32" if args.form == "fixed" else "f64",
        "data": "synthetic",
        "config": {"workload": f"MPMC hard disks N={args.N} eta={args.eta} delta={args.delta}, "
                               f"{args.form} form, {args.sweeps_per_step} sweeps + 1 pressure/psi6 measurement per step",
                   "N": args.N, "eta": args.eta, "sweeps_per_step": args.sweeps_per_step, "cells_per_side": geo["m"],
                   "trials_per_cell": geo["trials_per_cell"], "cell_side": geo["w"],
                   "acceptance": main["acceptance"], "l2": "flushed before each timed step (256 MB write)",
                   "graph_branches": geo["graph_branches"],
                   "parallelism": f"replicas{world}"},
        "roofline": roof,
        "gpu_launches": main["launches"],
        "clocks": main["clocks"],
        "kernel_ms_per_step": {k: v * scale for k, v in per.items()},
        "kernel_event_ms_per_step": per,
        "last_measurement": dict(zip(["betaP_over_rho", "g_contact", "psi6_re", "psi6_im"],
                                     main["last_measurement"] or [])),
        "sweeps_only": sweeps_only,
        "fp64": fp64,
        "e2e": e2e,
    }
    if extras:
        line.update(extras)
    if c5:
        line["config5"] = c5
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_oracle(args, args.form, args.cpu_seconds)
        allc = cpu_oracle(args, args.form, args.cpu_seconds, threads=host_cores()) if host_cores() > 1 else None
        if allc:
            line["cpu_baseline_all_cores"] = allc
    print(json.dumps(line), flush=True)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    t0 = time.perf_counter()
    per = []
    # each step is a bounded sample; the whole run takes about 3 x --cpu-seconds
    total_budget = max(1.0, 3.0 * args.cpu_seconds / max(1, args.steps + args.warmup))
    for k in range(args.warmup + args.steps):
        r = cpu_oracle(args, args.form, total_budget)
        if k >= args.warmup:
            per.append(r)
    value = statistics.mean(r["value"] for r in per)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": (time.perf_counter() - t0) * 1e3 / max(1, args.steps + args.warmup),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32" if args.form == "fixed" else "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": f"MPMC hard disks N={args.N} eta={args.eta} delta={args.delta}, {args.form} form "
                               f"(CPU oracle, bounded sample per step)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": per[-1]["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
