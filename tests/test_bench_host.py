"""Host-side logic of bench.py without a GPU: the multi-rank reduction used
under torchrun (world size 2, gloo, on CPU), the reference arm (the CPU
oracle) and the JSON contract of its line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


WORKER = r'''
import os, sys, json
sys.path.insert(0, os.environ["ROOT"])
import torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="env://")
rank, world = dist.get_rank(), dist.get_world_size()
bench.barrier(world)
tmax, tsum = bench.reduce_max_sum(world, 10.0 * (rank + 1), 100.0 + rank, "cpu")
print(json.dumps({"rank": rank, "tmax": tmax, "tsum": tsum}), flush=True)
dist.destroy_process_group()
'''


def test_two_rank_reduction_gloo(tmp_path):
    """Max of the step time and sum of the attempts over ranks, as rank 0
    reports them for weak scaling over independent replicas."""
    script = tmp_path / "worker.py"
    script.write_text(WORKER)
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, ROOT=ROOT, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                   WORLD_SIZE="2", LOCAL_RANK=str(rank))
        procs.append(subprocess.Popen([sys.executable, str(script)], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=180) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    res = [json.loads(o.strip().splitlines()[-1]) for o, _ in outs]
    for r in res:
        assert r["tmax"] == 20.0 and r["tsum"] == 201.0


def test_reference_arm_prints_contract_line():
    """--impl reference times the CPU oracle on a bounded sample and prints
    one JSON line with impl, cpu_baseline and e2e."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--N", "4096",
                          "--eta", "0.7", "--steps", "1", "--warmup", "0", "--cpu-seconds", "0.5"], capture_output=True, text=True,
                         timeout=300, env=dict(os.environ, RANK="0"))
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["unit"] == "trial moves/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["higher_is_better"] is True


def test_reference_arm_other_ranks_exit_quietly():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--N", "1024",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=120,
                         env=dict(os.environ, RANK="1"))
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_algorithmic_bytes():
    sys.path.insert(0, ROOT)
    import bench
    N, m = 1 << 20, 1072
    assert bench.algorithmic_bytes("sweep", N, m, "fixed") == 2 * (N * 12 + m * m)
    assert bench.algorithmic_bytes("pass", N, m, "fixed") == m * m + N * 8 + (N // 4) * 8
    assert bench.algorithmic_bytes("pass", N, m, "fp64") == m * m + N * 16 + (N // 4) * 16


def test_recorded_profile_figures_follow_kernel_sources(tmp_path, monkeypatch):
    """Traffic and counter lines of a profile summary are used only while the
    kernel's sources hash to the value recorded beside them."""
    import shutil
    sys.path.insert(0, ROOT)
    import bench
    src = os.path.join(ROOT, "paper_1211_1645_gb300", "csrc")
    dst = tmp_path / "paper_1211_1645_gb300" / "csrc"
    shutil.copytree(src, dst, ignore=shutil.ignore_patterns("*.o", "*.so"))
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_sources_hash("pass")
    (tmp_path / "profiles" / "k.md").write_text(
        "text\n"
        f"    traffic k_pass bytes_per_launch=999 workload=4194304_fixed sources={h}\n"
        f"    traffic k_pass bytes_per_launch=123 workload=1048576_fixed sources={h}\n"
        f"    counters k_pass l2_pct=14.5 issue_active_pct=45.25 workload=1048576_fixed sources={h}\n"
        "    traffic k_rebuild bytes_per_launch=456 workload=1048576_fixed sources=0000000000000000\n")
    w = "1048576_fixed"
    assert bench.recorded_traffic("pass", w) == 123
    assert bench.recorded_traffic("pass", "4194304_fixed") == 999
    assert bench.recorded_traffic("pass", "1048576_fp64") is None
    assert bench.recorded_counters("pass", w) == {"l2_pct": 14.5, "issue_active_pct": 45.25}
    assert bench.recorded_traffic("rebuild", w) is None
    assert bench.recorded_counters("rebuild", w) is None
    # a changed source invalidates the recorded figures
    with open(dst / "hd_sweep.cu", "a") as f:
        f.write("\n// changed\n")
    assert bench.recorded_traffic("pass", w) is None
    assert bench.recorded_counters("pass", w) is None


def test_in_step_times_fill_the_step():
    """Each kernel class is charged its share of the profiled event times x
    the graph-timed step, so the classes add up to ms_per_step whichever way
    the event times over- or under-shoot it."""
    sys.path.insert(0, ROOT)
    import bench
    run = {"kernel_times": {"pass": (8.0, 800), "rebuild": (2.0, 200), "psi6": (0.4, 2), "hist": (0.0, 0)}}
    for ms_step in (4.0, 20.0):
        per, n, total, scale = bench.in_step_times(run, ms_step)
        assert set(per) == {"pass", "rebuild", "psi6"} and n["pass"] == 400
        assert abs(sum(v * scale for v in per.values()) - ms_step) < 1e-12
        assert abs(per["pass"] * scale / n["pass"] - ms_step * 8.0 / 10.4 / 400) < 1e-15


def test_roofline_picks_the_binding_roof(monkeypatch):
    """The top-level roof is the one the committed counters show closest to
    saturation: issue (alu) when issue-active leads, HBM when DRAM leads;
    the rates follow from the in-step time per launch."""
    sys.path.insert(0, ROOT)
    import bench
    torch = pytest.importorskip("torch")

    class Props:
        multi_processor_count = 152

    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d: Props())
    monkeypatch.setattr(bench, "l2_copy_gbs", lambda: 8000.0)
    monkeypatch.setattr(bench, "peaks", lambda: (6800.0, "measured"))
    monkeypatch.setattr(bench, "recorded_traffic", lambda k, w: 123)
    counters = {"dram_pct": 20.0, "l2_pct": 13.0, "issue_active_pct": 41.0, "warp_instructions": 5.0e6}
    monkeypatch.setattr(bench, "recorded_counters", lambda k, w: dict(counters))
    per, nl = {"pass": 5.0, "rebuild": 1.0}, {"pass": 400.0, "rebuild": 100.0}
    N, m = 1 << 20, 1072
    r = bench.roofline(per, nl, 0.7, 4.2, N, m, "fixed", {"sm_mhz": 2000.0}, "x")
    t = 5.0 * 0.7 / 400 / 1e3
    assert r["kernel"] == "pass" and r["bound"] == "alu"
    assert abs(r["issue"]["achieved"] - 5.0e6 / t / 1e9) < 1e-6
    assert abs(r["issue"]["peak"] - 152 * 4 * 2000.0 * 1e6 / 1e9) < 1e-9
    alg = bench.algorithmic_bytes("pass", N, m, "fixed")
    assert alg == m * m + N * 8 + (N // 4) * 8
    assert abs(r["hbm"]["achieved"] - alg / t / 1e9) < 1e-6 and r["frac"] == r["issue"]["frac"]
    counters.update(dram_pct=60.0)
    r = bench.roofline(per, nl, 0.7, 4.2, N, m, "fixed", {"sm_mhz": 2000.0}, "x")
    assert r["bound"] == "hbm" and r["frac"] == r["hbm"]["frac"] and r["traffic"] == 123
