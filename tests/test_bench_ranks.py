"""Bench host logic on CPU. Multi-rank aggregation (gloo, world_size 2): each
rank runs its own replica; the job's step time is the slowest rank's and the
value sums the units of all ranks. The clock record: samples inside the timed
region, their median SM clock and the throttle reasons seen there. The
reference arm's JSON line (the CPU oracle, timed on a short run)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = [10.0, 25.0][rank]
    out = bench.aggregate_over_ranks(ms, 1000.0)
    q.put((rank, out))
    dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        ms, value = res[r]
        assert ms == 25.0
        assert abs(value - 2 * 1000.0 / 25e-3) < 1e-6


def test_aggregate_single_rank():
    import bench
    ms, value = bench.aggregate_over_ranks(20.0, 500.0)
    assert ms == 20.0 and abs(value - 500.0 / 20e-3) < 1e-9


# ---------------------------------------------------------------- clock record
def _row(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", pcap="Not Active"):
    return ["0", str(sm), str(mx), "900.0", "0x0", hw, hwt, swt, pcap]


def test_clock_summary_window_median_and_reasons():
    """The clock record keeps the samples inside the timed region (0.15 s of
    slack each side), reports their median SM clock, the maximum clock and
    every throttle reason seen active there."""
    import bench
    c = bench.ClockSampler(0)
    c.rows = [(9.0, _row(900, 2070, hw="Active")),     # before the region: dropped
              (10.0, _row(2070, 2070)),
              (10.1, _row(1980, 2070, pcap="Active")),
              (10.2, _row(2055, 2070)),
              (10.45, _row(600, 2070, hwt="Active"))]   # after the region: dropped
    c.t0, c.t1 = 10.0, 10.25
    s = c.summary()
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    c.t1 = 10.35  # the late sample now falls inside the slack
    assert c.summary()["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_summary_unsampled():
    import bench
    c = bench.ClockSampler(0)
    c.t0, c.t1 = 1.0, 2.0
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}


# ---------------------------------------------------------------- reference arm
def test_reference_arm_json_line():
    """`--impl reference` times the CPU oracle and prints one JSON line with
    the GPU arm's metric, unit and workload, a cpu_baseline of the oracle and
    an e2e record without host-device traffic (a short run of two schemes)."""
    import json
    import subprocess
    import sys
    import bench
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                          "--schemes", "MEG6,LAD_E4"], cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "cell-updates/s"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["value"] > 0 and abs(d["ms_per_step"] - bench.CPU_SAMPLE[0] * bench.CPU_SAMPLE[1] * 2 / d["value"] * 1e3) <= 1e-6 * d["ms_per_step"]
    assert d["config"]["workload"] == bench.bench_config(["MEG6", "LAD_E4"], 1)["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == os.cpu_count() and cb["value"] == d["value"] and cb["sample"]
    assert cb["cpu_model"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
