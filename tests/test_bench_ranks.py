"""Host logic of bench.py's multi-rank path, on CPU.

The GPU run launches one process per GPU under torchrun and reduces over
NCCL; here the same calls run as world size 2 over gloo: the max over ranks
of the timed region, the whole-job rate, and the reference arm, which rank 0
alone runs and prints.  The clock-log parser is checked on sample lines, and
the roofline figures on sample counters.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=2)
    try:
        dist.barrier()
        total_s = bench.max_over_ranks([1.25, 4.0][rank], dist, "cpu")
        out.put((rank, total_s, bench.job_throughput(1000, 5, dist.get_world_size(), total_s)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_world_2_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        rank, total_s, rate = q.get(timeout=180)
        res[rank] = (total_s, rate)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time; the job moved 2 x 5 x 1000 units in it
    assert res[0] == res[1] == (4.0, 2 * 5 * 1000 / 4.0)


def test_single_rank_needs_no_group():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_throughput(128, 10, 1, 2.0) == 640.0


def test_reference_arm_world_2_rank0_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-scale", "8"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["unit"] == "edges/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "edges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.mark.parametrize("lines,expect", [
    (["0, 2070, 2070, 905.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
      "0, 1900, 2070, 1391.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
      "0, 2040, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"],
     {"sm_mhz": 2040.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}),
    (["0, 1500, 2070, 700.0, 0x8, Active, Not Active, Active, Not Active", "garbage", "0, N/A, 2070"],
     {"sm_mhz": 1500.0, "sm_max_mhz": 2070.0, "reasons": ["hw_slowdown", "sw_thermal_slowdown"], "samples": 1}),
    ([], None),
])
def test_clock_log(lines, expect):
    assert bench.parse_clock_log(lines) == expect


def test_roofline_traffic_basis():
    """The roofline's traffic: the R-MAT 26 line takes the ratio captured at
    that scale, other workloads the R-MAT 20 ratio, scaled and said so; the
    fractions are algorithmic bytes (and DRAM bytes) over the kernels' time."""
    st = [{"move_bytes": [200e9, 33.5e9], "ms_move_kernels": [500.0, 140.0]}] * 2
    r = bench.roofline_from(st, 6784.8, "measured", "rmat26")
    assert r["algorithmic_bytes_per_step"] == 233.5e9
    assert r["achieved"] == round(233.5e9 / 0.64 / 1e9, 1)
    assert r["frac"] == round(r["achieved"] / 6784.8, 4)
    assert r["traffic"] == round(233.5e9 * 3.737) and r["traffic_basis"].find("measured") >= 0
    assert r["dram_gbs"] == round(r["traffic"] / 0.64 / 1e9, 1)
    s = bench.roofline_from(st, 6784.8, "measured", "grid")
    assert s["traffic"] == round(233.5e9 * 2.153) and s["traffic_basis"].find("scaled") >= 0
    assert bench.roofline_from([{"move_bytes": [0], "ms_move_kernels": [0.0]}], 6784.8, "measured") is None
