"""The benchmark's host logic on CPU: two gloo ranks (replicas, one medium
each) aggregate the slowest rank's time and the summed pairs, the reference arm
runs on rank 0 only, and the clock sampler's summary reads the median SM clock
and the throttle reasons seen during the timed region."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r: (10 + 5 r) ms for (r + 1) 1e9 pairs
    t, p = bench.reduce_over_ranks(dist, 10.0 + 5.0 * rank, 1e9 * (rank + 1), "cpu")
    q.put((rank, t, p))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_all_pairs():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 15.0, 3e9), (1, 15.0, 3e9)]


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(None, 12.5, 7.0, "cpu") == (12.5, 7.0)


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_clock_summary_reads_median_clock_and_throttle_reasons():
    # nvidia-smi --query-gpu=index,clocks.sm,clocks.max.sm,power.draw,
    # clocks_event_reasons.{active,hw_slowdown,hw_thermal_slowdown,sw_thermal_slowdown,sw_power_cap}
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1980, 2070, 1399.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 1100.5, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line",
               "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.lines = ["0, 1500, 2070, 1400, 0x40, Not Active, Active, Not Active, Not Active"]
    assert c.summary()["reasons"] == ["hw_thermal_slowdown"]
    c.lines = []
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
