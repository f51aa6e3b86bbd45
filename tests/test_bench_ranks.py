"""The N > 1 host logic of bench.py on CPU: replicas on gloo ranks agree on
the slowest rank's time, the whole-job figure counts every rank's maps, and
the reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.reduce_max(10.0 + 5.0 * rank, dist, "cpu")
        q.put((rank, slowest, bench.ms_per_map(slowest, 3, 8, world)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    # both ranks see rank 1's 15 ms; 2 ranks x 3 steps x 8 maps share it
    assert got == [(0, 15.0, 15.0 / 48), (1, 15.0, 15.0 / 48)]


def test_single_process_needs_no_group():
    assert bench.reduce_max(7.5, None, "cpu") == 7.5
    assert bench.ms_per_map(100.0, 2, 5, 1) == 10.0


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


@pytest.mark.parametrize("warmup", [0, 2])
def test_bench_rejects_short_warmup(warmup):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--warmup", str(warmup)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode != 0 and "warmup" in r.stderr


def test_reference_arm_line_on_rank_zero():
    """The reference arm (the CPU oracle on a bounded ring sample) prints one
    JSON line with the contract's keys and the same workload config object
    as the GPU arm would."""
    import json
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--nside", "16", "--lmax", "32", "--steps", "1", "--warmup", "3",
                        "--ref-rings", "8"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is False and line["value"] > 0

    class Args:
        nside, lmax, nmaps, eps, leaf_cols = 16, 32, 8, 1e-10, 32
    assert line["config"] == bench.workload_config(Args, 1)
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_plan_build_threads_are_shared_between_ranks():
    assert bench.build_threads(1, True) == 0 and bench.build_threads(1, False) == 0
    cores = os.cpu_count() or 1
    assert bench.build_threads(2, False) == max(1, cores // 2)
    assert bench.build_threads(8, True) == 2 * max(1, cores // 8)
