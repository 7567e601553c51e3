"""The N-rank path on the CPU: world-size-2 gloo process groups and torchrun.

Cells are independent, so N GPUs run N replicas of the solve on different
batches (weak scaling) with no data-path collective; what crosses ranks is
the benchmark's barrier and the max over ranks of the step time.  These tests
cover that host logic without a GPU: the max reduction, the whole-job rate,
distinct per-rank batches, and the reference arm under torchrun (rank 0
alone prints its line, the other rank exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, q):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        slowest = bench.max_over_ranks(times[rank], world, torch.device("cpu"))
        q.put((rank, slowest, bench.aggregate_rate(1000, world, slowest)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [0.25, 0.4]
    mp.start_processes(_rank_main, args=(2, _free_port(), times, q), nprocs=2, join=True,
                       start_method="spawn")
    got = sorted(q.get(timeout=60) for _ in range(2))
    for rank, slowest, rate in got:
        assert slowest == max(times)
        assert rate == pytest.approx(2 * 1000 / max(times))


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(1.5, 1, None) == 1.5
    assert bench.aggregate_rate(10, 1, 2.0) == 5.0


def test_each_rank_solves_its_own_batch():
    sys.path.insert(0, ROOT)
    import bench
    import synth

    a = synth.make_workload(bench.CONFIG_ID, cells=np.arange(4), seed=bench.shard_seed(0))
    b = synth.make_workload(bench.CONFIG_ID, cells=np.arange(4), seed=bench.shard_seed(1))
    assert bench.shard_seed(0) != bench.shard_seed(1)
    assert not np.array_equal(a.J, b.J)
    np.testing.assert_array_equal(a.C_abs, b.C_abs)  # same grains and grid on every rank


def test_reference_arm_under_torchrun_prints_once():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0", "--cpu-seconds", "0.3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
