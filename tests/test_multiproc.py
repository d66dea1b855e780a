"""The multi-GPU bench path on CPU: world-size-2 gloo process groups.

The path shards by replication (every rank runs its own copy of the
workload; envs are independent trajectories and nothing is exchanged), so
the only cross-rank step is the timing reduction: the job ends when the
slowest replica does, and the whole-job value counts every rank's units."""
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


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = [3.0, 5.0, 4.0, 1.0][rank]
        m = bench.max_over_ranks(local)
        v = bench.replica_value(world, 100, 4, m)
        q.put((rank, m, v, bench._dist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replica_timing_reduction_gloo(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in ps:
        p.join(60)
        assert p.exitcode == 0
    slowest = max([3.0, 5.0, 4.0, 1.0][:world])
    for rank, (r, m, v, (drank, dworld)) in enumerate(res):
        assert r == rank == drank and dworld == world
        assert m == slowest
        assert v == world * 100 * 4 / slowest


def test_single_process_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.replica_value(1, 10, 3, 2.0) == 15.0


def test_reference_arm_non_zero_rank_exits_quietly():
    # under torchrun only rank 0 runs and prints the reference arm
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--ref-envs", "2"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--ref-envs", "1"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "env-steps/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0


def test_bench_launches_its_own_replicas_gloo():
    # bench.py --gpus 2 outside a launcher starts two ranks itself (the same
    # launcher the GPU run uses); the CPU check reduces stand-in times 0.1 s
    # and 0.2 s over gloo: the job's time is the slower one
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--replica-check"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.strip().splitlines() if x.startswith("{")]
    assert len(lines) == 1                                   # rank 0 alone prints
    line = lines[0]
    assert line["replica_check"] and line["n_gpus"] == 2
    assert abs(line["max_s"] - 0.2) < 1e-12 and abs(line["value"] - 2 * 100 * 2 / 0.2) < 1e-6
