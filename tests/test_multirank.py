"""The bench's N > 1 path on CPU: two gloo ranks run the replica collectives (barrier,
maximum of the ranks' times) and the whole-job rate; the reference arm runs on rank 0 only.
No GPU and no CUDA call."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.rank_barrier(world)
        ms = 10.0 + 5.0 * rank                     # the second rank is slower
        mx = bench.rank_max(ms, world)
        q.put((rank, mx, bench.replica_rate(1000, 4, world, mx)))
    finally:
        dist.destroy_process_group()


def test_replica_collectives_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]               # both see the slowest rank
    assert out[0][2] == pytest.approx(2 * 1000 * 4 / 15e-3)  # units of both ranks / slowest


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    bench.rank_barrier(1)
    assert bench.rank_max(3.5, 1) == 3.5
    assert bench.replica_rate(10, 2, 1, 4.0) == pytest.approx(5000.0)


def test_reference_arm_runs_on_rank0_only():
    """Under torchrun the other ranks exit 0 without work or output."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_line_on_rank0():
    """The reference arm (the oracle on the host cores) prints one JSON line with the
    contract's keys; a small spacing keeps the CPU work short."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--l0", "0.025"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "particle-steps/s"
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["higher_is_better"] is True
