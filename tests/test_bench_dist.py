"""The multi-rank (replica) path of bench.py on CPU: world_size 2 over gloo.
Every rank runs its own replica; the job time is the slowest rank's and the
job rate counts every rank's moves.  The reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, l = bench.dist_env()
        ms = bench.job_ms(10.0 * (rank + 1), w)   # rank 1 is the slow one
        q.put((r, w, l, ms, bench.job_value(ms, w)))
    finally:
        dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    port = free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, (r, w, l, ms, v) in enumerate(out):
        assert (r, w, l) == (rank, 2, rank)
        assert ms == 20.0                     # MAX over ranks
        assert v == pytest.approx(2 * 1e3 / 20.0)


def test_reference_arm_prints_on_rank0_only(tmp_path):
    """Under torchrun the reference arm runs on rank 0; rank 1 exits 0
    without work.  Launched as two ranks with a tiny step count."""
    port = free_port()
    env = dict(os.environ, PYTHONPATH=ROOT)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env, cwd=str(tmp_path))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["cpu_baseline"]["kind"] == "oracle"


def _part_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = __import__("numpy").random.default_rng(5)
        costs = [float(x) for x in rng.uniform(1.0, 50.0, size=64) ** 2]
        mine = bench.batch_partition(costs, world)[rank]
        # every rank's share, gathered only to check it (the bench exchanges
        # no data: each rank derives its share from the same costs)
        got = [None] * world
        dist.all_gather_object(got, mine)
        load = sum(costs[i] for i in mine)
        ms = bench.job_ms(load, world)      # time proportional to the share
        q.put((rank, got, load, ms, costs))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_batch_partition_over_ranks(world):
    """The batch of independent contractions is split over the ranks with
    no exchange: every contraction lands on exactly one rank, the shares
    are balanced to within the largest contraction, and the job time is
    the largest share's."""
    port = free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_part_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    shares, costs = out[0][1], out[0][4]
    for r in range(world):
        assert out[r][1] == shares                      # every rank derives the same split
    flat = sorted(i for s in shares for i in s)
    assert flat == list(range(len(costs)))               # each contraction exactly once
    loads = [sum(costs[i] for i in s) for s in shares]
    assert max(loads) - min(loads) <= max(costs)
    for r in range(world):
        assert out[r][3] == pytest.approx(max(loads))    # job time: the slowest share
