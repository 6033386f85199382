"""The N > 1 paths on CPU with the gloo backend (world size 2): the batch shards its
independent instances across ranks with no data exchange, the bench takes the maximum time
over ranks, and `bench.py --impl reference` under torchrun prints one line from rank 0."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    import synthetic
    from paper_2109_02598_gb300.batch import shard_instances
    specs = synthetic.batch_instances(512, seed=4)
    sizes = [s["n"] ** 2 for s in specs]
    mine = shard_instances(sizes, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    tmax = bench._max_over_ranks(float(rank + 1), world)
    if rank == 0:
        q.put((gathered, tmax, sizes))
    dist.barrier()
    dist.destroy_process_group()


def test_batch_shards_partition_the_instances_and_balance_sites():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, tmax, sizes = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    allidx = sorted(gathered[0] + gathered[1])
    assert allidx == list(range(512))  # every instance exactly once
    loads = [sum(sizes[i] for i in g) for g in gathered]
    assert abs(loads[0] - loads[1]) <= max(sizes)  # balanced to within one instance
    assert tmax == 2.0  # the bench reports the slowest rank


def test_shard_is_deterministic_and_single_rank_takes_all():
    from paper_2109_02598_gb300.batch import shard_instances
    sizes = [5, 9, 9, 1, 7]
    assert shard_instances(sizes, 0, 1) == [0, 1, 2, 3, 4]
    a = shard_instances(sizes, 0, 2)
    b = shard_instances(sizes, 1, 2)
    assert sorted(a + b) == list(range(5)) and a == shard_instances(sizes, 0, 2)
    with pytest.raises(ValueError):
        shard_instances(sizes, 2, 2)


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
