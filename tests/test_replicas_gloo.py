"""Multi-process host logic (world size 2, gloo on CPU, rendezvous on 127.0.0.1).

The multi-GPU path runs independent replicas (or independent instances) with no
data-path collective; what crosses ranks is the benchmark's timing reduction and
the instance split.  Both are checked here with two CPU processes."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")

from paper_1712_10279_gb300 import replicas as R  # noqa: E402
from paper_1712_10279_gb300 import synthetic as S  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = R.rank_world()
        assert (r, w, lr) == (rank, world, rank)
        # timing reduction: slowest rank's time, sum of the work
        ms, units = R.aggregate_throughput(10.0 + 5.0 * rank, 1000.0 * (rank + 1), dist, "cpu")
        # instance split: every rank computes the same split and takes its part
        inst = S.batched_instances(24, seed=11)
        wts = [R.instance_weight(q["n"], q["k"], len(q["edges"])) for q in inst]
        mine = R.shard_instances(wts, world)[rank]
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        out.put((rank, ms, units, gathered))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_and_sharding():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units, gathered in results:
        assert ms == 15.0 and units == 3000.0
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(24))
        assert not set(gathered[0]) & set(gathered[1])


def test_shard_instances_balances_and_is_deterministic():
    w = [9, 7, 6, 5, 4, 3, 2, 2, 1]
    parts = R.shard_instances(w, 3)
    assert parts == R.shard_instances(w, 3)
    assert sorted(i for p in parts for i in p) == list(range(len(w)))
    loads = [sum(w[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(w)
    assert R.shard_instances(w, 1) == [list(range(len(w)))]
    with pytest.raises(ValueError):
        R.shard_instances(w, 0)


def test_single_process_aggregate_is_identity():
    assert R.aggregate_throughput(12.5, 7.0) == (12.5, 7.0)
