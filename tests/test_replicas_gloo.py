"""The N > 1 replica path on CPU: two gloo ranks, each with its own timing,
agree on the max-over-ranks time and the whole-job throughput; problems are
sharded round-robin with no overlap."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2504_10710_gb300 import replicas
    r, w = replicas.rank_world()
    replicas.barrier(w)
    secs = 0.010 * (r + 1)                       # rank 1 is the slower replica
    value = replicas.aggregate_throughput(263169.0, secs, w)
    mine = replicas.shard(list(range(10)), r, w)
    out.put((r, value, replicas.max_over_ranks(secs, w), mine))
    replicas.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time_and_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, v0, m0, s0), (r1, v1, m1, s1) = res
    assert m0 == m1 == pytest.approx(0.020)
    assert v0 == v1 == pytest.approx(2 * 263169.0 / 0.020)
    assert sorted(s0 + s1) == list(range(10)) and not set(s0) & set(s1)
