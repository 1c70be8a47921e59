"""Multi-process (world_size 2, gloo on CPU) checks of the replica helpers the
benchmark and serving loop use: round-robin sharding with no overlap or gap,
and the max/sum of per-rank values that the driver's timing relies on."""
import os
import socket

import torch.multiprocessing as mp

from paper_2602_03529_b300 import replicas as R


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    R.init("gloo")
    mine = R.shard(11, rank, world)
    R.barrier()
    mx = R.max_over_ranks(10.0 * (rank + 1))
    sm = R.sum_over_ranks(len(mine))
    q.put((rank, mine, mx, sm))
    R.finalize()


def test_two_rank_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, m0, c0), (r1, s1, m1, c1) = res
    assert sorted(s0 + s1) == list(range(11)) and not set(s0) & set(s1)
    assert m0 == m1 == 20.0
    assert c0 == c1 == 11


def test_single_process_defaults():
    assert R.shard(5, 0, 1) == [0, 1, 2, 3, 4]
    assert R.max_over_ranks(3.5) == 3.5
