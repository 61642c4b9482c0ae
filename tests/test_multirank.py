"""The multi-GPU logic of bench.py on CPU: two gloo ranks.  Frames are sharded
by rank with no data-path collective; only the timing (max over ranks) and
the frame count (sum) are reduced."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import workloads as W

        seed = bench.rank_seed(rank)
        # each rank's frames come from its own seed: disjoint streams
        msg = W.message_bits(seed, 4, 16)
        t = bench.reduce_max(1.0 + rank, world)
        n = bench.reduce_sum(10.0 * (rank + 1), world)
        bench.barrier(world)
        q.put((rank, seed, msg.tobytes(), t, n))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    (r0, s0, m0, t0, n0), (r1, s1, m1, t1, n1) = res
    assert s0 != s1 and m0 != m1          # different frames per rank
    assert t0 == t1 == 2.0                # slowest rank's time
    assert n0 == n1 == 30.0               # frames of all ranks


def test_single_rank_reductions_are_identity():
    import bench

    assert bench.reduce_max(3.5, 1) == 3.5 and bench.reduce_sum(7.0, 1) == 7.0
    bench.barrier(1)
