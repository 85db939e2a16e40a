"""Host logic of the N > 1 path on CPU (gloo, world size 2): distinct per-rank batches,
exact sharding, and the max-over-ranks step time."""
import os

import pytest
import torch.multiprocessing as mp


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2410_17084_b300 import dist as D
    from paper_2410_17084_b300 import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = D.rank_world()
    b = synth.plane_batch(20, seed=D.rank_seed(0, r))
    t = D.max_over_ranks(1.5 + r, dist)
    q.put((r, w, lr, float(b.xyz.sum()), D.shard(101, r, w), t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, s0, sh0, t0), (r1, w1, l1, s1, sh1, t1) = res
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert s0 != s1  # independent batches per rank
    assert sh0 == (0, 51) and sh1 == (51, 101)
    assert t0 == t1 == 2.5  # both ranks see the slowest rank's time


def test_shard_covers_exactly():
    from paper_2410_17084_b300 import dist as D
    for n in (0, 1, 7, 100):
        for w in (1, 2, 3, 8):
            parts = [D.shard(n, r, w) for r in range(w)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
