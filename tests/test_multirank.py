"""Multi-process path of the benchmark on CPU: every rank labels its own
scene (replicas, no collective on the data path); the job rate is the sum of
the ranks' pixels over the slowest rank's time.  Two gloo ranks."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import numpy as np
    import oracle
    import synth
    # each rank labels its own small scene with the oracle (stand-in for the
    # GPU step) and reports elapsed time and pixels
    img, _ = synth.scene(64 + 32 * rank, 96, 100 + rank, n_floes=3)
    _, counts, _, _ = oracle.label(img)
    elapsed = 1.0 + rank          # rank 1 is the slow one
    el, units = bench.aggregate(elapsed, float(img.shape[0] * img.shape[1]), world)
    # the class counts of the two replicas sum on the host, no device collective
    t = torch.tensor([int(c) for c in counts], dtype=torch.int64)
    dist.all_reduce(t)
    q.put((rank, el, units, t.tolist(), int(counts.sum())))
    dist.destroy_process_group()


def test_two_rank_aggregation():
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
    (r0, el0, u0, c0, n0), (r1, el1, u1, c1, n1) = res
    assert el0 == el1 == 2.0                  # max over ranks
    assert u0 == u1 == 64 * 96 + 96 * 96      # sum over ranks
    assert c0 == c1 and sum(c0) == n0 + n1


def test_oracle_pool_baseline():
    """The multi-core CPU baseline: spawned oracle workers share the scene and
    each labels its own whole chips; every chip is labelled at most once."""
    sys.path.insert(0, ROOT)
    import bench
    import synth
    img, _ = synth.scene(600, 520, 7, n_floes=4)
    pool = bench.OraclePool(img, cores=2)
    try:
        v, sample = pool.run(budget_s=0.2, seed=3)
    finally:
        pool.close()
    assert v > 0
    assert "on 2 worker processes" in sample
    n = int(sample.split()[0])
    assert 2 <= n <= 9      # 3 x 3 chips, at least one per worker
