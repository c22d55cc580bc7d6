"""The N > 1 path on CPU: two gloo ranks, one process each, as torchrun launches
the bench (RANK / LOCAL_RANK / WORLD_SIZE / MASTER_* from the environment).

Each rank reconciles its own block (weak scaling: its data seed is offset by
1000 * rank, so the blocks are disjoint); the only exchange is the final
reduction -- counters summed, times maxed over ranks -- checked here.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    import synth
    r, w, local = bench.rank_env()
    dist.init_process_group("gloo", init_method="env://")
    # each rank's own block: first samples of its seeded data
    x, _ = synth.gaussian_pair(bench.DATA_SEED[3.0] + 1000 * r, 8, 3.0)
    sums, maxes = bench.reduce_over_ranks([10.0 * (r + 1), 1.0], [5.0 + r, 2.0 * (w - r)], "cpu", w)
    out.put((r, w, local, x.tolist(), sums, maxes))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, x0, s0, m0), (r1, w1, l1, x1, s1, m1) = res
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert not np.allclose(x0, x1)                 # disjoint blocks
    assert s0 == s1 == [30.0, 2.0]                 # summed counters, identical on both ranks
    assert m0 == m1 == [6.0, 4.0]                  # max over ranks


def test_single_rank_reduction_is_identity():
    import bench
    assert bench.reduce_over_ranks([3.0, 4.0], [1.5], "cpu", 1) == ([3.0, 4.0], [1.5])
