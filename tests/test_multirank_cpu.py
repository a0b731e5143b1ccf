"""The multi-rank (N > 1) path of the benchmark on CPU: two gloo ranks.

Cells are independent, so N GPUs run N disjoint shares of one global batch with no collective on
the data path; the only collective is the max over ranks of the timings (the job ends with its
slowest rank).  Checked here with the same helpers the benchmark uses: the shares of the two
ranks are disjoint, cover the global batch in order, and both ranks see the slower rank's time.
"""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    from paper_2607_13740_b300 import workloads as W
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sh = W.shard(W.batched_additive(n_cells=64 * world), rank, world)
        ms = 10.0 + 5.0 * rank                  # rank 1 is the slower one
        q.put((rank, sh.n_cells, sh.ic_params.tolist(), sh.dt.tolist(), bench.max_over_ranks(ms, world, "cpu")))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_cells_and_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    from paper_2607_13740_b300 import workloads as W
    full = W.batched_additive(n_cells=64 * world)
    ic = np.concatenate([np.array(o[2]) for o in out])
    dt = np.concatenate([np.array(o[3]) for o in out])
    assert [o[1] for o in out] == [64, 64]
    np.testing.assert_array_equal(ic, full.ic_params)
    np.testing.assert_array_equal(dt, full.dt)
    assert [o[4] for o in out] == [15.0, 15.0]


def test_shard_rejects_bad_arguments():
    import pytest
    from paper_2607_13740_b300 import workloads as W
    wl = W.batched_additive(n_cells=10)
    with pytest.raises(ValueError):
        W.shard(wl, 2, 2)
    with pytest.raises(ValueError):
        W.shard(wl, 0, 3)
