"""The N > 1 path of the benchmark on CPU: the path shards into independent
replicas (one seeded instance per rank, no collective on the data path), so
the only exchange is the final MAX over ranks of the timed region.  Two
gloo ranks on 127.0.0.1 check that exchange and the whole-job totals, and
that ranks draw distinct instances of the same workload shape."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dev_ms, e2e_ms = 10.0 + 5.0 * rank, 12.0 + 1.0 * rank
        res = bench.replica_totals(dev_ms, e2e_ms, vox_step=1000, steps=3, world=world, dist=dist, device="cpu")
        out.put((rank, res))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_totals_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        dev_ms, e2e_ms, value, e2e_val = res[r]
        assert dev_ms == 15.0 and e2e_ms == 13.0            # slowest rank
        assert value == pytest.approx(1000 * 3 * 2 / 0.015)  # all ranks' voxels / max time
        assert e2e_val == pytest.approx(1000 * 3 * 2 / 0.013)


def test_single_rank_totals_without_collective():
    import bench
    dev_ms, e2e_ms, value, e2e_val = bench.replica_totals(20.0, 25.0, vox_step=500, steps=4, world=1)
    assert (dev_ms, e2e_ms) == (20.0, 25.0)
    assert value == pytest.approx(500 * 4 / 0.020)


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_ranks_get_distinct_instances_of_one_shape(name):
    """Weak scaling: every rank denoises its own seeded instance of the same
    workload (same shape and parameters, different draws)."""
    import bench
    (j0,), _ = bench.workload(name, 0)
    (j1,), _ = bench.workload(name, 1)
    assert j0.y.shape == j1.y.shape and j0.cfg == j1.cfg
    assert not np.array_equal(j0.y, j1.y)
