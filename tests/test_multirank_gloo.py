"""Multi-process host logic of the sharded path, world size 2 on CPU (gloo).

Each rank tracks its contiguous slice of an ensemble with the oracle (the
tracking is per particle, so the slices are independent); the gathered
slices equal the unsharded result bit for bit, and the throughput reduction
sums the units and takes the maximum time over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2310_00317_gb300 import sharding


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2310_00317_gb300 import inputs as I
    el, ref = I.fodo10()
    p = I.matched_gaussian(el, ref, 301, 2.5e-6, 3e-4, seed=9)
    p["x"][7] = 0.5  # one particle lost by the end-of-turn guard
    lo, hi = sharding.shard_range(301, world, rank)
    o = oracle.track(el, ref, I.subset(p, np.arange(lo, hi)), 40)
    gathered = [None] * world
    dist.all_gather_object(gathered, (lo, hi, {k: o[k] for k in oracle.FLOAT_FIELDS + oracle.INT_FIELDS}))
    units, ms = sharding.reduce_throughput(100 * (rank + 1), 10.0 * (rank + 1))
    if rank == 0:
        out.put((gathered, units, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_range_covers_everything():
    for n in (0, 1, 7, 1000, 999990):
        for w in (1, 2, 3, 8):
            r = [sharding.shard_range(n, w, k) for k in range(w)]
            assert r[0][0] == 0 and r[-1][1] == n
            assert all(r[k][1] == r[k + 1][0] for k in range(w - 1))
            assert max(b - a for a, b in r) - min(b - a for a, b in r) <= 1
    with pytest.raises(ValueError):
        sharding.shard_range(10, 2, 2)


def test_two_ranks_gloo_equal_unsharded():
    import oracle
    from paper_2310_00317_gb300 import inputs as I
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    gathered, units, ms = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    el, ref = I.fodo10()
    p = I.matched_gaussian(el, ref, 301, 2.5e-6, 3e-4, seed=9)
    p["x"][7] = 0.5
    full = oracle.track(el, ref, p, 40)
    for lo, hi, part in gathered:
        for k, v in part.items():
            assert np.array_equal(v, full[k][lo:hi]), k
    assert sum(hi - lo for lo, hi, _ in gathered) == 301
    assert full["state"][7] == -3
    assert units == 300.0 and ms == 20.0
