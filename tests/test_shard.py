"""Query sharding over ranks: the host logic with two gloo ranks on CPU, and
the property that makes it exact (a query's walk depends on its global query
id only), checked on the oracle."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2404_08364_gb300.shard import reduce_scalar, shard_range


def test_shard_ranges_partition():
    for total in (0, 1, 7, 1000, 2**20 + 3):
        for world in (1, 2, 3, 8):
            got = [shard_range(total, r, world) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == total
            assert all(got[i][1] == got[i + 1][0] for i in range(world - 1))
            sizes = [e - b for b, e in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b, e = shard_range(1000, rank, world)
    mx = reduce_scalar(float(rank * 10 + 1), "max")
    sm = reduce_scalar(float(e - b), "sum")
    out[rank] = (b, e, mx, sm)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][:2] == (0, 500) and out[1][:2] == (500, 1000)
    assert out[0][2] == out[1][2] == 11.0     # max over ranks
    assert out[0][3] == out[1][3] == 1000.0   # all queries counted once


def test_sharded_walks_equal_one_walk(orc):
    import tiny_graphs as tg
    g = tg.random_small(12, 0.4, seed=4)
    starts = np.arange(g.n).repeat(9).astype(np.int32)
    prm = orc.Params(p=2.0, q=0.5)
    full, flen = orc.walk_exact(orc.CSR(g), "node2vec", prm, starts, 25, 11)
    parts = []
    for r in range(3):
        b, e = shard_range(len(starts), r, 3)
        parts.append(orc.walk_exact(orc.CSR(g), "node2vec", prm, starts[b:e], 25, 11, q0=b))
    assert np.array_equal(np.concatenate([p for p, _ in parts]), full)
    assert np.array_equal(np.concatenate([l for _, l in parts]), flen)
