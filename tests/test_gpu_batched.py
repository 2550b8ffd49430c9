"""Walks in batches on two streams (fw_walk_batched, Section 5.2 and Eq. 3):
the paths equal the oracle's and one launch over all queries, whatever the
batch size."""

import numpy as np
import pytest
import torch

import fw_inputs as fi
from gpu_common import cached_graph, device_graph

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("algo", ["node2vec", "metapath", "ppr"])
def test_batched_equals_oracle_and_one_launch_exact(orc, algo):
    from paper_2404_08364_gb300 import _fw
    g = cached_graph("rmat", 12, 2)
    dg = device_graph(g)
    n_q, L = 3000, 30
    starts = fi.random_starts(g.n, n_q, 77)
    per_query = (L + 3) * 4
    budget = 2 * 400 * per_query + 17  # 400 queries per batch: 8 batches, the last one short
    paths, plen, bq = dg.walk_batched(algo, starts, L, 9, mode="exact", p=2.0, q=0.5, budget_bytes=budget,
                                      q_id0=1000)
    assert bq == 400 == _fw.lib().fw_batch_size(budget, L)
    ref_p, ref_l = orc.walk_exact(orc.CSR(g), algo, orc.Params(p=2.0, q=0.5), starts, L, 9, q0=1000)
    assert np.array_equal(plen.numpy(), ref_l)
    assert np.array_equal(paths.numpy(), ref_p)
    one_p, one_l = dg.walk(algo, starts.cuda(), L, 9, mode="exact", p=2.0, q=0.5, q_id0=1000)
    assert torch.equal(plen, one_l.cpu())
    assert torch.equal(paths, one_p.cpu())


def test_batched_fast_ragged_lengths_and_stats():
    g = cached_graph("rmat", 14, 2)
    dg = device_graph(g)
    n_q, L = 5000, 40
    starts = fi.random_starts(g.n, n_q, 5)
    lengths = fi.uniform_lengths(n_q, 0, L, 6)
    dg.stats_reset()
    paths, plen, bq = dg.walk_batched("weighted", starts, L, 3, mode="fast", lengths=lengths,
                                      budget_bytes=2 * 777 * (L + 3) * 4)
    st = dg.stats()
    assert bq == 777
    ref_p, ref_l = dg.walk("weighted", starts.cuda(), L, 3, mode="fast", lengths=lengths.cuda())
    assert torch.equal(plen, ref_l.cpu())
    assert torch.equal(paths, ref_p.cpu())
    assert st["walks"] == n_q
    assert st["steps"] == int((plen - 1).sum())


def test_batched_budget_too_small():
    from paper_2404_08364_gb300._fw import FwError
    g = cached_graph("rmat", 10, 2)
    dg = device_graph(g)
    with pytest.raises(FwError):
        dg.walk_batched("weighted", fi.random_starts(g.n, 10, 1), 80, 1, budget_bytes=100)


def test_batched_reports_out_of_range_starts():
    from paper_2404_08364_gb300 import _fw
    g = cached_graph("rmat", 10, 2)
    dg = device_graph(g)
    starts = fi.random_starts(g.n, 500, 2)
    starts[123] = g.n + 3
    paths = torch.empty((500, 11), dtype=torch.int32).pin_memory()
    plen = torch.empty(500, dtype=torch.int32).pin_memory()
    with pytest.raises(_fw.FwError) as e:
        dg.walk_batched("weighted", starts, 10, 4, budget_bytes=2 * 100 * 13 * 4, paths=paths, path_len=plen)
    assert e.value.status == _fw.FW_EINVAL
    # the bad query is written as an empty path; the others are walked
    assert int(plen[123]) == 0 and bool((paths[123] == -1).all())
    ok = torch.ones(500, dtype=torch.bool)
    ok[123] = False
    assert bool((plen[ok] >= 1).all())
