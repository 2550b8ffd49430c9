"""Walks in batches on two streams (fw_walk_batched, Section 5.2 and Eq. 3):
the paths equal one launch over all queries, whatever the batch size."""

import pytest
import torch

import fw_inputs as fi
from gpu_common import cached_graph, device_graph

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("algo", ["node2vec", "metapath", "ppr"])
def test_batched_equals_one_launch_exact(algo):
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
    ref_p, ref_l = dg.walk(algo, starts.cuda(), L, 9, mode="exact", p=2.0, q=0.5, q_id0=1000)
    assert torch.equal(plen, ref_l.cpu())
    assert torch.equal(paths, ref_p.cpu())


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
