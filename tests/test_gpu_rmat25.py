"""The headline workload itself: node2vec p=1, q=2 on the R-MAT scale-25
graph (1.05e9 CSR entries, int64 row offsets, column and weight arrays of
4.2 GB each, hub rows far beyond one 16K-entry segment), in the launch
configuration the benchmark times (2^21 queries, one per vertex v = 16 k,
default tuning).

  (a) fast mode: every move of the whole slice is an edge, padding is -1,
      and the engine's counters equal a host recount of the paths;
  (b) exact mode (S = 2: factors 2, 2, 1): the same launch with 20 of its
      starts moved to rows among the 100 largest; 300 queries (those 20 and
      280 drawn over the whole slice) recomputed by the oracle, bit for bit;
  (c) 10^7 one-step fast-mode samples at the max-degree row with a previous
      vertex that gives all three node2vec classes: TV <= 2e-3 on 64
      contiguous bins and Pearson chi-square p > 1e-3 against the oracle's
      exact law (Eq. 2).
"""

import numpy as np
import pytest
import torch

import fw_inputs as fi
from gpu_common import cached_graph, check_valid, chi2_tv, compare_sampled, device_graph, recount

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SCALE = 25
BATCH = 1 << 21
P1Q2 = dict(p=1.0, q=2.0)


@pytest.fixture(scope="module")
def g25():
    return cached_graph("rmat", SCALE)


@pytest.fixture(scope="module")
def dg25(g25):
    dg = device_graph(g25)
    yield dg
    dg.free()
    torch.cuda.empty_cache()


def _slice0(g):
    return torch.arange(0, g.n, g.n // BATCH, dtype=torch.int32, device="cuda")[:BATCH]


def test_a_fast_slice_valid_and_counted(g25, dg25):
    starts = _slice0(g25)
    dg25.stats_reset()
    paths, plen = dg25.walk("node2vec", starts, 80, 42, mode="fast", **P1Q2)
    st = dg25.stats()
    moves = check_valid(g25, paths, plen, "node2vec")
    deg = (g25.row_ptr[1:] - g25.row_ptr[:-1]).cuda()
    d0 = deg[starts.to(torch.int64)]
    # a walk stops early only at a dead end: isolated starts make no move, the rest make 80
    assert bool(((plen == 1) == (d0 == 0)).all()) and bool((plen[d0 > 0] == 81).all())
    n_moves, rows = recount(g25, paths, plen)
    assert st["steps"] == moves == n_moves
    assert st["rows_scanned"] == rows
    assert st["algo_bytes"] == 8 * rows + 20 * n_moves
    assert st["warp_steps"] + st["block_steps"] == n_moves
    assert st["block_steps"] > 0  # hub rows went through the CTA sampler
    del paths, plen
    torch.cuda.empty_cache()


def test_b_exact_slice_sampled_bit_exact(orc, g25, dg25):
    starts = _slice0(g25)
    deg = (g25.row_ptr[1:] - g25.row_ptr[:-1])
    top = torch.argsort(deg, descending=True)[:100]
    rng = np.random.default_rng(2025)
    hub_rows = rng.choice(100, 20, replace=False)
    hub_pos = rng.choice(BATCH, 20, replace=False)
    starts[torch.as_tensor(hub_pos, device="cuda")] = top[hub_rows].to(torch.int32).cuda()
    paths, plen = dg25.walk("node2vec", starts, 80, 42, mode="exact", scale=2, **P1Q2)
    torch.cuda.synchronize()
    check_valid(g25, paths, plen, "node2vec")
    others = rng.choice(np.setdiff1d(np.arange(BATCH), hub_pos), 280, replace=False)
    idx = np.concatenate([hub_pos, others])
    paths_h, plen_h, starts_h = paths.cpu(), plen.cpu(), starts.cpu()
    del paths, plen
    torch.cuda.empty_cache()
    assert int(deg[starts_h[hub_pos].long()].min()) >= int(deg[top[99]])
    compare_sampled(orc, g25, "node2vec", starts_h, 80, 42, paths_h, plen_h, orc.Params(scale=2, **P1Q2), idx)


def _mixed_prev(g, cur):
    rp, col = g.row_ptr.numpy(), g.col.numpy()
    ncur = col[rp[cur]:rp[cur + 1]]
    deg = np.diff(rp)
    best, best_ov = None, -1
    for v in ncur[:400]:
        if not 100 <= deg[v] <= 50000:
            continue
        ov = int(np.isin(col[rp[v]:rp[v + 1]], ncur, assume_unique=True).sum())
        if 0 < ov < ncur.size - 1 and ov > best_ov:
            best, best_ov = int(v), ov
    assert best is not None
    return best


def test_c_max_degree_row_one_step_law(orc, g25, dg25):
    N = 10_000_000
    deg = g25.row_ptr[1:] - g25.row_ptr[:-1]
    cur = int(deg.argmax())
    prev = _mixed_prev(g25, cur)
    t = 5
    starts = torch.full((N,), cur, dtype=torch.int32, device="cuda")
    pv = torch.full((N,), prev, dtype=torch.int32, device="cuda")
    s0 = torch.full((N,), t, dtype=torch.int32, device="cuda")
    paths, plen = dg25.walk("node2vec", starts, t + 1, 20241204, mode="fast", prev=pv, step0=s0, **P1Q2)
    assert bool((plen == 2).all())
    nxt = paths[:, 1].to(torch.int64)
    rp = g25.row_ptr
    nb = g25.col[int(rp[cur]):int(rp[cur + 1])].to(torch.int64).cuda()
    pos = torch.searchsorted(nb, nxt)
    assert bool((nb[torch.clamp(pos, max=nb.numel() - 1)] == nxt).all())
    counts = torch.bincount(pos, minlength=nb.numel()).cpu().numpy()
    w = orc.transition(orc.CSR(g25), "node2vec", orc.Params(**P1Q2), cur, prev, t, mode="fast")
    p = w / w.sum()
    # both factors of Eq. 2 occur in this row (p = 1 makes the return and the
    # in factor both 1; q = 2 gives the others 1/2)
    fac = w / g25.w_f32[int(rp[cur]):int(rp[cur + 1])].numpy().astype(np.float64)
    assert set(np.round(fac, 6)) == {1.0, 0.5}
    assert counts[p == 0].sum() == 0
    tv, pval = chi2_tv(counts, p, N, bins=64)
    assert tv <= 2e-3 and pval > 1e-3, (tv, pval)
