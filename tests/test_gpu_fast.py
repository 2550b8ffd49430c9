"""Fast mode (FP32 reservoir sampling): validity of every move and the
empirical one-step law against the oracle's exact transition probabilities.

Acceptance (fixed before running; the seeds are fixed here and never
re-drawn): for 10^7 one-step samples from a fixed (prev, cur, t) state, the
total-variation distance to the exact law is <= 2e-3 and Pearson's
chi-square (cells merged to expected >= 5) has p > 1e-3.
"""

import numpy as np
import pytest
import torch
from scipy import stats

import fw_inputs as fi
import tiny_graphs as tg
from gpu_common import cached_graph, check_valid, device_graph

pytestmark = pytest.mark.gpu

N = 10_000_000
TV_MAX = 2e-3
P_MIN = 1e-3


def _one_step(dg, algo, cur, prev, t, seed, **kw):
    starts = torch.full((N,), cur, dtype=torch.int32, device="cuda")
    pv = torch.full((N,), prev, dtype=torch.int32, device="cuda")
    s0 = torch.full((N,), t, dtype=torch.int32, device="cuda")
    paths, plen = dg.walk(algo, starts, t + 1, seed, mode="fast", prev=pv, step0=s0, **kw)
    assert bool((plen == 2).all())
    return paths[:, 1]


def _law(orc, g, algo, cur, prev, t, **kw):
    w = orc.transition(orc.CSR(g), algo, orc.Params(**kw), cur, prev, t, mode="fast")
    return w / w.sum()


def _compare(g, nxt, p, cur, bins=None):
    rp = g.row_ptr
    nb = g.col[int(rp[cur]):int(rp[cur + 1])].to(torch.int64).cuda()
    # map sampled vertex -> index in the row
    idx = torch.searchsorted(nb, nxt.to(torch.int64))
    assert bool((nb[torch.clamp(idx, max=nb.numel() - 1)] == nxt.to(torch.int64)).all())
    counts = torch.bincount(idx, minlength=nb.numel()).cpu().numpy().astype(np.float64)
    assert counts[p == 0].sum() == 0, "a zero-probability neighbour was sampled"
    if bins:
        edges = np.linspace(0, len(p), bins + 1).astype(int)
        cb = np.add.reduceat(counts, edges[:-1])
        pb = np.add.reduceat(p, edges[:-1])
    else:
        cb, pb = counts, p
    tv = 0.5 * np.abs(cb / N - pb).sum()
    # chi-square over all cells with p > 0, merging in index order to expected >= 5
    e = p[p > 0] * N
    c = counts[p > 0]
    mc, me, acc_c, acc_e = [], [], 0.0, 0.0
    for ci, ei in zip(c, e):
        acc_c += ci
        acc_e += ei
        if acc_e >= 5:
            mc.append(acc_c)
            me.append(acc_e)
            acc_c = acc_e = 0.0
    if acc_e > 0:
        mc[-1] += acc_c
        me[-1] += acc_e
    pval = stats.chisquare(mc, me).pvalue if len(mc) > 1 else 1.0
    return tv, pval


def _pick_vertex(g, lo, hi):
    d = (g.row_ptr[1:] - g.row_ptr[:-1])
    cand = torch.nonzero((d >= lo) & (d <= hi))[:, 0]
    return int(cand[len(cand) // 2])


def _pick_prev_with_mixed_classes(g, cur):
    rp, col = g.row_ptr, g.col
    ncur = set(col[int(rp[cur]):int(rp[cur + 1])].tolist())
    best, best_ov = None, -1
    for v in list(ncur)[:200]:
        nv = set(col[int(rp[v]):int(rp[v + 1])].tolist())
        ov = len(nv & ncur)
        if 0 < ov < len(ncur) - 1 and ov > best_ov:
            best, best_ov = v, ov
    assert best is not None
    return best


def test_T1_weighted_warp_tier(orc):
    g = cached_graph("rmat", 20)
    dg = device_graph(g)
    cur = _pick_vertex(g, 35, 45)
    nxt = _one_step(dg, "weighted", cur, -1, 0, 20240413)
    tv, pv = _compare(g, nxt, _law(orc, g, "weighted", cur, -1, 0), cur)
    assert tv <= TV_MAX and pv > P_MIN, (tv, pv)


def test_T2_node2vec_mixed_classes(orc):
    g = cached_graph("rmat", 20)
    dg = device_graph(g)
    cur = _pick_vertex(g, 60, 70)
    prev = _pick_prev_with_mixed_classes(g, cur)
    nxt = _one_step(dg, "node2vec", cur, prev, 3, 20240414, p=2.0, q=0.5)
    p = _law(orc, g, "node2vec", cur, prev, 3, p=2.0, q=0.5)
    assert len(set(np.round(p / p.min(), 3))) > 2
    tv, pv = _compare(g, nxt, p, cur)
    assert tv <= TV_MAX and pv > P_MIN, (tv, pv)


def test_T3_metapath_masked(orc):
    g = cached_graph("rmat", 20, 2)
    dg = device_graph(g)
    cur = _pick_vertex(g, 95, 110)
    nxt = _one_step(dg, "metapath", cur, -1, 2, 20240415)
    p = _law(orc, g, "metapath", cur, -1, 2)
    assert (p == 0).sum() > 0
    tv, pv = _compare(g, nxt, p, cur)
    assert tv <= TV_MAX and pv > P_MIN, (tv, pv)


def test_T4_hub_block_tier(orc):
    g = cached_graph("rmat", 20)
    dg = device_graph(g)
    dg.set_tuning(d_warp=4096)  # the max-degree row is far above d_t: the CTA sampler's tier
    cur = int((g.row_ptr[1:] - g.row_ptr[:-1]).argmax())
    nxt = _one_step(dg, "weighted", cur, -1, 0, 20240416)
    st = dg.stats()
    # hub rows go to the CTA sampler unless all of the CTA's hub-task entries
    # are taken, in which case the owner warp samples the row itself
    assert st["block_steps"] > N // 2 and st["block_steps"] + st["warp_steps"] == N
    tv, pv = _compare(g, nxt, _law(orc, g, "weighted", cur, -1, 0), cur, bins=64)
    assert tv <= TV_MAX and pv > P_MIN, (tv, pv)


def test_T4b_hub_node2vec_block_tier(orc):
    g = cached_graph("rmat", 20)
    dg = device_graph(g)
    d = g.row_ptr[1:] - g.row_ptr[:-1]
    cur = int(torch.nonzero((d > 3000) & (d < 6000))[0, 0])
    prev = _pick_prev_with_mixed_classes(g, cur)
    nxt = _one_step(dg, "node2vec", cur, prev, 5, 20240417, p=1.0, q=2.0)
    p = _law(orc, g, "node2vec", cur, prev, 5, p=1.0, q=2.0)
    tv, pv = _compare(g, nxt, p, cur, bins=64)
    assert tv <= TV_MAX and pv > P_MIN, (tv, pv)


def test_T5_two_step_joint_tiny_graph(orc):
    g = tg.random_small(12, 0.5, seed=5)
    g.w_f32 = (g.w_u32.astype(np.float64) + 0.25).astype(np.float32)
    dg = device_graph(g)
    s = 3
    starts = torch.full((N,), s, dtype=torch.int32, device="cuda")
    paths, plen = dg.walk("node2vec", starts, 2, 20240418, mode="fast", p=2.0, q=0.5)
    a = paths[:, 1].to(torch.int64)
    b = paths[:, 2].to(torch.int64)
    counts = torch.bincount(a * g.n + b, minlength=g.n * g.n).cpu().numpy().astype(np.float64)
    exact = np.zeros(g.n * g.n)
    csr = orc.CSR(g)
    p1 = orc.transition(csr, "node2vec", orc.Params(p=2.0, q=0.5), s, -1, 0, mode="fast")
    n1 = g.col[g.row_ptr[s]:g.row_ptr[s + 1]]
    for ai, av in enumerate(n1):
        p2 = orc.transition(csr, "node2vec", orc.Params(p=2.0, q=0.5), int(av), s, 1, mode="fast")
        n2 = g.col[g.row_ptr[av]:g.row_ptr[av + 1]]
        for bi, bv in enumerate(n2):
            exact[int(av) * g.n + int(bv)] += p1[ai] / p1.sum() * p2[bi] / p2.sum()
    assert counts[exact == 0].sum() == 0
    tv = 0.5 * np.abs(counts / N - exact).sum()
    m = exact > 0
    pv = stats.chisquare(counts[m], exact[m] * N).pvalue
    assert tv <= TV_MAX and pv > P_MIN, (tv, pv)


def test_validity_configs_fast():
    # config 1 weighted, config 2 node2vec, config 3 MetaPath + PPR (one launch)
    g1 = cached_graph("chunglu")
    d1 = device_graph(g1)
    s1 = fi.one_per_vertex(g1.n, "cuda")
    p, l = d1.walk("weighted", s1, 80, 42, mode="fast")
    check_valid(g1, p, l, "weighted")
    g2 = cached_graph("rmat", 20)
    d2 = device_graph(g2)
    s2 = fi.one_per_vertex(g2.n, "cuda")
    p, l = d2.walk("node2vec", s2, 80, 42, mode="fast", p=2.0, q=0.5)
    moves = check_valid(g2, p, l, "node2vec")
    assert d2.stats()["steps"] == moves
    deg = (g2.row_ptr[1:] - g2.row_ptr[:-1]).cuda()
    assert bool(((l == 1) == (deg == 0)).all()) and bool((l[deg > 0] == 81).all())
    g3 = cached_graph("rmat", 22, 2)
    d3 = device_graph(g3)
    s3 = fi.one_per_vertex(g3.n, "cuda")
    (mp, ml), (pp, pl) = d3.walk_multi([
        dict(algo="metapath", starts=s3, max_len=80, seed=42, mode="fast"),
        dict(algo="ppr", starts=s3, max_len=100, seed=42, mode="fast", ppr_stop=0.2)])
    check_valid(g3, mp, ml, "metapath")
    check_valid(g3, pp, pl, "ppr")
    deg3 = (g3.row_ptr[1:] - g3.row_ptr[:-1]).cuda()
    moves = (pl[deg3 > 0] - 1).cpu().numpy()
    cap = 100
    counts = np.bincount(moves, minlength=cap + 1)[1:]
    pk = np.array([0.8 ** (k - 1) * 0.2 for k in range(1, cap)] + [0.8 ** (cap - 1)])
    e = pk * moves.size
    keep = e >= 5
    c2 = np.append(counts[keep], counts[~keep].sum())
    e2 = np.append(e[keep], e[~keep].sum())
    assert stats.chisquare(c2, e2).pvalue > P_MIN


@pytest.fixture(scope="module")
def g_lognormal():
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    # the recipe uses float64 exp/log/cos: generate once and give the same
    # arrays to the GPU and to the oracle
    return fi.rmat(18, weights="lognormal3", device=dev).to("cpu")


def test_T6_lognormal_sigma3_weights(orc, g_lognormal):
    """Log-normal weights with sigma = 3 (Appendix C.1) span about eight
    decades, where an FP32 reservoir's running sums could drift: one step
    of the weighted rule from a row of about 5000 entries, and of node2vec
    (p=2, q=0.5) from the same row with a previous vertex that gives all
    three classes."""
    g = g_lognormal
    dg = device_graph(g)
    cur = _pick_vertex(g, 4000, 6000)
    w = g.w_f32[int(g.row_ptr[cur]):int(g.row_ptr[cur + 1])].double()
    assert float(w.max() / w.min()) > 1e6
    nxt = _one_step(dg, "weighted", cur, -1, 0, 20241205)
    tv, pv = _compare(g, nxt, _law(orc, g, "weighted", cur, -1, 0), cur, bins=64)
    assert tv <= TV_MAX and pv > P_MIN, ("weighted", tv, pv)
    prev = _pick_prev_with_mixed_classes(g, cur)
    nxt = _one_step(dg, "node2vec", cur, prev, 4, 20241206, p=2.0, q=0.5)
    p = _law(orc, g, "node2vec", cur, prev, 4, p=2.0, q=0.5)
    tv, pv = _compare(g, nxt, p, cur, bins=64)
    assert tv <= TV_MAX and pv > P_MIN, ("node2vec", tv, pv)


def test_fast_paths_do_not_depend_on_tuning():
    """Fast mode cuts every row into the same 16K-entry segments with one
    random stream each, whether a warp or a CTA hub task samples it: the
    paths are bit-identical under any d_t and launch shape."""
    g = cached_graph("rmat", 20, 2)
    dg = device_graph(g)
    d = g.row_ptr[1:] - g.row_ptr[:-1]
    assert int(d.max()) > 3 * 16384  # rows of several segments exist
    starts = fi.random_starts(g.n, 20000, 17, "cuda")
    starts[:64] = torch.argsort(d, descending=True)[:64].to(torch.int32).cuda()  # start on the hubs too
    outs = []
    for tu in (dict(), dict(d_warp=256), dict(d_warp=1 << 20), dict(block_threads=512, slots=64, d_warp=1024),
               dict(block_threads=256, slots=8, d_warp=100000)):
        dg.set_tuning(**tu)
        res = []
        for algo in ("weighted", "node2vec", "metapath"):
            p, l = dg.walk(algo, starts, 20, 31, mode="fast", p=2.0, q=0.5)
            res.append((p, l))
        outs.append(res)
    dg.set_tuning()
    for res in outs[1:]:
        for (p0, l0), (p1, l1) in zip(outs[0], res):
            assert torch.equal(l0, l1) and torch.equal(p0, p1)
