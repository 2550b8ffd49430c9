"""Pin the oracle's selection phase and walk loop.

* the exact pick (smallest i whose inclusive prefix exceeds r) hits neighbour i
  exactly w_i times when r runs over [0, W): inverse transform sampling;
* r = floor(x * W / 2^64) against Python's unbounded integers;
* whole walks against hand-derivable cases (a directed cycle, dead ends,
  MetaPath with no matching label), the special cases that reduce one
  algorithm to another, resumption, the output layout of Section 5.2 / Table 3,
  and empirical step laws against the exact-rational law (chi-square).
"""

import random
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import tiny_graphs as tg


@pytest.mark.parametrize("seed", range(6))
def test_pick_enumeration(orc, seed):
    rnd = random.Random(seed)
    d = rnd.randint(1, 9)
    w = [rnd.choice([0, 0, 1, 2, 3, 7]) for _ in range(d)]
    if sum(w) == 0:
        w[-1] = 3
    W = sum(w)
    hits = [0] * d
    for r in range(W):
        hits[orc.pick(w, r)] += 1
    assert hits == w
    assert orc.pick(w, W) == -1


def test_scale_draw_closed_form(orc):
    rnd = random.Random(7)
    for _ in range(2000):
        x = rnd.getrandbits(64)
        W = rnd.choice([1, 2, 3, 5, 2**19, 2**39 - 1, rnd.getrandbits(40) + 1])
        assert orc.scale_draw(x, W) == (x * W) >> 64
    for W in (1, 5, 81920 * 4 * 10**6):
        assert orc.scale_draw(0, W) == 0
        assert orc.scale_draw(2**64 - 1, W) == W - 1


def test_scale_draw_is_uniform_over_residues(orc):
    """Every r in [0, W) is hit by floor(2^64 / W) or that + 1 values of x:
    checked on the x-interval boundaries r * 2^64 / W."""
    for W in (3, 5, 7, 1000003):
        for r in (0, 1, W // 2, W - 1):
            lo = -(-(r << 64) // W)          # smallest x with x*W >= r*2^64
            hi = -(-((r + 1) << 64) // W) - 1  # largest x mapping to r
            assert orc.scale_draw(lo, W) == r and orc.scale_draw(hi, W) == r
            if lo > 0:
                assert orc.scale_draw(lo - 1, W) == r - 1
            assert hi - lo + 1 in (2**64 // W, 2**64 // W + 1)


def test_ppr_threshold(orc):
    assert orc.ppr_threshold(0.2) == 858993459  # floor(0.2 * 2^32)
    assert orc.ppr_threshold(0.0) == 0
    assert orc.ppr_threshold(0.5) == 2**31


def _walk(orc, g, algo, starts, L, seed=42, prm=None, **kw):
    return orc.walk_exact(orc.CSR(g), algo, prm or orc.Params(p=2.0, q=0.5), starts, L, seed, **kw)


def test_directed_cycle_is_deterministic(orc):
    n = 7
    g = tg.csr_from_edges(n, [(i, (i + 1) % n, 1 + i % 3, i % 5) for i in range(n)], directed=True)
    for algo in ("weighted", "node2vec", "ppr"):
        paths, plen = _walk(orc, g, algo, np.arange(n), 20)
        for s in range(n):
            k = plen[s]
            assert list(paths[s, :k]) == [(s + i) % n for i in range(k)]
            assert (paths[s, k:] == -1).all()
            if algo != "ppr":
                assert k == 21


def test_dead_ends_and_metapath_mismatch(orc):
    g = tg.csr_from_edges(4, [(0, 1, 2, 0), (1, 2, 3, 1)])  # vertex 3 isolated
    paths, plen = _walk(orc, g, "weighted", [3, 0], 5)
    assert plen[0] == 1 and list(paths[0]) == [3, -1, -1, -1, -1, -1]
    # schema wants label 4 first: nothing matches, no move is made
    prm = orc.Params(schema=(4, 0))
    paths, plen = _walk(orc, g, "metapath", [0, 1, 2], 5, prm=prm)
    assert list(plen) == [1, 1, 1]
    # schema (0, 1): 0 -> 1 (label 0), 1 -> 2 (label 1), then label 0 needed at 2: stop
    prm = orc.Params(schema=(0, 1))
    paths, plen = _walk(orc, g, "metapath", [0], 5, prm=prm)
    assert list(paths[0, :plen[0]]) == [0, 1, 2]


def test_special_cases_reduce_to_weighted(orc):
    g = tg.random_small(12, 0.35, seed=11)
    starts = np.arange(g.n).repeat(20)
    ref, rlen = _walk(orc, g, "weighted", starts, 30, seed=9)
    # node2vec with p = q = 1: factors (2, 2, 2) scale every weight, same picks
    a, alen = _walk(orc, g, "node2vec", starts, 30, seed=9, prm=orc.Params(p=1.0, q=1.0, scale=2))
    assert (a == ref).all() and (alen == rlen).all()
    # PPR with stop probability 0
    b, blen = _walk(orc, g, "ppr", starts, 30, seed=9, prm=orc.Params(ppr_stop=0.0))
    assert (b == ref).all() and (blen == rlen).all()
    # MetaPath on a single-label graph with the schema (0)
    g1 = tg.random_small(12, 0.35, seed=11)
    g1.etype[:] = 0
    c, clen = _walk(orc, g1, "metapath", starts, 30, seed=9, prm=orc.Params(schema=(0,)))
    assert (c == ref).all() and (clen == rlen).all()


@pytest.mark.parametrize("algo", ["weighted", "node2vec", "metapath"])
def test_resume_continues_bit_for_bit(orc, algo):
    g = tg.random_small(12, 0.5, seed=5)
    starts = np.arange(g.n).repeat(10)
    prm = orc.Params(p=2.0, q=0.5, schema=(0, 1, 2, 3, 4))
    full, flen = _walk(orc, g, algo, starts, 40, seed=3, prm=prm)
    k = 13
    ok = flen > k + 1
    cur = full[ok, k]
    prev = full[ok, k - 1]
    q_ids = np.nonzero(ok)[0]
    for i, q in enumerate(q_ids):
        tail, tlen = orc.walk_exact(orc.CSR(g), algo, prm, [cur[i]], 40, 3, prev=[prev[i]],
                                    step0=[k], q0=int(q))
        assert tlen[0] == flen[q] - k
        assert list(tail[0, :tlen[0]]) == list(full[q, k:flen[q]])


def test_output_layout_matches_table3_arithmetic():
    """Section 6.3: 10^6 queries of length 80 with 32-bit ids take ~309 MB:
    10^6 * (80 + 1) * 4 B = 324e6 B = 309.0 MiB (start vertex included)."""
    nbytes = 10**6 * (80 + 1) * 4
    assert round(nbytes / 2**20, 1) == 309.0


def test_walk_rows_are_edges_on_chung_lu(orc):
    import fw_inputs as fi
    g = fi.chung_lu()
    paths, plen = orc.walk_exact(orc.CSR(g), "weighted", orc.Params(), fi.one_per_vertex(g.n), 80, 42)
    rp = g.row_ptr.numpy()
    col = g.col.numpy()
    for q in range(g.n):
        k = plen[q]
        deg0 = rp[paths[q, 0] + 1] - rp[paths[q, 0]]
        assert (k == 1) == (deg0 == 0)
        if deg0:
            assert k == 81  # undirected graph: no dead end after the first move
        for i in range(k - 1):
            u, v = paths[q, i], paths[q, i + 1]
            assert v in col[rp[u]:rp[u + 1]]


@pytest.mark.parametrize("algo,prev,cur,t", [("weighted", -1, 4, 0), ("node2vec", 2, 4, 3),
                                             ("node2vec", 9, 3, 1), ("metapath", -1, 4, 2)])
def test_step_law_chi_square(orc, algo, prev, cur, t):
    """One-step samples of the walk (10^5 queries from the same state) follow
    the exact-rational law (Pearson chi-square, p > 1e-3)."""
    g = tg.random_small(12, 0.5, seed=5)
    assert prev < 0 or cur in g.adj[prev]
    N = 100000
    prm = orc.Params(p=2.0, q=0.5, schema=(0, 1, 2, 3, 4))
    while sum(f for _, f in tg.law(g, algo, cur, prev, t)) == 0:
        t += 1  # MetaPath: move on to a step whose label occurs at cur
    paths, plen = orc.walk_exact(orc.CSR(g), algo, prm, np.full(N, cur), t + 1, 1234,
                                 prev=np.full(N, prev), step0=np.full(N, t))
    law = tg.law(g, algo, cur, prev, t, a=Fraction(2), b=Fraction(1, 2))
    tot = sum(f for _, f in law)
    nbrs = [u for u, _ in law]
    moved = plen == 2
    assert moved.all()
    counts = np.array([(paths[:, 1] == u).sum() for u in nbrs])
    exp = np.array([float(f / tot) * N for _, f in law])
    assert counts[exp == 0].sum() == 0
    keep = exp > 0
    chi = stats.chisquare(counts[keep], exp[keep])
    assert chi.pvalue > 1e-3, (counts, exp)


def test_ppr_lengths_are_geometric(orc):
    """PPR on a graph without dead ends: the number of moves k follows
    P(k) = 0.8^(k-1) * 0.2 for k < cap and P(cap) = 0.8^(cap-1)."""
    g = tg.random_small(10, 0.8, seed=2)
    assert all(len(g.adj[v]) > 0 for v in range(g.n))
    N, cap = 60000, 12
    _, plen = orc.walk_exact(orc.CSR(g), "ppr", orc.Params(ppr_stop=0.2), np.arange(N) % g.n, cap, 77)
    moves = plen - 1
    counts = np.bincount(moves, minlength=cap + 1)[1:]
    pk = np.array([0.8 ** (k - 1) * 0.2 for k in range(1, cap)] + [0.8 ** (cap - 1)])
    assert stats.chisquare(counts, pk * N).pvalue > 1e-3
