"""Pin the oracle's transition law against exact rational brute force.

The reference law (tests/tiny_graphs.py) is written from Section 2.1, Eq. 1 and
Eq. 2 with breadth-first-search distances; the oracle uses integer weights and
a binary search in N(prev).  Every valid (prev, cur) state of several tiny
graphs is checked for every algorithm and several parameter choices.
"""

from fractions import Fraction

import numpy as np
import pytest

import tiny_graphs as tg

GRAPHS = {
    "triangle_pendant": tg.triangle_pendant,
    "star": tg.star,
    "path": tg.path_graph,
    "random9": tg.random_small,
    "random12": lambda: tg.random_small(12, 0.35, seed=11),
}

# (p, q) pairs whose exact-mode factors S/p, S, S/q are integers for S = 2
N2V = [(2.0, 0.5), (1.0, 2.0), (1.0, 1.0), (0.5, 2.0), (2.0, 1.0)]


def _norm(pairs):
    tot = sum(f for _, f in pairs)
    return [f / tot if tot else Fraction(0) for _, f in pairs], tot


@pytest.mark.parametrize("gname", list(GRAPHS))
@pytest.mark.parametrize("algo", ["weighted", "ppr", "metapath", "node2vec"])
def test_exact_law_matches_brute_force(orc, gname, algo):
    g = GRAPHS[gname]()
    csr = orc.CSR(g)
    pq_list = N2V if algo == "node2vec" else [(1.0, 1.0)]
    schemas = [(0, 1, 2, 3, 4), (3, 1), (2,)] if algo == "metapath" else [(0, 1, 2, 3, 4)]
    for (p, q) in pq_list:
        for schema in schemas:
            prm = orc.Params(p=p, q=q, scale=2, schema=schema)
            for (prev, cur) in tg.valid_states(g):
                for t in range(0, 6):
                    got = orc.transition(csr, algo, prm, cur, prev, t, mode="exact")
                    ref = tg.law(g, algo, cur, prev, t, a=Fraction(p), b=Fraction(q), schema=schema)
                    assert len(got) == len(ref)
                    # the support (zero weights) must agree exactly
                    assert [int(x) == 0 for x in got] == [f == 0 for _, f in ref]
                    tot = int(np.sum(got, dtype=np.uint64))
                    pref, rtot = _norm(ref)
                    if rtot == 0:
                        assert tot == 0
                        continue
                    pgot = [Fraction(int(x), tot) for x in got]
                    assert pgot == pref, (gname, algo, p, q, schema, prev, cur, t)


@pytest.mark.parametrize("gname", list(GRAPHS))
@pytest.mark.parametrize("algo", ["weighted", "metapath", "node2vec"])
def test_fast_law_matches_brute_force(orc, gname, algo):
    g = GRAPHS[gname]()
    # fast mode reads FP32 weights: give them non-integer values on the 2^-14 grid
    g.w_f32 = (g.w_u32.astype(np.float64) + 0.375).astype(np.float32)
    csr = orc.CSR(g)
    for (p, q) in (N2V if algo == "node2vec" else [(1.0, 1.0)]):
        prm = orc.Params(p=p, q=q, scale=2)
        for (prev, cur) in tg.valid_states(g):
            for t in range(3):
                got = orc.transition(csr, algo, prm, cur, prev, t, mode="fast")
                ref = tg.law(g, algo, cur, prev, t, a=Fraction(p), b=Fraction(q),
                             weight_of=lambda w: Fraction(float(np.float32(w + 0.375))))
                pref, rtot = _norm(ref)
                if rtot == 0:
                    assert float(np.sum(got)) == 0.0
                    continue
                pg = got / got.sum()
                assert np.allclose(pg, [float(x) for x in pref], rtol=1e-14, atol=0)


def test_star_node2vec_by_hand(orc):
    """Star: a leaf always returns to the hub; at the hub, coming from leaf l,
    leaf l has factor 1/p and every other leaf 1/q (their only neighbour is the
    hub, so their distance from l is 2)."""
    g = tg.star(5)
    csr = orc.CSR(g)
    prm = orc.Params(p=2.0, q=0.5, scale=2)  # factors 1, 2, 4
    for leaf in range(1, 6):
        w = orc.transition(csr, "node2vec", prm, leaf, 0, 1)
        assert list(w) == [1 * g.adj[leaf][0][0]]  # only the hub, which is prev: factor S/p = 1
    for l in range(1, 6):
        w = orc.transition(csr, "node2vec", prm, 0, l, 1)
        expect = [(1 if u == l else 4) * u for u in range(1, 6)]  # leaf weight i
        assert list(w) == expect


def test_first_move_is_first_order(orc):
    """With no previous vertex node2vec takes a first-order weighted step."""
    g = tg.random_small()
    csr = orc.CSR(g)
    prm = orc.Params(p=2.0, q=0.5, scale=2)
    for cur in range(g.n):
        a = orc.transition(csr, "node2vec", prm, cur, -1, 0)
        b = orc.transition(csr, "weighted", prm, cur, -1, 0)
        assert list(a) == list(b)
