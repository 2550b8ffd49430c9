"""Hand-made tiny graphs and an exact-rational statement of the transition law.

The law here is written straight from the paper's definitions, independently of
the oracle: Section 2.1 (p(u) proportional to f(e(v, u)), weighted f = w),
Eq. 1 (MetaPath: keep u iff l(v, u) equals the schema label of this move) and
Eq. 2 (node2vec: 1/a, 1, 1/b for dist(v', u) = 0, 1, 2, where dist is computed
here by breadth-first search, not by a row lookup), each multiplied by the edge
weight (weighted variants).
"""

from __future__ import annotations

import random
from fractions import Fraction
from types import SimpleNamespace

import numpy as np


def csr_from_edges(n, edges, directed=False):
    """edges: list of (u, v, w_int, label); returns a Graph-like namespace with
    sorted rows.  Undirected edges are stored in both directions with the same
    weight and label."""
    adj = {v: {} for v in range(n)}
    for (u, v, w, lab) in edges:
        adj[u][v] = (w, lab)
        if not directed:
            adj[v][u] = (w, lab)
    row_ptr = [0]
    col, wu, lb = [], [], []
    for v in range(n):
        for u in sorted(adj[v]):
            col.append(u)
            wu.append(adj[v][u][0])
            lb.append(adj[v][u][1])
        row_ptr.append(len(col))
    return SimpleNamespace(
        n=n, m=len(col),
        row_ptr=np.array(row_ptr, dtype=np.int64),
        col=np.array(col, dtype=np.int32),
        w_u32=np.array(wu, dtype=np.uint32),
        w_f32=np.array(wu, dtype=np.float32),
        etype=np.array(lb, dtype=np.int8),
        adj=adj,
    )


def bfs_dist(g, src, limit=4):
    dist = {src: 0}
    frontier = [src]
    for d in range(1, limit + 1):
        nxt = []
        for x in frontier:
            for y in g.adj[x]:
                if y not in dist:
                    dist[y] = d
                    nxt.append(y)
        frontier = nxt
    return dist


def law(g, algo, cur, prev=-1, t=0, a=Fraction(1), b=Fraction(1), schema=(0, 1, 2, 3, 4),
        weight_of=lambda w: Fraction(int(w))):
    """Unnormalised transition weights {u: Fraction} for the neighbours of cur,
    in the sorted row order, from the paper's definitions."""
    out = []
    dist = bfs_dist(g, prev) if (algo == "node2vec" and prev >= 0) else None
    for u in sorted(g.adj[cur]):
        w, lab = g.adj[cur][u]
        f = weight_of(w)
        if algo == "metapath":
            f = f if lab == schema[t % len(schema)] else Fraction(0)
        elif algo == "node2vec" and prev >= 0:
            dd = dist.get(u, 99)
            if dd == 0:
                f = f / a
            elif dd == 1:
                f = f * 1
            elif dd == 2:
                f = f / b
            else:
                f = Fraction(0)
        out.append((u, f))
    return out


def triangle_pendant():
    # 0-1-2 triangle, 3 hangs off 2; labels chosen so every label 0..4 appears
    return csr_from_edges(4, [(0, 1, 3, 0), (1, 2, 5, 1), (0, 2, 2, 2), (2, 3, 4, 3)])


def star(leaves=5):
    return csr_from_edges(leaves + 1, [(0, i, i, i % 5) for i in range(1, leaves + 1)])


def path_graph(n=5):
    return csr_from_edges(n, [(i, i + 1, 1 + i % 5, i % 5) for i in range(n - 1)])


def random_small(n=9, p_edge=0.45, seed=3):
    rnd = random.Random(seed)
    edges = []
    for i in range(n):
        for j in range(i + 1, n):
            if rnd.random() < p_edge:
                edges.append((i, j, rnd.randint(1, 5), rnd.randint(0, 4)))
    return csr_from_edges(n, edges)


def valid_states(g):
    """All (prev, cur) with cur in N(prev), plus (-1, cur) for every cur."""
    st = [(-1, c) for c in range(g.n)]
    for p in range(g.n):
        for c in g.adj[p]:
            st.append((p, c))
    return st
