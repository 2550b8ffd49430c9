"""Helpers shared by the GPU tests: build the library, move graphs to the
device, check walks for validity with torch ops on the device."""

import functools

import numpy as np
import pytest
import torch

import fw_inputs as fi


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


@functools.lru_cache(maxsize=None)
def built():
    from paper_2404_08364_gb300.build import build
    return build()


def device_graph(g, **kw):
    need_gpu()
    built()
    from paper_2404_08364_gb300 import DeviceGraph
    return DeviceGraph.from_graph(g, device="cuda", **kw)


@functools.lru_cache(maxsize=None)
def cached_graph(kind, scale=0, types_seed=None):
    """Graphs generated once per session (on the GPU when it is there)."""
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    if kind == "chunglu":
        return fi.chung_lu(device=dev).to("cpu")
    return fi.rmat(scale, types_seed=types_seed, device=dev).to("cpu")


def edge_lookup(g, dev="cuda"):
    """Sorted keys u*n+v of every CSR entry (device) and the edge labels."""
    rp = g.row_ptr.to(dev)
    src = torch.repeat_interleave(torch.arange(g.n, device=dev), rp[1:] - rp[:-1])
    keys = src * g.n + g.col.to(dev).to(torch.int64)
    return keys, None if g.etype is None else g.etype.to(dev)


def check_valid(g, paths, plen, algo, schema=(0, 1, 2, 3, 4), max_len=None):
    """Every move is an edge; MetaPath moves carry schema[t mod len]; padding
    is -1; a walk that stopped early stopped for a reason the rule allows."""
    dev = paths.device
    keys, et = edge_lookup(g, dev)
    n_q, width = paths.shape
    t = torch.arange(width, device=dev)[None, :]
    valid = t < plen[:, None].to(torch.int64)
    assert bool((paths[~valid] == -1).all()), "padding must be -1"
    assert bool((plen >= 1).all())
    u = paths[:, :-1].to(torch.int64)
    v = paths[:, 1:].to(torch.int64)
    mv = valid[:, 1:]
    uu, vv = u[mv], v[mv]
    k = uu * g.n + vv
    pos = torch.searchsorted(keys, k)
    pos = torch.clamp(pos, max=keys.numel() - 1)
    assert bool((keys[pos] == k).all()), "a move is not an edge"
    if algo == "metapath":
        tt = torch.arange(width - 1, device=dev)[None, :].expand(n_q, -1)[mv]
        want = torch.tensor(list(schema), device=dev, dtype=torch.int8)[tt % len(schema)]
        assert bool((et[pos] == want).all()), "a MetaPath move has the wrong label"
    return int(mv.sum())


def compare_sampled(orc, g, algo, starts, L, seed, paths, plen, prm, idx, q_id0=0, **kw):
    """Recompute queries idx of a launch one by one with the oracle (query id
    q_id0 + index, as the launch used) and compare them element by element."""
    csr = orc.CSR(g) if not isinstance(g, orc.CSR) else g
    for q in idx:
        q = int(q)
        rp, rl = orc.walk_exact(csr, algo, prm, starts[q:q + 1], L, seed, q0=q_id0 + q,
                                **{k: v[q:q + 1] for k, v in kw.items()})
        assert int(plen[q]) == int(rl[0]), (algo, q, int(plen[q]), int(rl[0]))
        assert np.array_equal(paths[q].numpy(), rp[0]), (algo, q)


def recount(g, paths, plen):
    """Host-side recount of the engine's counters from returned paths: moves
    and the sum of deg(cur) over every move."""
    deg = (g.row_ptr[1:] - g.row_ptr[:-1]).to(torch.int64).to(paths.device)
    width = paths.shape[1]
    t = torch.arange(width, device=paths.device)[None, :]
    moved_from = (t < (plen[:, None].to(torch.int64) - 1)) & (paths >= 0)
    d = torch.where(moved_from, deg[paths.clamp(min=0).to(torch.int64)], torch.zeros_like(paths, dtype=torch.int64))
    return int((plen - 1).sum()), int(d.sum())


def chi2_tv(counts, p, n, bins=None):
    """Total-variation distance (optionally over `bins` contiguous index bins)
    and Pearson chi-square p-value (cells merged in index order to expected
    >= 5) of sampled counts against the law p."""
    from scipy import stats
    counts = np.asarray(counts, dtype=np.float64)
    if bins:
        edges = np.linspace(0, len(p), bins + 1).astype(int)
        cb, pb = np.add.reduceat(counts, edges[:-1]), np.add.reduceat(p, edges[:-1])
    else:
        cb, pb = counts, p
    tv = 0.5 * np.abs(cb / n - pb).sum()
    e = p[p > 0] * n
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
