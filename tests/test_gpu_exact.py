"""Exact mode: the CUDA path against the CPU oracle, bit for bit.

Small graphs run in full (several tiles per row, ragged tails, both sampler
tiers, every algorithm, several tunings); the full-size R-MAT workloads are
compared on a fixed sample of queries, each recomputed alone by the oracle.
"""

import numpy as np
import pytest
import torch

import fw_inputs as fi
from gpu_common import cached_graph, check_valid, device_graph

pytestmark = pytest.mark.gpu

P2 = dict(p=2.0, q=0.5)


def _oracle(orc, g, algo, starts, L, seed, prm, **kw):
    return orc.walk_exact(orc.CSR(g), algo, prm, starts, L, seed, **kw)


def _cmp(dev_paths, dev_len, ref_paths, ref_len):
    dp, dl = dev_paths.cpu().numpy(), dev_len.cpu().numpy()
    assert np.array_equal(dl, ref_len), f"path_len differs at {np.nonzero(dl != ref_len)[0][:10]}"
    bad = np.nonzero((dp != ref_paths).any(1))[0]
    assert bad.size == 0, f"paths differ for queries {bad[:10]}"


def test_config1_chung_lu_weighted(orc):
    g = cached_graph("chunglu")
    dg = device_graph(g)
    starts = fi.one_per_vertex(g.n, "cuda")
    paths, plen = dg.walk("weighted", starts, 80, 42, mode="exact")
    ref = _oracle(orc, g, "weighted", starts.cpu(), 80, 42, orc.Params())
    _cmp(paths, plen, *ref)
    st = dg.stats()
    assert st["steps"] == int((plen - 1).sum())
    assert st["walks"] == g.n


@pytest.mark.parametrize("algo", ["weighted", "node2vec", "metapath", "ppr"])
@pytest.mark.parametrize("tuning", [dict(), dict(block_threads=128, slots=16, d_warp=64),
                                    dict(block_threads=512, slots=128, d_warp=32),
                                    dict(block_threads=256, slots=7, d_warp=4096)])
def test_rmat12_all_algos_all_tunings(orc, algo, tuning):
    g = cached_graph("rmat", 12, 2)
    dg = device_graph(g)
    dg.set_tuning(**tuning)
    starts = fi.one_per_vertex(g.n, "cuda")
    L = 100 if algo == "ppr" else 40
    paths, plen = dg.walk(algo, starts, L, 1234, mode="exact", **P2)
    ref = _oracle(orc, g, algo, starts.cpu(), L, 1234, orc.Params(**P2))
    _cmp(paths, plen, *ref)
    check_valid(g, paths, plen, algo)
    st = dg.stats()
    assert st["steps"] == int((plen - 1).sum())
    if tuning.get("d_warp") == 32:
        assert st["block_steps"] > 0 and st["warp_steps"] > 0


def test_ragged_lengths_resume_and_offsets(orc):
    g = cached_graph("rmat", 12, 2)
    dg = device_graph(g)
    n_q = 3001
    starts = fi.random_starts(g.n, n_q, 3, "cuda")
    lengths = fi.uniform_lengths(n_q, 0, 50, 4, "cuda")
    # resume from an arbitrary (prev, cur) state on an edge at step 7
    src = torch.repeat_interleave(torch.arange(g.n), g.row_ptr[1:] - g.row_ptr[:-1])
    pick = torch.randint(0, g.m, (n_q,), generator=torch.Generator().manual_seed(1))
    prev = src[pick].to(torch.int32)
    cur = g.col[pick]
    step0 = torch.full((n_q,), 7, dtype=torch.int32)
    for algo in ("node2vec", "metapath", "ppr"):
        paths, plen = dg.walk(algo, cur.cuda(), 60, 99, mode="exact", lengths=lengths, prev=prev.cuda(),
                              step0=step0.cuda(), q_id0=12345, **P2)
        ref = _oracle(orc, g, algo, cur, 60, 99, orc.Params(**P2), lengths=lengths.cpu(), prev=prev,
                      step0=step0, q0=12345)
        _cmp(paths, plen, *ref)
    # a query range split over two calls (two "devices") equals one call
    p_all, l_all = dg.walk("node2vec", starts, 30, 5, mode="exact", **P2)
    p_a, l_a = dg.walk("node2vec", starts[:1000], 30, 5, mode="exact", **P2)
    p_b, l_b = dg.walk("node2vec", starts[1000:], 30, 5, mode="exact", q_id0=1000, **P2)
    assert torch.equal(torch.cat([p_a, p_b]), p_all) and torch.equal(torch.cat([l_a, l_b]), l_all)


def test_edge_cases(orc):
    g = cached_graph("rmat", 10, 2)
    dg = device_graph(g)
    deg = (g.row_ptr[1:] - g.row_ptr[:-1])
    iso = torch.nonzero(deg == 0)[:5, 0].to(torch.int32)
    # empty batch
    p, l = dg.walk("weighted", torch.empty(0, dtype=torch.int32, device="cuda"), 10, 1)
    assert p.shape == (0, 11)
    # max_len = 0: only the start vertex
    s = fi.one_per_vertex(g.n, "cuda")
    p, l = dg.walk("weighted", s, 0, 1)
    assert bool((l == 1).all()) and torch.equal(p[:, 0], s)
    # isolated starts: path_len 1, padded
    p, l = dg.walk("node2vec", iso.cuda(), 5, 1, **P2)
    assert bool((l == 1).all()) and bool((p[:, 1:] == -1).all())
    # the hub (vertex 0) and ragged tails: every start, one huge max_len
    p, l = dg.walk("weighted", s[:64], 1000, 8)
    ref = _oracle(orc, g, "weighted", s[:64].cpu(), 1000, 8, orc.Params())
    _cmp(p, l, *ref)


def test_host_buffers_equal_device_buffers(orc):
    g = cached_graph("rmat", 12, 2)
    dg = device_graph(g)
    s = fi.random_starts(g.n, 2000, 11)
    pd, ld = dg.walk("node2vec", s.cuda(), 30, 3, **P2)
    ph, lh = dg.walk("node2vec", s, 30, 3, **P2)            # host tensors: staged by the library
    assert ph.device.type == "cpu"
    assert torch.equal(ph, pd.cpu()) and torch.equal(lh, ld.cpu())
    pin = s.pin_memory()
    pp = torch.empty((2000, 31), dtype=torch.int32).pin_memory()
    lp = torch.empty(2000, dtype=torch.int32).pin_memory()
    dg.walk("node2vec", pin, 30, 3, paths=pp, path_len=lp, **P2)
    assert torch.equal(pp, pd.cpu()) and torch.equal(lp, ld.cpu())


def test_validation_errors():
    from paper_2404_08364_gb300 import DeviceGraph, _fw
    g = cached_graph("rmat", 8)
    bad = g.col.clone()
    rp = g.row_ptr
    r0 = int(torch.nonzero(rp[1:] - rp[:-1] >= 3)[0, 0])
    a = int(rp[r0])
    bad[a], bad[a + 1] = g.col[a + 1], g.col[a]
    with pytest.raises(_fw.FwError) as e:
        DeviceGraph.from_tensors(rp, bad, g.w_f32, g.w_u32)
    assert e.value.status == _fw.FW_EUNSORTED
    wz = g.w_f32.clone()
    wz[3] = 0
    with pytest.raises(_fw.FwError) as e:
        DeviceGraph.from_tensors(rp, g.col, wz, g.w_u32)
    assert e.value.status == _fw.FW_EINVAL
    # without validation an unsorted row loads (its results are undefined) ...
    DeviceGraph.from_tensors(rp, bad, g.w_f32, g.w_u32, validate=False).free()
    # ... but offsets and column ranges, which the kernels index by, are always checked
    oob = g.col.clone()
    oob[0] = g.n
    with pytest.raises(_fw.FwError) as e:
        DeviceGraph.from_tensors(rp, oob, g.w_f32, g.w_u32, validate=False)
    assert e.value.status == _fw.FW_EINVAL
    dg = device_graph(g)
    with pytest.raises(_fw.FwError):
        dg.walk("node2vec", torch.zeros(4, dtype=torch.int32), 5, 1, p=3.0, q=0.5)  # 2/3 not integral
    with pytest.raises(_fw.FwError):
        dg.walk("weighted", torch.tensor([g.n], dtype=torch.int32), 5, 1)        # start out of range (host)
    # device starts out of range: written as empty paths, reported by stats
    p, l = dg.walk("weighted", torch.tensor([0, g.n + 5], dtype=torch.int32, device="cuda"), 5, 1)
    with pytest.raises(_fw.FwError):
        dg.stats()
    assert int(l[1]) == 0 and bool((p[1] == -1).all())


def _sampled(orc, g, algo, starts, L, seed, paths, plen, prm, idx, **kw):
    for q in idx:
        q = int(q)
        rp, rl = orc.walk_exact(orc.CSR(g), algo, prm, starts[q:q + 1], L, seed, q0=q,
                                **{k: v[q:q + 1] for k, v in kw.items()})
        assert int(plen[q]) == int(rl[0]), (algo, q)
        assert np.array_equal(paths[q].numpy(), rp[0]), (algo, q)


@pytest.mark.slow
def test_config2_rmat20_node2vec_full_size_sampled(orc):
    g = cached_graph("rmat", 20)
    dg = device_graph(g)
    starts = fi.one_per_vertex(g.n, "cuda")
    paths, plen = dg.walk("node2vec", starts, 80, 42, mode="exact", **P2)
    torch.cuda.synchronize()
    n_moves = check_valid(g, paths, plen, "node2vec")
    st = dg.stats()
    assert st["steps"] == n_moves
    paths, plen = paths.cpu(), plen.cpu()
    idx = np.random.default_rng(0).choice(g.n, 300, replace=False)
    _sampled(orc, g, "node2vec", starts.cpu(), 80, 42, paths, plen, orc.Params(**P2), idx)


@pytest.mark.slow
def test_config3_rmat22_metapath_and_ppr_one_launch(orc):
    g = cached_graph("rmat", 22, 2)
    dg = device_graph(g)
    starts = fi.one_per_vertex(g.n, "cuda")
    outs = dg.walk_multi([
        dict(algo="metapath", starts=starts, max_len=80, seed=42, mode="exact"),
        dict(algo="ppr", starts=starts, max_len=100, seed=42, mode="exact", ppr_stop=0.2),
    ])
    torch.cuda.synchronize()
    (mp, ml), (pp, pl) = outs
    check_valid(g, mp, ml, "metapath")
    check_valid(g, pp, pl, "ppr")
    mp, ml, pp, pl = mp.cpu(), ml.cpu(), pp.cpu(), pl.cpu()
    idx = np.random.default_rng(1).choice(g.n, 200, replace=False)
    _sampled(orc, g, "metapath", starts.cpu(), 80, 42, mp, ml, orc.Params(), idx)
    _sampled(orc, g, "ppr", starts.cpu(), 100, 42, pp, pl, orc.Params(ppr_stop=0.2), idx)


@pytest.mark.slow
def test_rmat22_ppr_from_max_degree_vertex_sampled(orc):
    """The paper's PPR workload (Section 6.1): every query starts at the
    max-degree vertex (stop 0.2, cap 100), so every walk's first step
    competes for the CTAs' hub-task entries; 2^20 queries in one launch with
    the default tuning, 200 of them recomputed by the oracle."""
    g = cached_graph("rmat", 22, 2)
    dg = device_graph(g)
    deg = g.row_ptr[1:] - g.row_ptr[:-1]
    hub = int(deg.argmax())
    n_q = 1 << 20
    starts = torch.full((n_q,), hub, dtype=torch.int32, device="cuda")
    dg.stats_reset()
    paths, plen = dg.walk("ppr", starts, 100, 42, mode="exact", ppr_stop=0.2)
    st = dg.stats()
    check_valid(g, paths, plen, "ppr")
    assert st["block_steps"] >= n_q  # the first step of every walk is a hub row
    paths, plen = paths.cpu(), plen.cpu()
    idx = np.random.default_rng(5).choice(n_q, 200, replace=False)
    _sampled(orc, g, "ppr", starts.cpu(), 100, 42, paths, plen, orc.Params(ppr_stop=0.2), idx)
