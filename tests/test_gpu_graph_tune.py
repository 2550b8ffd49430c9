"""CUDA-graph replay of a mixed-length multi-request launch and the engine
autotuner: replays and tuned launches give the oracle's walks (exact mode)
and the same walks as direct launches (both modes)."""

import numpy as np
import pytest
import torch

import fw_inputs as fi
from gpu_common import cached_graph, check_valid, compare_sampled, device_graph

pytestmark = pytest.mark.gpu


def _mixed(g, seed, mode="exact", n=3000):
    s = fi.random_starts(g.n, n, seed, "cuda")
    return [dict(algo="metapath", starts=s, max_len=80, seed=seed, mode=mode),
            dict(algo="ppr", starts=s.clone(), max_len=100, seed=seed + 1, mode=mode, ppr_stop=0.2)]


def _oracle_equal(orc, g, reqs, outs):
    csr = orc.CSR(g)
    for r, (p, l) in zip(reqs, outs):
        prm = orc.Params(ppr_stop=r.get("ppr_stop", 0.2))
        ref_p, ref_l = orc.walk_exact(csr, r["algo"], prm, r["starts"].cpu(), r["max_len"], r["seed"])
        assert np.array_equal(l.cpu().numpy(), ref_l), r["algo"]
        assert np.array_equal(p.cpu().numpy(), ref_p), r["algo"]


def test_graph_replay_equals_oracle_and_direct_launch(orc):
    g = cached_graph("rmat", 12, 2)
    dg = device_graph(g)
    reqs = _mixed(g, 3)
    ex = dg.capture_multi(reqs)
    (mp, ml), (pp, pl) = ex.launch()
    torch.cuda.synchronize()
    _oracle_equal(orc, g, reqs, [(mp, ml), (pp, pl)])
    (rmp, rml), (rpp, rpl) = dg.walk_multi(reqs)
    torch.cuda.synchronize()
    assert torch.equal(mp, rmp) and torch.equal(ml, rml) and torch.equal(pp, rpp) and torch.equal(pl, rpl)
    # rewrite the starts in place and replay: the graph reads the new inputs
    new = fi.random_starts(g.n, 3000, 99, "cuda")
    reqs[0]["starts"].copy_(new)
    reqs[1]["starts"].copy_(new)
    (mp, ml), (pp, pl) = ex.launch()
    torch.cuda.synchronize()
    _oracle_equal(orc, g, reqs, [(mp, ml), (pp, pl)])
    (rmp, rml), (rpp, rpl) = dg.walk_multi([dict(r, starts=new) for r in reqs])
    torch.cuda.synchronize()
    assert torch.equal(mp, rmp) and torch.equal(pp, rpp) and torch.equal(pl, rpl)
    check_valid(g, mp, ml, "metapath")
    ex.close()


@pytest.mark.parametrize("mode", ["exact", "fast"])
def test_autotune_keeps_results(orc, mode):
    from paper_2404_08364_gb300 import _fw
    _fw.lib().fw_autotune_clear_cache()
    g = cached_graph("rmat", 14, 2)
    dg = device_graph(g)
    reqs = _mixed(g, 5, mode)
    before = dg.walk_multi(reqs)
    torch.cuda.synchronize()
    t = dg.autotune(reqs, reps=1)
    assert t["block_threads"] in (128, 256, 512) and t["steps_per_s"] > 0
    assert dg.get_tuning()["d_warp"] == t["d_warp"]
    after = dg.walk_multi(reqs)
    torch.cuda.synchronize()
    # no tuning changes a result, in either mode
    for (a, al), (b, bl) in zip(before, after):
        assert torch.equal(a, b) and torch.equal(al, bl)
    if mode == "exact":
        _oracle_equal(orc, g, reqs, after)
    t2 = dg.autotune(reqs, reps=1)  # cached
    assert t2["steps_per_s"] == 0.0 and t2["d_warp"] == t["d_warp"]


@pytest.mark.slow
def test_config3_autotuned_one_launch_matches_oracle(orc):
    """Config 3 as stated: MetaPath (schema 0..4 repeated, length 80) and PPR
    (stop 0.2, cap 100) on labeled R-MAT-22, one query per vertex each,
    batched in one launch with the autotuner's sampler threshold and launch
    shape; 200 sampled queries of each recomputed by the oracle."""
    from paper_2404_08364_gb300 import _fw
    _fw.lib().fw_autotune_clear_cache()
    g = cached_graph("rmat", 22, 2)
    dg = device_graph(g)
    starts = fi.one_per_vertex(g.n, "cuda")
    reqs = [dict(algo="metapath", starts=starts, max_len=80, seed=42, mode="exact"),
            dict(algo="ppr", starts=starts, max_len=100, seed=42, mode="exact", ppr_stop=0.2)]
    sample = [dict(r, starts=fi.random_starts(g.n, 1 << 16, 8, "cuda")) for r in reqs]
    t = dg.autotune(sample, reps=1)
    assert dg.get_tuning() == {k: t[k] for k in ("block_threads", "slots", "d_warp", "ctas_per_sm")}
    (mp, ml), (pp, pl) = dg.walk_multi(reqs)
    torch.cuda.synchronize()
    check_valid(g, mp, ml, "metapath")
    check_valid(g, pp, pl, "ppr")
    mp, ml, pp, pl = mp.cpu(), ml.cpu(), pp.cpu(), pl.cpu()
    idx = np.random.default_rng(3).choice(g.n, 200, replace=False)
    compare_sampled(orc, g, "metapath", starts.cpu(), 80, 42, mp, ml, orc.Params(), idx)
    compare_sampled(orc, g, "ppr", starts.cpu(), 100, 42, pp, pl, orc.Params(ppr_stop=0.2), idx)
