"""CUDA-graph replay of a mixed-length multi-request launch and the engine
autotuner: replays and tuned launches give the same walks as direct ones."""

import torch
import pytest

import fw_inputs as fi
from gpu_common import cached_graph, check_valid, device_graph

pytestmark = pytest.mark.gpu


def _mixed(g, seed):
    s = fi.random_starts(g.n, 3000, seed, "cuda")
    return [dict(algo="metapath", starts=s, max_len=80, seed=seed, mode="exact"),
            dict(algo="ppr", starts=s.clone(), max_len=100, seed=seed + 1, mode="exact", ppr_stop=0.2)]


def test_graph_replay_equals_direct_launch():
    g = cached_graph("rmat", 12, 2)
    dg = device_graph(g)
    reqs = _mixed(g, 3)
    ex = dg.capture_multi(reqs)
    (mp, ml), (pp, pl) = ex.launch()
    torch.cuda.synchronize()
    (rmp, rml), (rpp, rpl) = dg.walk_multi(reqs)
    torch.cuda.synchronize()
    assert torch.equal(mp, rmp) and torch.equal(ml, rml) and torch.equal(pp, rpp) and torch.equal(pl, rpl)
    # rewrite the starts in place and replay: the graph reads the new inputs
    new = fi.random_starts(g.n, 3000, 99, "cuda")
    reqs[0]["starts"].copy_(new)
    reqs[1]["starts"].copy_(new)
    (mp, ml), (pp, pl) = ex.launch()
    torch.cuda.synchronize()
    (rmp, rml), (rpp, rpl) = dg.walk_multi([dict(r, starts=new) for r in reqs])
    torch.cuda.synchronize()
    assert torch.equal(mp, rmp) and torch.equal(pp, rpp) and torch.equal(pl, rpl)
    check_valid(g, mp, ml, "metapath")
    ex.close()


def test_autotune_keeps_exact_results():
    from paper_2404_08364_gb300 import _fw
    _fw.lib().fw_autotune_clear_cache()
    g = cached_graph("rmat", 14, 2)
    dg = device_graph(g)
    reqs = _mixed(g, 5)
    before = dg.walk_multi(reqs)
    torch.cuda.synchronize()
    t = dg.autotune(reqs, reps=1)
    assert t["block_threads"] in (128, 256, 512) and t["steps_per_s"] > 0
    assert dg.get_tuning()["d_warp"] == t["d_warp"]
    after = dg.walk_multi(reqs)
    torch.cuda.synchronize()
    for (a, al), (b, bl) in zip(before, after):
        assert torch.equal(a, b) and torch.equal(al, bl)
    t2 = dg.autotune(reqs, reps=1)  # cached
    assert t2["steps_per_s"] == 0.0 and t2["d_warp"] == t["d_warp"]
