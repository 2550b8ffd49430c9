"""The engine's counters recount on the host: rows scanned = the sum of
deg(cur) over every move of the returned paths, steps = moves, algorithmic
bytes = 8 d + (1 d for MetaPath labels) + 16 + 4 per move, warp + CTA steps =
steps.  Checked with the default tuning and with d_t = 256 (many rows go to
the CTA hub tasks)."""

import pytest
import torch

import fw_inputs as fi
from gpu_common import cached_graph, device_graph

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d_warp", [0, 256])
@pytest.mark.parametrize("mode", ["exact", "fast"])
@pytest.mark.parametrize("algo", ["weighted", "node2vec", "metapath"])
def test_counters_recount(algo, mode, d_warp):
    g = cached_graph("rmat", 14, 2)
    dg = device_graph(g)
    if d_warp:
        dg.set_tuning(d_warp=d_warp)
    n_q, L = 4000, 40
    starts = fi.random_starts(g.n, n_q, 31).cuda()
    dg.stats_reset()
    paths, plen = dg.walk(algo, starts, L, 5, mode=mode, p=2.0, q=0.5)
    st = dg.stats()
    deg = (g.row_ptr[1:] - g.row_ptr[:-1]).to(torch.int64).cuda()
    t = torch.arange(L + 1, device="cuda")[None, :]
    moved_from = (t < (plen[:, None].to(torch.int64) - 1)) & (paths >= 0)
    d = torch.where(moved_from, deg[paths.clamp(min=0).to(torch.int64)], torch.zeros_like(paths, dtype=torch.int64))
    rows = int(d.sum())
    moves = int((plen - 1).sum())
    assert st["steps"] == moves
    assert st["rows_scanned"] == rows
    assert st["warp_steps"] + st["block_steps"] == moves
    per_entry = 9 if algo == "metapath" else 8
    assert st["algo_bytes"] == per_entry * rows + 20 * moves
    assert st["n2v_tests"] == (rows if algo == "node2vec" else 0)
    if d_warp:
        assert st["block_steps"] > 0
