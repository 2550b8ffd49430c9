"""fw_walk_noalloc: the walk launch for callers that cannot allocate device
memory when they walk (a serving loop that must not stall the device on an
allocation, or an application whose allocator owns all device memory).  Its
scratch is a static device array inside the library; its walks must equal the
allocating entry points' walks, call after call, in both modes, up to the
array's 1024-request limit, and the errors of its launches must reach
fw_stats.

Collected last on purpose: a failure here leaves every other test already run.
"""

import pytest
import torch

import fw_inputs as fi
from gpu_common import cached_graph, device_graph

pytestmark = pytest.mark.gpu


def _reqs(g, n_req, seed0, mode="exact", sizes=None):
    out = []
    algos = ["weighted", "node2vec", "metapath", "ppr"]
    for i in range(n_req):
        n_q = sizes(i) if sizes else 37 + 11 * i
        starts = fi.random_starts(g.n, n_q, seed0 + i, "cuda")
        a = algos[i % 4]
        out.append(dict(algo=a, starts=starts, max_len=100 if a == "ppr" else 30, seed=seed0 * 1000 + i,
                        mode=mode, p=2.0, q=0.5, q_id0=1000 * i))
    return out


def _alone(dg, reqs):
    return [dg.walk(r["algo"], r["starts"], r["max_len"], r["seed"], mode=r["mode"], p=2.0, q=0.5,
                    q_id0=r["q_id0"]) for r in reqs]


def _equal(got, ref):
    # the same mode, seed and query ids on both sides: the tolerance is zero
    for (gp, gl), (rp, rl) in zip(got, ref):
        assert torch.equal(gl, rl)
        assert torch.equal(gp, rp)


def test_noalloc_equals_allocating_entry_points_twice_in_a_row():
    g = cached_graph("rmat", 12, 2)
    dg = device_graph(g)
    for call, n_req in ((0, 12), (1, 40)):
        reqs = _reqs(g, n_req, 7 + call)
        got = dg.walk_noalloc(reqs)
        # within fw_walk_multi's inline table: one launch; beyond: one fw_walk per request
        ref = dg.walk_multi(reqs) if n_req <= 16 else _alone(dg, reqs)
        torch.cuda.synchronize()
        _equal(got, ref)


def test_noalloc_fast_mode_twice_in_a_row():
    g = cached_graph("rmat", 14, 2)
    dg = device_graph(g)
    for call in range(2):
        reqs = _reqs(g, 16, 50 + call, mode="fast")
        got = dg.walk_noalloc(reqs)
        ref = dg.walk_multi(reqs)
        torch.cuda.synchronize()
        _equal(got, ref)


def test_noalloc_full_table_with_empty_requests():
    g = cached_graph("rmat", 10, 2)
    dg = device_graph(g)
    reqs = _reqs(g, 1024, 3, sizes=lambda i: 0 if i % 9 == 4 else 1 + i % 5)
    got = dg.walk_noalloc(reqs)
    ref = _alone(dg, reqs)
    torch.cuda.synchronize()
    _equal(got, ref)
    assert sum(1 for r in reqs if r["starts"].numel() == 0) > 100


def test_noalloc_errors_reach_stats():
    from paper_2404_08364_gb300 import _fw
    g = cached_graph("rmat", 10, 2)
    dg = device_graph(g)
    dg.stats_reset()
    reqs = _reqs(g, 3, 9)
    reqs[1]["starts"][5] = -1
    reqs[2]["starts"][0] = g.n
    got = dg.walk_noalloc(reqs)
    torch.cuda.synchronize()
    with pytest.raises(_fw.FwError) as e:
        dg.stats()
    assert e.value.status == _fw.FW_EINVAL
    assert int(got[1][1][5]) == 0 and bool((got[1][0][5] == -1).all())
    assert int(got[2][1][0]) == 0
    dg.stats_reset()
    ok = _reqs(g, 3, 9)
    got = dg.walk_noalloc(ok)
    st = dg.stats()
    assert st["walks"] == sum(r["starts"].numel() for r in ok)
    assert st["steps"] == sum(int((l - 1).sum()) for _, l in got)


def test_noalloc_rejects_too_many_requests():
    from paper_2404_08364_gb300 import _fw
    g = cached_graph("rmat", 8)
    dg = device_graph(g)
    s = torch.zeros(1, dtype=torch.int32, device="cuda")
    reqs = [dict(algo="weighted", starts=s, max_len=1, seed=1, mode="exact")] * 1025
    with pytest.raises(_fw.FwError) as e:
        dg.walk_noalloc(reqs)
    assert e.value.status == _fw.FW_EINVAL
