"""fw_walk_noalloc: the walk launch for callers that cannot allocate device
memory when they walk (a serving loop that must not stall the device on an
allocation, or an application whose allocator owns all device memory).  Its
scratch is a static device array inside the library; its walks must equal the
allocating entry points' walks, call after call.

Collected last on purpose: a failure here leaves every other test already run.
"""

import numpy as np
import pytest
import torch

import fw_inputs as fi
from gpu_common import cached_graph, device_graph

pytestmark = pytest.mark.gpu


def _reqs(g, n_req, seed0):
    out = []
    algos = ["weighted", "node2vec", "metapath", "ppr"]
    for i in range(n_req):
        n_q = 37 + 11 * i
        starts = fi.random_starts(g.n, n_q, seed0 + i, "cuda")
        a = algos[i % 4]
        out.append(dict(algo=a, starts=starts, max_len=100 if a == "ppr" else 30, seed=seed0 * 1000 + i,
                        mode="exact", p=2.0, q=0.5, q_id0=1000 * i))
    return out


def test_noalloc_equals_allocating_entry_points_twice_in_a_row():
    g = cached_graph("rmat", 12, 2)
    dg = device_graph(g)
    for call, n_req in ((0, 12), (1, 40)):
        reqs = _reqs(g, n_req, 7 + call)
        got = dg.walk_noalloc(reqs)
        if n_req <= 16:
            ref = dg.walk_multi(reqs)
        else:  # beyond fw_walk_multi's inline table: one fw_walk per request
            ref = [dg.walk(r["algo"], r["starts"], r["max_len"], r["seed"], mode="exact", p=2.0, q=0.5,
                           q_id0=r["q_id0"]) for r in reqs]
        torch.cuda.synchronize()
        for (gp, gl), (rp, rl) in zip(got, ref):
            # exact mode: the tolerance is zero
            assert torch.equal(gl, rl)
            assert torch.equal(gp, rp)


def test_noalloc_rejects_too_many_requests():
    from paper_2404_08364_gb300 import _fw
    g = cached_graph("rmat", 8)
    dg = device_graph(g)
    s = torch.zeros(1, dtype=torch.int32, device="cuda")
    reqs = [dict(algo="weighted", starts=s, max_len=1, seed=1, mode="exact")] * 1025
    with pytest.raises(_fw.FwError) as e:
        dg.walk_noalloc(reqs)
    assert e.value.status == _fw.FW_EINVAL
