"""Served form: continuous batching keeps every request's result equal to the
same request run alone, whatever else is on the GPU, and serves requests
that arrive while others run."""

import threading
import time

import numpy as np
import pytest
import torch

import fw_inputs as fi
from gpu_common import cached_graph, check_valid, device_graph

# a served run that stops making progress fails the test instead of hanging it
pytestmark = [pytest.mark.gpu, pytest.mark.timeout(180)]

ALGOS = ["weighted", "node2vec", "metapath", "ppr"]


def _mix(g, n_req, seed0, rng):
    reqs = []
    for i in range(n_req):
        n_q = int(2 ** rng.uniform(0, 11))
        a = ALGOS[i % 4]
        L = 100 if a == "ppr" else int(rng.integers(10, 81))
        reqs.append(dict(algo=a, starts=fi.random_starts(g.n, n_q, seed0 + i), max_len=L, seed=seed0 * 977 + i,
                         p=2.0, q=0.5, lengths=fi.uniform_lengths(n_q, 0, L, seed0 + 3 * i) if i % 3 == 0 else None))
    return reqs


@pytest.mark.parametrize("mode", ["exact", "fast"])
def test_alone_equals_in_the_mix(orc, mode):
    from paper_2404_08364_gb300 import Server
    g = cached_graph("rmat", 14, 2)
    dg = device_graph(g)
    rng = np.random.default_rng(3)
    reqs = _mix(g, 24, 11, rng)
    srv = Server(dg, mode=mode, mem_budget=64 << 20)
    tickets = [srv.submit(**r) for r in reqs]
    outs = [srv.result(t) for t in tickets]
    srv.close()
    csr = orc.CSR(g)
    for r, (paths, plen, lat) in zip(reqs, outs):
        alone_p, alone_l = dg.walk(r["algo"], r["starts"].cuda(), r["max_len"], r["seed"], mode=mode, p=2.0, q=0.5,
                                   lengths=None if r["lengths"] is None else r["lengths"].cuda())
        assert torch.equal(plen, alone_l.cpu()), r["algo"]
        assert torch.equal(paths, alone_p.cpu()), r["algo"]
        assert lat > 0
        if mode == "exact":
            # and both equal the oracle, element by element
            ref_p, ref_l = orc.walk_exact(csr, r["algo"], orc.Params(p=2.0, q=0.5), r["starts"], r["max_len"],
                                          r["seed"], lengths=r["lengths"])
            assert np.array_equal(plen.numpy(), ref_l), r["algo"]
            assert np.array_equal(paths.numpy(), ref_p), r["algo"]


def test_requests_arriving_while_others_run():
    from paper_2404_08364_gb300 import Server
    g = cached_graph("rmat", 16, 2)
    dg = device_graph(g)
    rng = np.random.default_rng(5)
    srv = Server(dg, mode="fast", mem_budget=16 << 20, idle_ms=5.0)  # small arena: admission must wait for memory
    reqs = _mix(g, 60, 101, rng)
    tickets = []
    for i, r in enumerate(reqs):
        tickets.append(srv.submit(**r))
        if i % 7 == 0:
            time.sleep(0.002)
    lat = []
    for r, t in zip(reqs, tickets):
        paths, plen, l = srv.result(t)
        lat.append(l)
        check_valid(g, paths.cuda(), plen.cuda(), r["algo"])
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs)
    assert st["arena_used"] == 0
    assert st["steps"] > 0


def test_idle_engine_is_relaunched():
    from paper_2404_08364_gb300 import Server
    g = cached_graph("rmat", 12, 2)
    dg = device_graph(g)
    srv = Server(dg, mode="exact", mem_budget=8 << 20, idle_ms=2.0)
    s = fi.random_starts(g.n, 100, 1)
    a = srv.result(srv.submit("weighted", s, 20, 5))
    time.sleep(0.1)  # the engine returns after 2 ms of idleness
    b = srv.result(srv.submit("weighted", s, 20, 5))
    st = srv.stats()
    srv.close()
    assert torch.equal(a[0], b[0])
    assert st["launches"] >= 2


def test_ring_slots_reused_many_times():
    """A 4-entry request ring for 40 requests: each slot is refilled about
    ten times while the engine keeps running, and every result still equals
    the request run alone (exact mode: bit for bit)."""
    from paper_2404_08364_gb300 import Server
    g = cached_graph("rmat", 14, 2)
    dg = device_graph(g)
    rng = np.random.default_rng(9)
    reqs = _mix(g, 40, 303, rng)
    srv = Server(dg, mode="exact", mem_budget=64 << 20, max_requests=4, idle_ms=50.0)
    tickets = [srv.submit(**r) for r in reqs]
    outs = [srv.result(t) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs)
    for r, (paths, plen, _) in zip(reqs, outs):
        alone_p, alone_l = dg.walk(r["algo"], r["starts"].cuda(), r["max_len"], r["seed"], mode="exact", p=2.0,
                                   q=0.5, lengths=None if r["lengths"] is None else r["lengths"].cuda())
        assert torch.equal(plen, alone_l.cpu()), r["algo"]
        assert torch.equal(paths, alone_p.cpu()), r["algo"]


def test_engine_returns_on_its_own_idle_limit_and_is_relaunched(orc):
    """The host's idle stop (idle_ms) is set above the engine's own 2-s
    device-side idle limit, so the engine's warps return by themselves after
    2 s without work (a bounded wait running out, with no fault); the next
    request must still be served, by a relaunched engine, with the right
    result."""
    from paper_2404_08364_gb300 import Server
    g = cached_graph("rmat", 12, 2)
    dg = device_graph(g)
    srv = Server(dg, mode="exact", mem_budget=8 << 20, idle_ms=60000.0)
    s = fi.random_starts(g.n, 200, 3)
    a = srv.result(srv.submit("node2vec", s, 20, 5, p=2.0, q=0.5))
    launches0 = srv.stats()["launches"]
    time.sleep(3.0)  # longer than the engine's 2 s device idle limit, far below idle_ms
    b = srv.result(srv.submit("node2vec", s, 20, 5, p=2.0, q=0.5))
    st = srv.stats()
    srv.close()
    assert launches0 == 1 and st["launches"] == 2
    ref_p, ref_l = orc.walk_exact(orc.CSR(g), "node2vec", orc.Params(p=2.0, q=0.5), s, 20, 5)
    for paths, plen, _ in (a, b):
        assert np.array_equal(plen.numpy(), ref_l)
        assert np.array_equal(paths.numpy(), ref_p)
