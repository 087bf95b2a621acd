"""Serving runtime (continuous batching) on the GPU: results of requests in a mixed,
overlapping load equal the same request run alone and the oracle; admission by the
memory budget; shutdown and graph-lifetime rules."""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
RTOL, ATOL = 1e-9, 1e-12


@pytest.fixture(scope="module")
def nk():
    import torch
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    from paper_1403_3005_gb300 import nk as _nk
    _nk.lib()
    return _nk


MIX = [("er", 3000, 11, dict(avg_deg=8.0), 64), ("ba", 20000, 12, dict(m0=4), 300),
       ("rmat", 13, 13, {}, 1024), ("er", 1200, 14, dict(avg_deg=8.0), 200),
       ("rmat", 15, 15, {}, 77), ("ba", 5000, 16, dict(m0=4), 129)]


def test_mixed_load_equals_alone_and_oracle(nk):
    graphs = [(nk.graph_generate(kind, size, seed, **p), oracle.generate(kind, size, seed, **p), k)
              for kind, size, seed, p, k in MIX]
    srv = nk.Server(max_inflight=4)
    reqs = []
    for rep in range(3):  # every graph three times, with different seeds, all in flight
        for i, (g, _, k) in enumerate(graphs):
            rid, out = srv.submit(g, 100 * rep + i, k)
            reqs.append((rid, out, i, 100 * rep + i))
    for rid, out, i, seed in reqs:
        assert srv.wait(rid, 300.0) == nk.OK
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["peak_inflight"] >= 2, st          # requests overlapped on the device
    assert st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()
    for rid, out, i, seed in reqs:
        g, (n, rp, col), k = graphs[i]
        alone = nk.betweenness_sampled(g, seed, k, nk.run_opts(mode=nk.MODE_BATCHED, batch=64))
        assert np.allclose(out, alone, rtol=RTOL, atol=ATOL)
        if seed < 100:
            assert np.allclose(out, oracle.betweenness_sampled(rp, col, seed, k), rtol=RTOL, atol=ATOL)


def test_small_requests_packed_into_one_launch(nk):
    # many small requests on different graphs (and the same graph twice), k <= 128:
    # packed launches on the union of their graphs; each result equals the request alone
    # and the oracle
    specs = [("er", 900, 31, dict(avg_deg=6.0), 40), ("ba", 2000, 32, dict(m0=3), 100),
             ("rmat", 10, 33, {}, 64), ("er", 300, 34, dict(avg_deg=4.0), 7),
             ("ba", 5000, 35, dict(m0=4), 128), ("rmat", 12, 36, {}, 90)]
    graphs = [(nk.graph_generate(kd, sz, sd, **p), oracle.generate(kd, sz, sd, **p), k)
              for kd, sz, sd, p, k in specs]
    for pack in (True, False):
        srv = nk.Server(max_inflight=1, pack=pack)   # one slot: the queue forms packs
        reqs = []
        for rep in range(2):
            for i, (g, _, k) in enumerate(graphs):
                rid, out = srv.submit(g, 7 + rep, k)
                reqs.append((rid, out, i, 7 + rep))
        for rid, out, i, seed in reqs:
            assert srv.wait(rid, 300.0) == nk.OK
        st = srv.stats()
        srv.close()
        if pack:
            assert st["packed_requests"] >= 2 and st["jobs"] < len(reqs), st
        else:
            assert st["packed_requests"] == 0 and st["jobs"] == len(reqs), st
        for rid, out, i, seed in reqs:
            g, (n, rp, col), k = graphs[i]
            assert np.allclose(out, oracle.betweenness_sampled(rp, col, seed, k), rtol=RTOL, atol=ATOL), (pack, i)


def test_admission_by_budget_and_rejection(nk):
    g = nk.graph_generate("rmat", 14, 3)
    probe = nk.Server(max_inflight=1, pack=False)
    assert probe.wait(probe.submit(g, 0, 100)[0], 300.0) == nk.OK
    need = probe.stats()["peak_bytes"]          # device bytes admitted for one request
    probe.close()
    assert need > 0
    # a budget that holds one request at a time: requests queue, then all finish
    srv = nk.Server(mem_budget_bytes=1.5 * need, max_inflight=4, pack=False)
    ids = [srv.submit(g, s, 100)[0] for s in range(5)]
    for i in ids:
        assert srv.wait(i, 300.0) == nk.OK
    assert srv.stats()["peak_inflight"] == 1
    srv.close()
    small = nk.Server(mem_budget_bytes=1e5)
    with pytest.raises(nk.NkError) as e:
        small.submit(g, 1, 100)
    assert e.value.rc == nk.ERR_NOMEM
    assert small.stats()["rejected"] == 1
    small.close()


def test_graph_free_refused_while_pending_and_poll(nk):
    g = nk.graph_generate("ba", 200000, 5, m0=4)
    srv = nk.Server(max_inflight=1)
    ids = [srv.submit(g, s, 1024)[0] for s in range(4)]
    with pytest.raises(nk.NkError) as e:
        g.free()
    assert e.value.rc == nk.ERR_ARG
    states = {i: srv.poll(i) for i in ids}
    assert states[ids[-1]] == nk.PENDING      # one slot, four requests: the last still waits
    for i, rc in states.items():
        assert (srv.wait(i, 300.0) if rc == nk.PENDING else rc) == nk.OK
    srv.close()
    g.free()


def test_submit_argument_errors(nk):
    g = nk.graph_generate("er", 100, 1, avg_deg=4.0)
    srv = nk.Server()
    for k in (0, 101):
        with pytest.raises(nk.NkError) as e:
            srv.submit(g, 1, k)
        assert e.value.rc == nk.ERR_ARG
    assert nk.lib().nk_serve_poll(srv._h, 12345) == nk.ERR_ARG
    srv.close()
