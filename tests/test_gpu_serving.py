"""Serving form: several resident graphs, requests admitted as slots and memory allow,
concurrent updates of different graphs, continuous batching of one graph's queue.

The check the serving form must pass: each graph's result is the same alone and in the
mix.  Without coalescing the mixed run performs exactly the standalone sequence of updates
per graph, so the ranks are bit-identical; with coalescing a queue of requests is served
by one Dynamic Frontier call, so the ranks agree within the path's tolerance.
"""
import numpy as np
import pytest

import __graft_entry__
import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    from paper_2401_03256_gb300 import prdf

    prdf.load()
    return prdf, torch


def _workload(scales, per_graph, seed):
    rng = np.random.default_rng(seed)
    gs = [synth.rmat(int(s), 8, seed=seed + i) for i, s in enumerate(scales)]
    reqs = []
    for i, g in enumerate(gs):
        st = synth.BatchStream(g, seed=seed + 50 + i)
        fr = np.exp(rng.uniform(np.log(1e-4), np.log(3e-2), per_graph))
        reqs.append([st.next(float(f)) for f in fr])
    return gs, reqs


def _params(prdf, prec):
    p = prdf.pr_params_default()
    p.precision = prec
    return p


def _alone(prdf, torch, g, batches, params):
    s = torch.cuda.Stream()
    with prdf.Graph(g.n, g.src, g.dst, params, s.cuda_stream) as A:
        A.static()
        for b in batches:
            A.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            A.frontier()
        return A.ranks().copy()


def _mixed(prdf, torch, gs, reqs, params, slots, coalesce, reserve=0):
    streams = [torch.cuda.Stream() for _ in gs]
    hs = [prdf.Graph(g.n, g.src, g.dst, params, s.cuda_stream) for g, s in zip(gs, streams)]
    for h in hs:
        h.static()
    srv = prdf.Server(slots=slots, max_coalesce=coalesce, hbm_reserve_bytes=reserve)
    idx = [srv.add(h) for h in hs]
    order = [(gi, k) for k in range(len(reqs[0])) for gi in range(len(gs))]
    rng = np.random.default_rng(3)
    rng.shuffle(order)
    order.sort(key=lambda t: t[1])  # each graph's requests in sequence, graphs interleaved
    tickets = {}
    for gi, k in order:
        b = reqs[gi][k]
        tickets[(gi, k)] = srv.submit(idx[gi], b.del_src, b.del_dst, b.ins_src, b.ins_dst)
    info = srv.drain()
    results = {key: srv.wait(t) for key, t in tickets.items()}
    srv.close()
    ranks = [h.ranks().copy() for h in hs]
    for h in hs:
        h.close()
    return ranks, results, info


def test_mixed_equals_alone_bitwise_without_coalescing(env):
    prdf, torch = env
    gs, reqs = _workload([11, 12, 13, 14], 12, seed=10)
    p = _params(prdf, prdf.PR_F64)
    ranks, results, info = _mixed(prdf, torch, gs, reqs, p, slots=3, coalesce=1)
    assert info.completed == info.submitted == 4 * 12
    assert all(r.status == prdf.PR_OK and r.coalesced == 1 for r in results.values())
    for gi, g in enumerate(gs):
        assert np.array_equal(ranks[gi], _alone(prdf, torch, g, reqs[gi], p)), gi
        # per graph, requests finished in submission order
        done = [results[(gi, k)].t_done_ms for k in range(12)]
        assert done == sorted(done)


def test_mixed_matches_oracle_chain(env):
    prdf, torch = env
    gs, reqs = _workload([10, 11], 6, seed=20)
    p = _params(prdf, prdf.PR_F64)
    ranks, _, _ = _mixed(prdf, torch, gs, reqs, p, slots=2, coalesce=1)
    for gi, g in enumerate(gs):
        G = oracle.Graph.build(g.n, g.src, g.dst)
        R, _ = oracle.static_pr(G)
        for b in reqs[gi]:
            H, ed, ei = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            R, _, _ = oracle.df_sync(G, H, ed, ei, R)
            G = H
        assert np.max(np.abs(ranks[gi] - R)) <= 1e-9


def test_coalesced_within_tolerance_fp32(env):
    prdf, torch = env
    gs, reqs = _workload([12, 13, 14], 16, seed=30)
    p = _params(prdf, prdf.PR_F32)
    ranks, results, info = _mixed(prdf, torch, gs, reqs, p, slots=2, coalesce=64)
    assert info.completed == 3 * 16
    assert max(r.coalesced for r in results.values()) > 1
    for gi, g in enumerate(gs):
        alone = _alone(prdf, torch, g, reqs[gi], p)
        assert np.max(np.abs(ranks[gi] - alone)) <= 1e-6


def test_memory_admission_serialises_when_reserve_is_unmet(env):
    prdf, torch = env
    gs, reqs = _workload([10, 10, 10], 4, seed=40)
    p = _params(prdf, prdf.PR_F64)
    total = torch.cuda.get_device_properties(0).total_memory
    ranks, results, info = _mixed(prdf, torch, gs, reqs, p, slots=3, coalesce=1, reserve=2 * total)
    assert info.completed == 12 and info.waited_for_memory >= 1
    # with no headroom the device admits one request at a time: the updates never overlap
    spans = sorted((r.t_start_ms, r.t_done_ms) for r in results.values())
    for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
        assert s1 >= e0 - 1e-6
    for gi, g in enumerate(gs):
        assert np.array_equal(ranks[gi], _alone(prdf, torch, g, reqs[gi], p))


def test_server_rejects_bad_graph_index(env):
    prdf, torch = env
    srv = prdf.Server(slots=1)
    with pytest.raises(prdf.PrdfError):
        srv.submit(0, [1], [2], [], [])
    srv.close()
