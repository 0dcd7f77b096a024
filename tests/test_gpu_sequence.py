"""Sequences of batches applied by one call (pr_apply_batches).

The graph after a sequence must be exactly the graph after applying its batches one by
one (Section 3.2 per batch: deletions, then insertions, the insertion winning when a pair
is both deleted and inserted), CSR compared bit for bit; a Dynamic Frontier call after it
must reach the oracle's ranks for the final graph.
"""
import numpy as np
import pytest

import __graft_entry__
import oracle
import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-9


@pytest.fixture(scope="module")
def prdf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    from paper_2401_03256_gb300 import prdf as mod

    mod.load()
    return mod


def _stream_batches(g, k, frac, seed):
    st = synth.BatchStream(g, seed=seed)
    return [st.next(frac) for _ in range(k)]


def _as_tuple(b):
    return (b.del_src, b.del_dst, b.ins_src, b.ins_dst)


def _same_csr(A, B):
    for d in (0, 1):
        oa, ca = A.csr(d)
        ob, cb = B.csr(d)
        assert np.array_equal(oa, ob) and np.array_equal(ca, cb), d


@pytest.mark.parametrize("scale,k,frac", [(8, 5, 2e-2), (12, 8, 1e-2), (14, 3, 5e-2)])
def test_sequence_equals_one_by_one(prdf, scale, k, frac):
    # small sequences use the one-block sort, larger ones the radix sort
    g = synth.rmat(scale, 8, seed=scale)
    bs = _stream_batches(g, k, frac, seed=scale + 1)
    with prdf.Graph(g.n, g.src, g.dst) as S, prdf.Graph(g.n, g.src, g.dst) as Q:
        for b in bs:
            S.apply(*_as_tuple(b))
        Q.apply_batches([_as_tuple(b) for b in bs])
        _same_csr(S, Q)


def test_cancelling_requests_across_batches(prdf):
    # an edge deleted then re-inserted, inserted then deleted, inserted twice, deleted
    # twice, plus pairs deleted and inserted inside one batch and self pairs
    n = 64
    pairs = [(i, (i * 7 + 3) % n) for i in range(n) if i != (i * 7 + 3) % n]
    g = synth.from_pairs(n, pairs, "ring7")
    e0, e1, e2 = pairs[0], pairs[1], pairs[2]
    new = [(5, 40), (6, 41), (7, 42)]
    seq = [
        ([e0, e1], [new[0], (9, 9)]),            # delete e0, e1; insert new0 and a self pair
        ([new[0]], [e0, new[1], new[1]]),        # delete new0; re-insert e0; insert new1 twice
        ([new[1], new[1], e2], [e2, new[2]]),    # delete new1 twice; e2 deleted and inserted
        ([], []),                                # empty batch
        ([new[2]], [new[2]]),                    # deleted and inserted in one batch: present
    ]

    def arr(ps):
        a = np.asarray(ps, dtype=np.uint32).reshape(-1, 2)
        return a[:, 0].copy(), a[:, 1].copy()

    bts = [(*arr(d), *arr(i)) for d, i in seq]
    with prdf.Graph(g.n, g.src, g.dst) as S, prdf.Graph(g.n, g.src, g.dst) as Q:
        for b in bts:
            S.apply(*b)
        Q.apply_batches(bts)
        _same_csr(S, Q)
        off, col = Q.csr(0)
        have = {(u, int(v)) for u in range(n) for v in col[off[u]:off[u + 1]]}
        assert e0 in have and e2 in have and new[2] in have
        assert e1 not in have and new[0] not in have and new[1] not in have
        assert (9, 9) in have  # the fixed self-loop (Section 5.1.4), untouched


def test_sequence_then_frontier_matches_oracle(prdf):
    g = synth.rmat(12, 8, seed=31)
    bs = _stream_batches(g, 6, 5e-3, seed=32)
    G = oracle.Graph.build(g.n, g.src, g.dst)
    R0, _ = oracle.static_pr(G)
    H = G
    for b in bs:
        H, _, _ = H.apply(*_as_tuple(b))
    Rref, _ = oracle.static_pr(H)
    with prdf.Graph(g.n, g.src, g.dst) as Q:
        Q.set_ranks(R0)
        Q.apply_batches([_as_tuple(b) for b in bs])
        st = Q.frontier()
        assert st.converged
        # the converged ranks of the final graph, within the path's L-inf bound
        assert np.max(np.abs(Q.ranks() - Rref)) <= 1e-8
        oq, cq = Q.csr(0)
        oh, ch = H.csr(0)
        assert np.array_equal(oq, oh) and np.array_equal(cq, ch)


def test_sequence_rejects_bad_offsets_and_ids(prdf):
    g = synth.rmat(8, 8, seed=2)
    lib = prdf.load()
    with prdf.Graph(g.n, g.src, g.dst) as Q:
        before = Q.csr(0)
        with pytest.raises(prdf.PrdfError) as e:
            Q.apply_batches([([1], [2], [], []), ([g.n], [0], [], [])])
        assert e.value.status == prdf.PR_ERR_VERTEX_RANGE
        z = np.zeros(1, np.uint32)
        bad = np.asarray([0, 2, 1], dtype=np.int64)  # decreasing offsets
        ok = np.asarray([0, 0, 0], dtype=np.int64)
        st = lib.pr_apply_batches(Q.h, 2, bad.ctypes.data, z.ctypes.data, z.ctypes.data, ok.ctypes.data,
                                  z.ctypes.data, z.ctypes.data)
        assert st == prdf.PR_ERR_INVALID_ARG
        after = Q.csr(0)
        assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])


@pytest.mark.parametrize("order", [1, 0])
def test_long_row_merges(prdf, order):
    # a hub with 20,000 in- and out-edges: its rows are merged by the long-row pass (rows of
    # more than 8192 entries); insertions below, between and above its present columns and
    # deletions among them must give the oracle's CSR bit for bit, then its ranks
    rng = np.random.default_rng(41)
    n = 60000
    hub = 777
    others = rng.choice(np.setdiff1d(np.arange(n), [hub]), size=40000, replace=False)
    ins_to, outs_from = others[:20000], others[20000:]
    pairs = [(int(u), hub) for u in ins_to] + [(hub, int(v)) for v in outs_from]
    extra = rng.integers(0, n, size=(120000, 2))
    pairs += [(int(a), int(b)) for a, b in extra]
    g = synth.from_pairs(n, pairs, "hub")
    G = oracle.Graph.build(g.n, g.src, g.dst)
    R0, _ = oracle.static_pr(G)
    free_in = np.setdiff1d(np.arange(n), np.concatenate([ins_to, [hub]]))
    new_in = rng.choice(free_in, size=3000, replace=False)
    del_in = rng.choice(ins_to, size=2500, replace=False)
    free_out = np.setdiff1d(np.arange(n), np.concatenate([outs_from, [hub]]))
    new_out = rng.choice(free_out, size=3000, replace=False)
    del_out = rng.choice(outs_from, size=2500, replace=False)
    u32 = lambda a: np.asarray(a, np.uint32)
    ds = u32(np.concatenate([del_in, np.full(len(del_out), hub)]))
    dd = u32(np.concatenate([np.full(len(del_in), hub), del_out]))
    is_ = u32(np.concatenate([new_in, np.full(len(new_out), hub)]))
    id_ = u32(np.concatenate([np.full(len(new_in), hub), new_out]))
    p = prdf.pr_params_default()
    p.vertex_order = order
    with prdf.Graph(g.n, g.src, g.dst, p) as Q:
        Q.set_ranks(R0)
        Q.apply(ds, dd, is_, id_)
        H, ed, ei = G.apply(ds, dd, is_, id_)
        for d in (0, 1):
            off, col = Q.csr(d)
            eoff, ecol = H.csr(d)
            assert np.array_equal(off, eoff) and np.array_equal(col, ecol)
        Q.frontier()
        R_df, _, _ = oracle.df_sync(G, H, ed, ei, R0)
        assert np.max(np.abs(Q.ranks() - R_df)) <= TOL64
