"""Batched form: many independent graphs in one handle, one launch per rank call.

Each graph of a batched handle must give the ranks of a run of that graph alone: the same
values as a standalone handle (bit for bit in 64-bit mode, whose sums are exact) and the
oracle's within the usual L-inf bound, with its own iteration count.
"""
import numpy as np
import pytest

import __graft_entry__
import oracle
import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-9
TOL32 = 1e-6


@pytest.fixture(scope="module")
def prdf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    from paper_2401_03256_gb300 import prdf as mod

    mod.load()
    return mod


def _graphs(seed=0):
    rng = np.random.default_rng(seed)
    gs = [synth.rmat(int(s), 8, seed=100 + i) for i, s in enumerate(rng.integers(6, 12, 9))]
    n = 17
    gs.append(synth.from_pairs(n, [(i, (i + 1) % n) for i in range(n)], "cycle"))
    gs.append(synth.from_pairs(21, [(i, 0) for i in range(1, 21)], "star"))
    gs.append(synth.from_pairs(3, [], "empty"))
    return gs


def _union(gs):
    firsts = np.cumsum([0] + [g.n for g in gs])
    src = np.concatenate([g.src.astype(np.uint64) + firsts[i] for i, g in enumerate(gs)]).astype(np.uint32)
    dst = np.concatenate([g.dst.astype(np.uint64) + firsts[i] for i, g in enumerate(gs)]).astype(np.uint32)
    return firsts, src, dst


def _params(prdf, **kw):
    p = prdf.pr_params_default()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("graph_launch", [False, True])
def test_batched_static_equals_standalone_and_oracle(prdf, graph_launch):
    gs = _graphs()
    firsts, src, dst = _union(gs)
    with prdf.Graph.batched([g.n for g in gs], src, dst) as B:
        B.set_graph_launch(graph_launch)
        st = B.static()
        R = B.ranks()
        cs = B.component_stats()
        assert st.converged and st.iterations == max(c.iterations for c in cs)
        for i, g in enumerate(gs):
            part = R[firsts[i]:firsts[i + 1]]
            with prdf.Graph(g.n, g.src, g.dst) as A:
                sa = A.static()
                assert np.array_equal(A.ranks(), part), g.name
                assert cs[i].iterations == sa.iterations and cs[i].converged
            G = oracle.Graph.build(g.n, g.src, g.dst)
            Ro, so = oracle.static_pr(G)
            assert np.max(np.abs(part - Ro)) <= TOL64
            assert abs(cs[i].iterations - so.iterations) <= 1


def test_batched_apply_and_frontier(prdf):
    gs = _graphs(1)
    firsts, src, dst = _union(gs)
    streams = [synth.BatchStream(g, seed=7 + i) for i, g in enumerate(gs)]
    Gs = [oracle.Graph.build(g.n, g.src, g.dst) for g in gs]
    Rs = [oracle.static_pr(G)[0] for G in Gs]
    U = oracle.Graph.build(int(firsts[-1]), src, dst)
    with prdf.Graph.batched([g.n for g in gs], src, dst) as B:
        B.set_ranks(np.concatenate(Rs))
        for t in range(3):
            bs = [s.next(1e-2) for s in streams]
            off = lambda a, i: (a.astype(np.uint64) + firsts[i]).astype(np.uint32)
            ds = np.concatenate([off(b.del_src, i) for i, b in enumerate(bs)])
            dd = np.concatenate([off(b.del_dst, i) for i, b in enumerate(bs)])
            is_ = np.concatenate([off(b.ins_src, i) for i, b in enumerate(bs)])
            id_ = np.concatenate([off(b.ins_dst, i) for i, b in enumerate(bs)])
            B.set_ranks(np.concatenate(Rs))
            B.apply(ds, dd, is_, id_)
            U, _, _ = U.apply(ds, dd, is_, id_)
            for d in (0, 1):
                off_b, col_b = B.csr(d)
                off_u, col_u = U.csr(d)
                assert np.array_equal(off_b, off_u) and np.array_equal(col_b, col_u)
            B.frontier()
            R = B.ranks()
            cs = B.component_stats()
            for i, b in enumerate(bs):
                H, ed, ei = Gs[i].apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
                Rn, aff, so = oracle.df_sync(Gs[i], H, ed, ei, Rs[i])
                part = R[firsts[i]:firsts[i + 1]]
                assert np.max(np.abs(part - Rn)) <= TOL64, gs[i].name
                assert abs(cs[i].iterations - so.iterations) <= 1
                assert abs(cs[i].affected_final - so.affected_final) <= max(2, 0.01 * so.affected_final)
                Gs[i], Rs[i] = H, Rn


def test_batched_df_equals_standalone_bitwise(prdf):
    gs = _graphs(2)
    firsts, src, dst = _union(gs)
    bs = [synth.BatchStream(g, seed=3 + i).next(1e-2) for i, g in enumerate(gs)]
    off = lambda a, i: (a.astype(np.uint64) + firsts[i]).astype(np.uint32)
    with prdf.Graph.batched([g.n for g in gs], src, dst) as B:
        B.static()
        R0 = B.ranks().copy()
        B.set_ranks(R0)  # both sides start from the same doubles (a rank near 1 does not
        #                  survive the double round trip of its 2^-62 value bit for bit)
        B.apply(np.concatenate([off(b.del_src, i) for i, b in enumerate(bs)]),
                np.concatenate([off(b.del_dst, i) for i, b in enumerate(bs)]),
                np.concatenate([off(b.ins_src, i) for i, b in enumerate(bs)]),
                np.concatenate([off(b.ins_dst, i) for i, b in enumerate(bs)]))
        B.frontier()
        R = B.ranks()
        cs = B.component_stats()
    for i, g in enumerate(gs):
        with prdf.Graph(g.n, g.src, g.dst) as A:
            A.set_ranks(R0[firsts[i]:firsts[i + 1]])
            b = bs[i]
            A.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            sa = A.frontier()
            assert np.array_equal(A.ranks(), R[firsts[i]:firsts[i + 1]]), g.name
            assert sa.iterations == cs[i].iterations


def test_batched_rejects_cross_graph_pairs(prdf):
    gs = _graphs(3)[:3]
    firsts, src, dst = _union(gs)
    with pytest.raises(prdf.PrdfError) as e:
        prdf.Graph.batched([g.n for g in gs], np.append(src, 0), np.append(dst, firsts[1]))
    assert e.value.status == prdf.PR_ERR_INVALID_ARG
    with prdf.Graph.batched([g.n for g in gs], src, dst) as B:
        before = B.csr(0)
        with pytest.raises(prdf.PrdfError) as e:
            B.apply([], [], [0], [int(firsts[2])])
        assert e.value.status == prdf.PR_ERR_INVALID_ARG
        after = B.csr(0)
        assert np.array_equal(before[1], after[1])


def test_batched_fp32(prdf):
    gs = _graphs(4)
    firsts, src, dst = _union(gs)
    p = _params(prdf, precision=prdf.PR_F32)
    with prdf.Graph.batched([g.n for g in gs], src, dst, p) as B:
        B.static()
        R = B.ranks()
    for i, g in enumerate(gs):
        Ro, _ = oracle.static_pr(oracle.Graph.build(g.n, g.src, g.dst))
        assert np.max(np.abs(R[firsts[i]:firsts[i + 1]] - Ro)) <= TOL32


def test_autotune_keeps_ranks_and_pending_marks(prdf):
    g = synth.rmat(13, 8, seed=5)
    G = oracle.Graph.build(g.n, g.src, g.dst)
    R0, _ = oracle.static_pr(G)
    b = synth.BatchStream(g, seed=5).next(1e-3)
    H, ed, ei = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
    Rdf, _, _ = oracle.df_sync(G, H, ed, ei, R0)
    with prdf.Graph(g.n, g.src, g.dst) as A:
        A.set_ranks(R0)
        A.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        before = A.ranks().copy()
        t = A.autotune(4)
        assert t.bin_lo in (4, 8, 16, 32) and t.blocks_per_sm >= 1 and t.ms > 0
        assert t.chunk_len in (128, 256, 512) and t.group_max in (16, 32, 64)
        assert np.array_equal(A.ranks(), before)
        cur = A.tuning()
        assert (cur.bin_lo, cur.blocks_per_sm, cur.chunk_len, cur.group_max) == \
            (t.bin_lo, t.blocks_per_sm, t.chunk_len, t.group_max)
        A.frontier()  # pending marks of the batch survive the autotuner
        assert np.max(np.abs(A.ranks() - Rdf)) <= TOL64


_TILINGS = [(1, 1, 512, 64), (4, 2, 128, 16), (32, 3, 256, 32), (8, 1, 32, 0), (16, 2, 64, 8)]


@pytest.mark.parametrize("lo,bps,chunk,gmax", _TILINGS)
@pytest.mark.parametrize("dead_end", ["selfloop", "teleport"])
def test_results_do_not_depend_on_tuning(prdf, lo, bps, chunk, gmax, dead_end):
    # fixed-point sums are exact in any order: any work distribution and sweep tiling gives
    # bit-identical ranks, in per-iteration launches (self-loop) and in the persistent launch
    # (teleport).  rmat(14, 16) has rows of several chunks at every chunk length
    p = _params(prdf, dead_end=prdf.PR_DEADEND_TELEPORT if dead_end == "teleport" else prdf.PR_DEADEND_SELFLOOP)
    g = synth.rmat(14, 16, seed=9)
    assert np.bincount(g.dst, minlength=g.n).max() > 4 * 512
    bs = [synth.BatchStream(g, seed=9).next(f) for f in (1e-4, 1e-3)]
    out = []
    for tune in (None, (lo, max(lo, 64), 4, bps)):
        with prdf.Graph(g.n, g.src, g.dst, p) as A:
            if tune:
                A.set_tuning(*tune, chunk_len=chunk, group_max=gmax)
                t = A.tuning()
                assert (t.bin_lo, t.chunk_len, t.group_max) == (lo, chunk, gmax)
            res = [A.static().iterations, A.ranks().copy()]
            for b in bs:
                A.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
                res += [A.frontier().affected_final, A.ranks().copy(), A.naive().iterations, A.ranks().copy()]
            out.append(res)
    for x, y in zip(out[0], out[1]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("chunk,gmax", [(128, 16), (32, 0)])
def test_fp32_tiling_changes_only_rounding(prdf, chunk, gmax):
    # FP32 sums follow the tiling's order: a different tiling moves ranks by rounding only
    g = synth.rmat(14, 16, seed=10)
    b = synth.BatchStream(g, seed=10).next(1e-3)
    out = []
    for tune in (False, True):
        with prdf.Graph(g.n, g.src, g.dst, _params(prdf, precision=prdf.PR_F32)) as A:
            if tune:
                t = A.tuning()
                A.set_tuning(t.bin_lo, t.bin_hi, t.dense_div, t.blocks_per_sm, chunk_len=chunk, group_max=gmax)
            A.static()
            A.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            st = A.frontier()
            assert st.converged
            out.append((A.ranks().copy(), st.iterations))
    assert np.max(np.abs(out[0][0] - out[1][0])) <= 1e-6
    # near the fixed point the FP32 L-inf change is a few float ulps of the largest ranks,
    # about tau, so the iteration at which it first falls to tau follows the rounding: the
    # counts agree to within a tenth (measured: 70 against 74 on this graph)
    assert abs(out[0][1] - out[1][1]) <= max(2, out[0][1] // 10)


def test_tiling_is_validated_and_a_refused_tile_keeps_the_old_one(prdf):
    g = synth.rmat(10, 8, seed=11)
    with prdf.Graph(g.n, g.src, g.dst) as A:
        t = A.tuning()
        assert (t.chunk_len, t.group_max) == (512, 64)
        for chunk, gmax in [(0, 64), (48, 64), (1024, 64), (512, -1), (512, 65)]:
            with pytest.raises(prdf.PrdfError) as e:
                A.set_tuning(t.bin_lo, t.bin_hi, t.dense_div, t.blocks_per_sm, chunk_len=chunk, group_max=gmax)
            assert e.value.status == prdf.PR_ERR_INVALID_ARG
        t2 = A.tuning()
        assert (t2.chunk_len, t2.group_max) == (512, 64)
        A.static()


@pytest.mark.parametrize("mode", ["frontier", "traversal"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_split_frontier_call_equals_single_launch(prdf, prec, mode):
    # a Dynamic Frontier call whose dense iterations run in per-iteration launches (growing
    # the set by pulls or pushes) gives exactly the single-launch result: the same sets and
    # the same sums in the same order.  Dynamic Traversal continues there after its search
    g = synth.rmat(14, 16, seed=21)
    bs = [b for b in (synth.BatchStream(g, seed=22).next(f) for f in (1e-5, 1e-4, 1e-3))]
    p = _params(prdf, precision=prdf.PR_F32 if prec == "f32" else prdf.PR_F64)
    out, kinds = [], []
    for split in (0, 1):
        with prdf.Graph(g.n, g.src, g.dst, p) as A:
            t = A.tuning()
            A.set_tuning(t.bin_lo, t.bin_hi, t.dense_div, t.blocks_per_sm, split)
            A.static()
            res = []
            for b in bs:
                A.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
                st = getattr(A, mode)()
                res.append((A.ranks().copy(), st.iterations, st.affected_final, sorted(A.affected().tolist())))
                kinds.append((split, list(A.trace()["kind"])))
            out.append(res)
    for (r0, i0, a0, s0), (r1, i1, a1, s1) in zip(out[0], out[1]):
        assert np.array_equal(r0, r1) and i0 == i1 and a0 == a1 and s0 == s1
    # split calls ran their dense iterations in the per-iteration launches (trace kinds >= 5)
    assert any(max(k) >= 5 for sp, k in kinds if sp == 1)
    assert not any(max(k) >= 5 for sp, k in kinds if sp == 0)


@pytest.mark.parametrize("split", [0, 1])
def test_late_expansions_are_pushed_by_the_dense_loop(prdf, split):
    # a hub makes a 12-vertex chain affected from the start, the batch changes the flow
    # into the chain's far end, and the change reaches vertex 1 only after 11 iterations;
    # its expansion then marks a new vertex (its leaf, 50).  Until then the affected set is
    # settled: with split calls the per-iteration loop records each late first expansion and
    # pushes its out-row (marking nothing while the chain neighbours are affected) until
    # vertex 1's marks the leaf.  Starting from fully converged ranks, so that nothing else
    # crosses tau_f.  Ranks, iterations and affected set must match the single launch and
    # the oracle.
    n = 64
    pairs = [(0, v) for v in range(1, 13)] + [(v, v - 1) for v in range(2, 13)] + [(1, 50), (41, 0), (42, 41)]
    g = synth.from_pairs(n, pairs, "hub-chain-leaf")
    G = oracle.Graph.build(g.n, g.src, g.dst)
    R0 = oracle.reference_static(G)
    R0 = R0[0] if isinstance(R0, tuple) else R0
    H, ed, ei = G.apply([0], [12], [0], [40])
    Rn, aff, so = oracle.df_sync(G, H, ed, ei, R0)
    assert aff[50]  # the late expansion happened in the oracle too
    with prdf.Graph(g.n, g.src, g.dst) as A:
        t = A.tuning()
        A.set_tuning(t.bin_lo, t.bin_hi, t.dense_div, t.blocks_per_sm, split)
        A.set_ranks(R0)
        A.apply([0], [12], [0], [40])
        l0 = prdf.pr_kernel_launches()
        st = A.frontier()
        launches = prdf.pr_kernel_launches() - l0
        kinds = "".join(str(int(k)) for k in A.trace()["kind"])
        assert np.max(np.abs(A.ranks() - Rn)) <= TOL64
        assert abs(st.iterations - so.iterations) <= 1
        assert st.affected_final == so.affected_final
        assert sorted(A.affected().tolist()) == np.nonzero(aff)[0].tolist()
    if split:
        # the per-iteration loop ran (trace kinds >= 5): more launches than the marking one
        assert max(int(k) for k in kinds) >= 5 and launches > 3, (kinds, launches)
    else:
        assert launches == 1 and max(int(k) for k in kinds) < 5, (kinds, launches)
