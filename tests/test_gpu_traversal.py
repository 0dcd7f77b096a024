"""Dynamic Traversal (Section 3.3.2) on the GPU against the FP64 oracle's reading of it.

The affected set is pure reachability, so it must match the oracle exactly; ranks
within 1e-9 (FP64) or 1e-6 (FP32) of the oracle, iteration counts within one.
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


def _params(prdf, **kw):
    p = prdf.pr_params_default()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _dt_step(dg, G, R_or, dels, inss, oparams=None, tol=TOL64):
    """One batch on both sides from the same R^{t-1}; returns (G^t, oracle ranks)."""
    ds, dd = (np.asarray(x, np.uint32) for x in dels)
    is_, id_ = (np.asarray(x, np.uint32) for x in inss)
    dg.set_ranks(R_or)
    dg.apply(ds, dd, is_, id_)
    H, ed, ei = G.apply(ds, dd, is_, id_)
    st = dg.traversal()
    R_dt, aff, st_or = oracle.dt_sync(G, H, ed, ei, R_or, oparams)
    assert st.converged == st_or.converged
    assert abs(st.iterations - st_or.iterations) <= 1, (st.iterations, st_or.iterations)
    want = sorted(np.nonzero(aff)[0].tolist())
    got = sorted(dg.affected().tolist())
    assert got == want, (len(got), len(want))
    assert st.affected_final == len(want)
    err = float(np.max(np.abs(dg.ranks() - R_dt))) if G.n else 0.0
    assert err <= tol, err
    return H, R_dt


@pytest.mark.parametrize("frac", [1e-4, 1e-3, 1e-2])
def test_dt_rmat_batches(prdf, frac):
    """R-MAT scale 14, edge factor 8, three successive 80/20 batches."""
    g = synth.rmat(14, 8, seed=4)
    G = oracle.Graph.build(g.n, g.src, g.dst)
    R_or, _ = oracle.static_pr(G)
    s = synth.BatchStream(g, seed=4)
    with prdf.Graph(g.n, g.src, g.dst) as dg:
        for _ in range(3):
            b = s.next(frac)
            G, R_or = _dt_step(dg, G, R_or, (b.del_src, b.del_dst), (b.ins_src, b.ins_dst))


def test_dt_grid_deep_search(prdf):
    """A 2-D grid: the search runs many rounds before it closes."""
    g = synth.grid(60, 50, seed=5)
    G = oracle.Graph.build(g.n, g.src, g.dst)
    R_or, _ = oracle.static_pr(G)
    s = synth.BatchStream(g, seed=5)
    with prdf.Graph(g.n, g.src, g.dst) as dg:
        for frac in (1e-4, 1e-3):
            b = s.next(frac)
            G, R_or = _dt_step(dg, G, R_or, (b.del_src, b.del_dst), (b.ins_src, b.ins_dst))


def test_dt_deleted_subtree_is_reached_through_the_old_graph(prdf):
    """Deleting 0->1 cuts 1's subtree off from 0 in G^t; it was reachable in G^{t-1}."""
    src = [0, 1, 2, 0, 4, 6, 7]
    dst = [1, 2, 3, 4, 5, 7, 8]
    n = 9
    G = oracle.Graph.build(n, src, dst)
    R_or, _ = oracle.static_pr(G)
    with prdf.Graph(n, np.array(src, np.uint32), np.array(dst, np.uint32)) as dg:
        H, _ = _dt_step(dg, G, R_or, ([0], [1]), ([], []))
        assert sorted(dg.affected().tolist()) == [0, 1, 2, 3, 4, 5]


@pytest.mark.parametrize("n", [900, 1300])
def test_dt_chain_depth(prdf, n):
    """A path 0->1->...->n-1 changed at its head: every vertex is reached. At n = 1300 the
    search is deeper than the round limit and the kernel takes all of V as affected, which
    is the same set here."""
    src = np.arange(n - 1, dtype=np.uint32)
    dst = src + 1
    G = oracle.Graph.build(n, src, dst)
    R_or, _ = oracle.static_pr(G)
    with prdf.Graph(n, src, dst) as dg:
        _dt_step(dg, G, R_or, ([], []), ([0], [2]))
        assert dg.affected().shape[0] == n


def test_dt_empty_and_no_effect_batches(prdf):
    g = synth.rmat(12, 8, seed=3)
    with prdf.Graph(g.n, g.src, g.dst) as dg:
        dg.static()
        R0 = dg.ranks().copy()
        st = dg.traversal()
        assert st.iterations == 1 and st.converged and st.affected_final == 0
        assert np.array_equal(dg.ranks(), R0)
        dg.apply([5], [5], [7, 9], [7, 9])
        st = dg.traversal()
        assert st.affected_final == 0 and np.array_equal(dg.ranks(), R0)


def test_dt_then_df_on_the_same_graph(prdf):
    """Traversal leaves no marking state behind: a Dynamic Frontier call after it agrees
    with the oracle, and so does a Traversal call after that."""
    g = synth.rmat(13, 8, seed=11)
    G = oracle.Graph.build(g.n, g.src, g.dst)
    R_or, _ = oracle.static_pr(G)
    s = synth.BatchStream(g, seed=11)
    with prdf.Graph(g.n, g.src, g.dst) as dg:
        b = s.next(1e-3)
        G, R_or = _dt_step(dg, G, R_or, (b.del_src, b.del_dst), (b.ins_src, b.ins_dst))
        b = s.next(1e-3)
        dg.set_ranks(R_or)
        dg.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        H, ed, ei = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        dg.frontier()
        R_df, _, _ = oracle.df_sync(G, H, ed, ei, R_or)
        assert np.max(np.abs(dg.ranks() - R_df)) <= TOL64
        G, R_or = H, R_df
        b = s.next(1e-3)
        _dt_step(dg, G, R_or, (b.del_src, b.del_dst), (b.ins_src, b.ins_dst))


def test_dt_teleport(prdf):
    """Without self-loops a change moves the teleport share of every vertex: all of V."""
    g = synth.rmat(10, 4, seed=8)
    p = _params(prdf, dead_end=prdf.PR_DEADEND_TELEPORT)
    op = oracle.Params(dead_end=oracle.TELEPORT)
    G = oracle.Graph.build(g.n, g.src, g.dst, self_loops=False)
    R_or, _ = oracle.static_pr(G, op)
    s = synth.BatchStream(g, seed=8)
    with prdf.Graph(g.n, g.src, g.dst, p) as dg:
        b = s.next(1e-3)
        _dt_step(dg, G, R_or, (b.del_src, b.del_dst), (b.ins_src, b.ins_dst), oparams=op)


def test_dt_fp32(prdf):
    g = synth.rmat(14, 8, seed=1)
    p = _params(prdf, precision=prdf.PR_F32)
    G = oracle.Graph.build(g.n, g.src, g.dst)
    R_or, _ = oracle.static_pr(G)
    s = synth.BatchStream(g, seed=1)
    with prdf.Graph(g.n, g.src, g.dst, p) as dg:
        for _ in range(2):
            b = s.next(1e-3)
            dg.set_ranks(R_or)
            dg.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            H, ed, ei = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            dg.traversal()
            R_or, aff, _ = oracle.dt_sync(G, H, ed, ei, R_or)
            assert sorted(dg.affected().tolist()) == sorted(np.nonzero(aff)[0].tolist())
            assert np.max(np.abs(dg.ranks() - R_or)) <= TOL32
            G = H


@pytest.mark.parametrize("split", [0, 1])
def test_dt_beyond_the_round_limit_iterates_as_naive(prdf, split):
    """A search deeper than the round limit takes all of V, so the iterations are exactly
    Naive-dynamic's from the same ranks (bit for bit in 64-bit mode); with split calls they
    run in the same per-iteration full sweeps as Naive-dynamic."""
    n = 1300
    src = np.arange(n - 1, dtype=np.uint32)
    dst = src + 1
    G = oracle.Graph.build(n, src, dst)
    R_or, _ = oracle.static_pr(G)
    out = []
    for call in ("traversal", "naive"):
        with prdf.Graph(n, src, dst) as dg:
            t = dg.tuning()
            dg.set_tuning(t.bin_lo, t.bin_hi, t.dense_div, t.blocks_per_sm, split)
            dg.set_ranks(R_or)
            dg.apply([], [], [0], [2])
            l0 = prdf.pr_kernel_launches()
            st = getattr(dg, call)()
            out.append((dg.ranks().copy(), st.iterations, prdf.pr_kernel_launches() - l0))
            if call == "traversal":
                assert dg.affected().shape[0] == n
    (r_dt, it_dt, l_dt), (r_nv, it_nv, l_nv) = out
    assert np.array_equal(r_dt, r_nv) and it_dt == it_nv
    # Naive-dynamic: the per-iteration loop (one launch per iteration, its init and
    # writeback) after the same refresh launches; split: the marking launch that ran the
    # search, then the same loop; otherwise the search and the iterations in that one launch
    refresh = l_nv - it_nv - 2
    assert l_dt - refresh == (1 + it_nv + 2 if split else 1), (l_dt, l_nv, it_nv)
