"""Parity of the CUDA library (through the C ABI) with the FP64 oracle.

Bar (spec reading): CSR bit-exact; FP64 ranks within L-inf 1e-9 of the oracle;
FP32 ranks within 1e-6 of the FP64 oracle.  Iteration counts may differ by one where a
last L-inf value lands within rounding of tau; affected-set sizes within 1% (a rank
change within rounding of tau_f can flip one marking decision).
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


def _oracle_params(**kw):
    return oracle.Params(**kw)


def _assert_csr_equal(dg, G):
    n, m = dg.info()
    assert m == G.m
    for d in (0, 1):
        off, col = dg.csr(d)
        eoff, ecol = G.csr(d)
        assert np.array_equal(off, eoff), f"offsets differ (dir {d})"
        assert np.array_equal(col, ecol), f"columns differ (dir {d})"


def _random_pairs(rng, n, k):
    src = rng.integers(0, n, k, dtype=np.uint32)
    dst = rng.integers(0, n, k, dtype=np.uint32)
    dup = rng.integers(0, k, k // 4) if k else np.zeros(0, int)
    return np.concatenate([src, src[dup]]), np.concatenate([dst, dst[dup]])


# ------------------------------------------------------------------ graph store ----

@pytest.mark.parametrize("teleport", [False, True])
@pytest.mark.parametrize("seed,n,k", [(0, 1, 0), (1, 2, 3), (2, 17, 60), (3, 50, 400), (4, 300, 5000),
                                      (5, 1000, 20000)])
def test_build_csr_bit_exact(prdf, seed, n, k, teleport):
    rng = np.random.default_rng(seed)
    src, dst = _random_pairs(rng, n, k)
    p = _params(prdf, dead_end=prdf.PR_DEADEND_TELEPORT if teleport else prdf.PR_DEADEND_SELFLOOP)
    G = oracle.Graph.build(n, src, dst, self_loops=not teleport)
    with prdf.Graph(n, src, dst, p) as dg:
        _assert_csr_equal(dg, G)


def test_build_rmat_and_grid_bit_exact(prdf):
    for g in (synth.rmat(14, 8, seed=1), synth.grid(40, 37, seed=2)):
        G = oracle.Graph.build(g.n, g.src, g.dst)
        with prdf.Graph(g.n, g.src, g.dst) as dg:
            _assert_csr_equal(dg, G)


def test_build_from_device_arrays(prdf):
    import torch

    g = synth.rmat(12, 8, seed=4)
    s = torch.from_numpy(g.src.astype(np.int32)).cuda()
    d = torch.from_numpy(g.dst.astype(np.int32)).cuda()
    G = oracle.Graph.build(g.n, g.src, g.dst)
    with prdf.Graph(g.n, s, d) as dg:
        _assert_csr_equal(dg, G)


def test_build_rejects_bad_id(prdf):
    with pytest.raises(prdf.PrdfError) as e:
        prdf.Graph(10, np.array([1, 10], np.uint32), np.array([2, 3], np.uint32))
    assert e.value.status == prdf.PR_ERR_VERTEX_RANGE


@pytest.mark.parametrize("frac", [1e-4, 1e-3, 1e-2, 1e-1])
def test_apply_successive_batches_bit_exact(prdf, frac):
    """Config-1 graph (R-MAT scale 14, edge factor 8) under 5 successive 80/20 batches."""
    g = synth.rmat(14, 8, seed=1)
    G = oracle.Graph.build(g.n, g.src, g.dst)
    s = synth.BatchStream(g, seed=1)
    with prdf.Graph(g.n, g.src, g.dst) as dg:
        for t in range(5):
            b = s.next(frac)
            dg.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            G, _, _ = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            _assert_csr_equal(dg, G)


def test_apply_edge_cases_bit_exact(prdf):
    rng = np.random.default_rng(7)
    n = 200
    src, dst = _random_pairs(rng, n, 1500)
    G = oracle.Graph.build(n, src, dst)
    E = sorted(set(zip(src.tolist(), dst.tolist())) - {(u, u) for u in range(n)})
    with prdf.Graph(n, src, dst) as dg:
        for t in range(6):
            dels = [E[i] for i in rng.integers(0, len(E), 30)]           # present (with repeats)
            dels += [tuple(x) for x in rng.integers(0, n, (10, 2))]      # maybe absent
            ins = [tuple(x) for x in rng.integers(0, n, (40, 2))]        # maybe present
            ins += dels[:5]                                              # deleted and re-inserted
            ins += [(3, 3), (7, 7)]                                      # self pairs: no effect
            dels += [(4, 4)]
            ds = np.array([d[0] for d in dels], np.uint32)
            dd = np.array([d[1] for d in dels], np.uint32)
            is_ = np.array([i[0] for i in ins], np.uint32)
            id_ = np.array([i[1] for i in ins], np.uint32)
            dg.apply(ds, dd, is_, id_)
            G, _, _ = G.apply(ds, dd, is_, id_)
            _assert_csr_equal(dg, G)
            E = _edges(G)


def _edges(G):
    off, col = G.csr(0)
    out = []
    for u in range(len(off) - 1):
        for v in col[off[u]:off[u + 1]]:
            if v != u:
                out.append((u, int(v)))
    return out


def test_apply_rejects_bad_id_and_leaves_graph(prdf):
    g = synth.rmat(10, 8, seed=2)
    G = oracle.Graph.build(g.n, g.src, g.dst)
    with prdf.Graph(g.n, g.src, g.dst) as dg:
        with pytest.raises(prdf.PrdfError) as e:
            dg.apply([1], [2], [3, g.n], [4, 5])
        assert e.value.status == prdf.PR_ERR_VERTEX_RANGE
        _assert_csr_equal(dg, G)


def test_apply_device_arrays_and_bad_device_id(prdf):
    import torch

    g = synth.rmat(12, 8, seed=5)
    G = oracle.Graph.build(g.n, g.src, g.dst)
    s = synth.BatchStream(g, seed=5)
    b = s.next(1e-2)
    t = lambda a: torch.from_numpy(a.astype(np.int32)).cuda()
    with prdf.Graph(g.n, g.src, g.dst) as dg:
        dg.apply(t(b.del_src), t(b.del_dst), t(b.ins_src), t(b.ins_dst))
        G, _, _ = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        _assert_csr_equal(dg, G)
        bad = t(np.array([g.n + 3], np.uint32))
        with pytest.raises(prdf.PrdfError) as e:
            dg.apply(None, None, bad, t(np.array([1], np.uint32)))
        assert e.value.status == prdf.PR_ERR_VERTEX_RANGE
        _assert_csr_equal(dg, G)


def test_apply_many_moves_and_repack(prdf):
    """Heavy insertion into few rows forces row moves, tail growth and repacks."""
    n = 3000
    rng = np.random.default_rng(11)
    src, dst = _random_pairs(rng, n, 6000)
    G = oracle.Graph.build(n, src, dst)
    with prdf.Graph(n, src, dst) as dg:
        for t in range(6):
            hubs = rng.integers(0, n, 3)
            is_ = np.repeat(hubs, 2000).astype(np.uint32)
            id_ = rng.integers(0, n, is_.size).astype(np.uint32)
            # and the transposed direction: many sources into few targets
            is2 = rng.integers(0, n, 3000).astype(np.uint32)
            id2 = np.repeat(rng.integers(0, n, 3), 1000).astype(np.uint32)
            e = _edges(G)
            pick = rng.integers(0, len(e), 500)
            ds = np.array([e[i][0] for i in pick], np.uint32)
            dd = np.array([e[i][1] for i in pick], np.uint32)
            ins_s = np.concatenate([is_, is2])
            ins_d = np.concatenate([id_, id2])
            dg.apply(ds, dd, ins_s, ins_d)
            G, _, _ = G.apply(ds, dd, ins_s, ins_d)
            _assert_csr_equal(dg, G)


# ---------------------------------------------------------------------- ranks ----

def test_static_cycle_and_star(prdf):
    n = 33
    with prdf.Graph(n, np.arange(n, dtype=np.uint32), (np.arange(n, dtype=np.uint32) + 1) % n) as dg:
        st = dg.static()
        assert st.iterations == 1 and st.converged
        assert np.max(np.abs(dg.ranks() - 1.0 / n)) <= 4 * np.spacing(1.0 / n)
    k = 40
    with prdf.Graph(k + 1, np.arange(1, k + 1, dtype=np.uint32), np.zeros(k, np.uint32)) as dg:
        dg.static()
        G = oracle.Graph.build(k + 1, np.arange(1, k + 1), np.zeros(k))
        R, _ = oracle.static_pr(G)
        assert np.max(np.abs(dg.ranks() - R)) <= TOL64


@pytest.mark.parametrize("scale,ef", [(10, 8), (14, 8), (16, 4)])
def test_static_and_naive_parity(prdf, scale, ef):
    g = synth.rmat(scale, ef, seed=scale)
    G = oracle.Graph.build(g.n, g.src, g.dst)
    R_or, st_or = oracle.static_pr(G)
    with prdf.Graph(g.n, g.src, g.dst) as dg:
        st = dg.static()
        assert st.converged and abs(st.iterations - st_or.iterations) <= 1
        R = dg.ranks()
        assert np.max(np.abs(R - R_or)) <= TOL64
        assert abs(R.sum() - 1.0) <= 1e-9
        assert st.vertices_processed == g.n * st.iterations
        b = synth.BatchStream(g, seed=scale).next(1e-3)
        dg.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        H, _, _ = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        dg.set_ranks(R_or)
        stn = dg.naive()
        Rn_or, stn_or = oracle.naive_pr(H, R_or)
        assert abs(stn.iterations - stn_or.iterations) <= 1
        assert np.max(np.abs(dg.ranks() - Rn_or)) <= TOL64


def _df_case(prdf, g, frac, batches, seed, params=None, oparams=None, check_affected=True):
    G = oracle.Graph.build(g.n, g.src, g.dst, self_loops=(oparams is None or oparams.dead_end == 0))
    R_or, _ = oracle.static_pr(G, oparams)
    s = synth.BatchStream(g, seed=seed)
    out = []
    with prdf.Graph(g.n, g.src, g.dst, params) as dg:
        for t in range(batches):
            b = s.next(frac)
            dg.set_ranks(R_or)                 # both sides start from the same R^{t-1} on G^{t-1}
            dg.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            H, ed, ei = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            st = dg.frontier()
            R_df, aff, st_or = oracle.df_sync(G, H, ed, ei, R_or, oparams)
            R = dg.ranks()
            err = float(np.max(np.abs(R - R_df)))
            out.append((st, st_or, err))
            assert st.converged == st_or.converged
            assert abs(st.iterations - st_or.iterations) <= 1, (st.iterations, st_or.iterations)
            if check_affected:
                assert abs(st.affected_final - st_or.affected_final) <= max(2, 0.01 * st_or.affected_final)
                got = set(dg.affected().tolist())
                assert len(got) == st.affected_final
                want = set(np.nonzero(aff)[0].tolist())
                assert len(got ^ want) <= max(2, 0.01 * len(want))
            G, R_or = H, R_df
            out[-1] = out[-1] + (R, R_df)
    return out


@pytest.mark.parametrize("frac", [1e-4, 1e-3, 1e-2])
def test_df_parity_config1(prdf, frac):
    """R-MAT scale 14, edge factor 8, 5 successive 80/20 batches, FP64 (config 1 shape)."""
    g = synth.rmat(14, 8, seed=1)
    for st, st_or, err, R, R_df in _df_case(prdf, g, frac, 5, 1):
        assert err <= TOL64, err


def test_df_parity_forced_bins(prdf):
    """Tiny thresholds push most vertices into the warp and block bins."""
    g = synth.rmat(13, 16, seed=9)
    p = _params(prdf, bin_lo=1, bin_hi=24)
    for st, st_or, err, R, R_df in _df_case(prdf, g, 1e-3, 3, 9, params=p):
        assert err <= TOL64, err


def test_df_chained_matches_chained_oracle(prdf):
    """Each side chains its own outputs over 5 batches from its own Static start."""
    g = synth.rmat(14, 8, seed=1)
    G = oracle.Graph.build(g.n, g.src, g.dst)
    R_or, _ = oracle.static_pr(G)
    s = synth.BatchStream(g, seed=1)
    with prdf.Graph(g.n, g.src, g.dst) as dg:
        dg.static()
        for t in range(5):
            b = s.next(1e-4)
            dg.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            H, ed, ei = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            dg.frontier()
            R_or, _, _ = oracle.df_sync(G, H, ed, ei, R_or)
            G = H
        assert np.max(np.abs(dg.ranks() - R_or)) <= TOL64


def test_df_empty_batch_and_no_effect_batch(prdf):
    g = synth.rmat(12, 8, seed=3)
    with prdf.Graph(g.n, g.src, g.dst) as dg:
        dg.static()
        R0 = dg.ranks().copy()
        st = dg.frontier()
        assert st.iterations == 1 and st.converged and st.affected_final == 0
        assert np.array_equal(dg.ranks(), R0)
        # a batch whose every pair is a no-op: self pairs and an absent deletion
        dg.apply([5], [5], [7, 9], [7, 9])
        st = dg.frontier()
        assert st.iterations == 1 and st.affected_final == 0
        assert np.array_equal(dg.ranks(), R0)


def test_df_max_iter_zero_marks_only(prdf):
    g = synth.rmat(10, 8, seed=2)
    G = oracle.Graph.build(g.n, g.src, g.dst)
    R_or, _ = oracle.static_pr(G)
    p = _params(prdf, max_iter=0)
    b = synth.BatchStream(g, seed=2).next(1e-2)
    H, ed, ei = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
    _, aff, _ = oracle.df_sync(G, H, ed, ei, R_or, oracle.Params(max_iter=0))
    with prdf.Graph(g.n, g.src, g.dst, p) as dg:
        dg.set_ranks(R_or)
        before = dg.ranks().copy()
        assert np.max(np.abs(before - R_or)) <= 1e-18
        dg.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        st = dg.frontier()
        assert st.iterations == 0
        assert sorted(dg.affected().tolist()) == sorted(np.nonzero(aff)[0].tolist())
        assert np.array_equal(dg.ranks(), before)


def test_df_deterministic(prdf):
    g = synth.rmat(14, 8, seed=6)
    b = synth.BatchStream(g, seed=6).next(1e-3)
    res = []
    for _ in range(2):
        with prdf.Graph(g.n, g.src, g.dst) as dg:
            dg.static()
            dg.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            dg.frontier()
            res.append(dg.ranks().copy())
    assert np.array_equal(res[0], res[1])


def test_paper_example_initial_marks(prdf):
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "fig1_example.json")) as f:
        ex = json.load(f)
    edges = np.array(ex["stated_edges"] + ex["filler_edges"], np.uint32)
    for teleport, key in ((True, "initial_affected_no_self_loops"), (False, "initial_affected_with_self_loops")):
        p = _params(prdf, max_iter=0,
                    dead_end=prdf.PR_DEADEND_TELEPORT if teleport else prdf.PR_DEADEND_SELFLOOP)
        with prdf.Graph(ex["n"], edges[:, 0].copy(), edges[:, 1].copy(), p) as dg:
            dg.apply([2], [1], [4], [12])
            dg.frontier()
            assert sorted(dg.affected().tolist()) == ex[key]


def test_tiny_graphs(prdf):
    with prdf.Graph(1, np.zeros(0, np.uint32), np.zeros(0, np.uint32)) as dg:
        st = dg.static()
        assert dg.ranks().tolist() == [1.0] and st.converged
        dg.apply([], [], [0], [0])
        st = dg.frontier()
        assert st.affected_final == 0
    with prdf.Graph(5, np.zeros(0, np.uint32), np.zeros(0, np.uint32)) as dg:
        dg.static()
        assert np.allclose(dg.ranks(), 0.2, atol=1e-16)


# ------------------------------------------------------------------ teleport ----

def test_teleport_static_naive_df(prdf):
    g = synth.rmat(10, 4, seed=8)  # many vertices without out-edges
    p = _params(prdf, dead_end=prdf.PR_DEADEND_TELEPORT)
    op = oracle.Params(dead_end=oracle.TELEPORT)
    G = oracle.Graph.build(g.n, g.src, g.dst, self_loops=False)
    R_or, st_or = oracle.static_pr(G, op)
    with prdf.Graph(g.n, g.src, g.dst, p) as dg:
        st = dg.static()
        assert np.max(np.abs(dg.ranks() - R_or)) <= TOL64
        assert abs(dg.ranks().sum() - 1.0) <= 1e-9
    exact = oracle.dense_solve(g.n, g.src, g.dst, self_loops=False) if g.n <= 1024 else None
    if exact is not None:
        assert np.max(np.abs(R_or - exact)) <= 1e-9
    for st, st_or, err, R, R_df in _df_case(prdf, g, 1e-3, 3, 8, params=p, oparams=op, check_affected=False):
        assert err <= TOL64, err


# ---------------------------------------------------------------- precision ----

def test_fp32_static_and_df_against_fp64_oracle(prdf):
    g = synth.rmat(14, 8, seed=1)
    p = _params(prdf, precision=prdf.PR_F32)
    G = oracle.Graph.build(g.n, g.src, g.dst)
    R_or, _ = oracle.static_pr(G)
    s = synth.BatchStream(g, seed=1)
    with prdf.Graph(g.n, g.src, g.dst, p) as dg:
        st = dg.static()
        assert np.max(np.abs(dg.ranks() - R_or)) <= TOL32
        for t in range(3):
            b = s.next(1e-3)
            dg.set_ranks(R_or)
            dg.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            H, ed, ei = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            dg.frontier()
            R_or, _, _ = oracle.df_sync(G, H, ed, ei, R_or)
            G = H
            assert np.max(np.abs(dg.ranks() - R_or)) <= TOL32
