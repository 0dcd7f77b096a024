"""Parity at the full size of the headline workload: R-MAT scale 22, edge factor 16 (the
benchmark's graph), batches of the benchmark's stream, in the launch configuration the
benchmark times (default grid, bins and split calls).

Element by element against the oracle: Static PageRank from 1/n, then Dynamic Frontier
updates at f = 1e-7 and 1e-3 |E| chained from the oracle's own ranks, in 64-bit mode
(L-inf <= 1e-9) and FP32 (<= 1e-6), affected sets within 1% of the oracle's.  The oracle
runs in a spawned process on all host cores (its -fopenmp build, which equals the
sequential build bit for bit), about a minute in all.

Besides, on every vertex, what holds at any size:

* the CSR after an update equals the set semantics of Section 3.2 (bit for bit, built on
  the host with numpy);
* a synchronous sweep stopped by the L-inf test (Eq. 1, tau) leaves each updated vertex
  within alpha * sum_{u in in(v)} tau / |out(u)| of one more sweep of its own output, a
  bound that follows from |R_k - R_{k-1}| <= tau;
* Dynamic Frontier leaves every vertex it did not mark bit-identical, and marks at least
  the out-neighbours (in G^t) of every changed edge's source and every deleted target;
* Dynamic Traversal marks exactly the vertices reachable from a changed edge's source in
  G^{t-1} or G^t (breadth-first search on the host with scipy).
"""
import multiprocessing as mp

import numpy as np
import pytest

import __graft_entry__
import oracle
import synth

pytestmark = pytest.mark.gpu

ALPHA = 0.85
TAU = 1e-10


@pytest.fixture(scope="module")
def prdf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    from paper_2401_03256_gb300 import prdf as mod

    mod.load()
    return mod


# Edge sets are sorted unique uint64 keys (source << 32 | target); a batch is small, so
# updates are merges by binary search (O(m) copies, no sort of the whole set).
def _keys(s, d):
    k = (np.asarray(s, np.uint64) << np.uint64(32)) | np.asarray(d, np.uint64)
    return np.unique(k[(k >> np.uint64(32)) != (k & np.uint64(0xFFFFFFFF))])  # self pairs are no-ops


def _member(keys, q):
    pos = np.searchsorted(keys, q)
    return (pos < keys.shape[0]) & (keys[np.minimum(pos, keys.shape[0] - 1)] == q)


def _merge(keys, q):
    """keys union q, for sorted q disjoint from keys."""
    return np.insert(keys, np.searchsorted(keys, q), q)


@pytest.fixture(scope="module")
def big():
    g = synth.rmat(22, 16, seed=1)  # the benchmark's graph (replica 0)
    loops = np.arange(g.n, dtype=np.uint64)
    keys = _merge(g.keys(), (loops << np.uint64(32)) | loops)  # self-loops on every vertex
    return g, keys


def _changes(keys, b):
    """Effective deletions and insertions of batch b against E^{t-1} (Section 3.2):
    Delta^- = E^{t-1} minus E^t, Delta^+ = E^t minus E^{t-1}."""
    dk, ik = _keys(b.del_src, b.del_dst), _keys(b.ins_src, b.ins_dst)
    eff_del = dk[_member(keys, dk) & ~np.isin(dk, ik)]
    eff_ins = ik[~_member(keys, ik)]
    return eff_del, eff_ins


def _apply_keys(keys, b):
    """E^t = (E^{t-1} minus D) union I."""
    eff_del, eff_ins = _changes(keys, b)
    kept = np.delete(keys, np.searchsorted(keys, eff_del))
    return _merge(kept, eff_ins)


def _csr(n, keys, direction):
    src = (keys >> np.uint64(32)).astype(np.int64)
    dst = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    if direction == 1:
        rk = np.sort((dst.astype(np.uint64) << np.uint64(32)) | src.astype(np.uint64))
        src, dst = (rk >> np.uint64(32)).astype(np.int64), (rk & np.uint64(0xFFFFFFFF)).astype(np.int64)
    off = np.zeros(n + 1, np.uint64)
    off[1:] = np.cumsum(np.bincount(src, minlength=n)).astype(np.uint64)
    return off, dst.astype(np.uint32)


def _sweep_residual_ok(n, keys, R, which):
    """|R - T(R)| <= alpha * sum_{u in in(v)} tau / |out(u)| (+ rounding) on `which`."""
    src = (keys >> np.uint64(32)).astype(np.int64)
    dst = (keys & np.uint64(0xFFFFFFFF)).astype(np.int64)
    deg = np.bincount(src, minlength=n).astype(np.float64)
    T = (1.0 - ALPHA) / n + ALPHA * np.bincount(dst, weights=R[src] / deg[src], minlength=n)
    bound = ALPHA * TAU * np.bincount(dst, weights=1.0 / deg[src], minlength=n) + 1e-15
    bad = np.abs(R - T)[which] > bound[which]
    return int(bad.sum())


def test_fullsize_csr_after_updates(prdf, big):
    g, keys = big
    s = synth.BatchStream(g, seed=1)
    with prdf.Graph(g.n, g.src, g.dst) as dg:
        for f in (1e-5, 1e-3):
            b = s.next(f)
            dg.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            keys = _apply_keys(keys, b)
        n, m = dg.info()
        assert m == keys.shape[0]
        for d in (0, 1):
            off, col = dg.csr(d)
            eoff, ecol = _csr(g.n, keys, d)
            assert np.array_equal(off, eoff), f"offsets differ (dir {d})"
            assert np.array_equal(col, ecol), f"columns differ (dir {d})"


def test_fullsize_static_and_naive_residual(prdf, big):
    g, keys = big
    with prdf.Graph(g.n, g.src, g.dst) as dg:
        st = dg.static()
        R = dg.ranks()
        assert st.converged and abs(R.sum() - 1.0) <= 1e-9
        assert _sweep_residual_ok(g.n, keys, R, np.ones(g.n, bool)) == 0
        b = synth.BatchStream(g, seed=1).next(1e-4)
        dg.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        keys_t = _apply_keys(keys, b)
        st = dg.naive()
        R = dg.ranks()
        assert st.converged and abs(R.sum() - 1.0) <= 1e-9
        assert _sweep_residual_ok(g.n, keys_t, R, np.ones(g.n, bool)) == 0


@pytest.mark.parametrize("frac", [1e-7, 1e-5, 1e-3])
def test_fullsize_dynamic_frontier(prdf, big, frac):
    g, keys = big
    s = synth.BatchStream(g, seed=1)
    with prdf.Graph(g.n, g.src, g.dst) as dg:
        dg.static()
        R0 = dg.ranks().copy()
        b = s.next(frac)
        dg.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        keys_t = _apply_keys(keys, b)
        st = dg.frontier()
        R = dg.ranks()
        aff = np.zeros(g.n, bool)
        aff[dg.affected()] = True
        assert st.converged and st.affected_final == int(aff.sum())
        # unmarked vertices keep their ranks bit for bit
        assert np.array_equal(R[~aff], R0[~aff])
        # the initial marking is contained in the affected set
        dk, ik = _changes(keys, b)
        srcs = np.unique(np.concatenate([dk >> np.uint64(32), ik >> np.uint64(32)]).astype(np.int64))
        off, col = _csr(g.n, keys_t, 0)
        first = [col[int(off[u]):int(off[u + 1])] for u in srcs]
        first.append((dk & np.uint64(0xFFFFFFFF)).astype(np.uint32))
        first = np.unique(np.concatenate(first).astype(np.int64))
        assert aff[first].all()
        # every vertex the sweeps updated satisfies the synchronous stopping bound of the
        # last sweep (vertices marked in the last iteration were never swept)
        assert _sweep_residual_ok(g.n, keys_t, R, aff & (R != R0)) == 0


def test_fullsize_dynamic_traversal_is_reachability(prdf, big):
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    g, keys = big
    b = synth.BatchStream(g, seed=1).next(1e-6)
    keys_t = _apply_keys(keys, b)
    with prdf.Graph(g.n, g.src, g.dst) as dg:
        dg.static()
        dg.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        st = dg.traversal()
        got = np.sort(dg.affected().astype(np.int64))
        assert st.converged
    dk, ik = _changes(keys, b)
    srcs = np.unique(np.concatenate([dk >> np.uint64(32), ik >> np.uint64(32)]).astype(np.int64))
    # reachable from some source in the union of both graphs (every edge in only one of
    # them starts at a source, so this is the union of the per-graph reachable sets),
    # through a virtual vertex n joined to every source
    union = _merge(keys_t, dk)
    src = np.concatenate([(union >> np.uint64(32)).astype(np.int64), np.full(srcs.shape[0], g.n)])
    dst = np.concatenate([(union & np.uint64(0xFFFFFFFF)).astype(np.int64), srcs])
    A = sp.csr_matrix((np.ones(src.shape[0], np.int8), (src, dst)), shape=(g.n + 1, g.n + 1))
    reach = csgraph.breadth_first_order(A, g.n, directed=True, return_predecessors=False)
    want = np.sort(reach[reach != g.n].astype(np.int64))
    assert np.array_equal(got, want)


def test_fullsize_fp32_and_async_against_64bit(prdf, big):
    g, _ = big
    b = synth.BatchStream(g, seed=1).next(1e-4)
    p32 = prdf.pr_params_default()
    p32.precision = prdf.PR_F32
    with prdf.Graph(g.n, g.src, g.dst) as A, prdf.Graph(g.n, g.src, g.dst, p32) as F, \
            prdf.Graph(g.n, g.src, g.dst) as S:
        A.static()
        R0 = A.ranks()
        F.static()
        assert np.max(np.abs(F.ranks() - R0)) <= 1e-6
        for h in (A, F, S):
            h.set_ranks(R0)
            h.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        A.frontier()
        F.frontier()
        S.frontier_async()
        R = A.ranks()
        assert np.max(np.abs(F.ranks() - R)) <= 1e-6
        assert np.max(np.abs(S.ranks() - R)) <= 2e-9


FULL_FRACS = (1e-7, 1e-3)


def _oracle_chain(q):
    """Oracle results for the full-size parity test (in a spawned process): Static ranks,
    then each batch of FULL_FRACS from the benchmark's stream, chained."""
    oracle.use_threads(oracle.host_cores())
    g = synth.rmat(22, 16, seed=1)
    G = oracle.Graph.build(g.n, g.src, g.dst)
    R, st = oracle.static_pr(G)
    out = {"static": (R.copy(), st.iterations), "threads": oracle.threads()}
    s = synth.BatchStream(g, seed=1)
    for f in FULL_FRACS:
        b = s.next(f)
        H, ed, ei = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        Rn, aff, st = oracle.df_sync(G, H, ed, ei, R)
        out[f] = (R.copy(), Rn.copy(), np.flatnonzero(aff).astype(np.uint32), st.iterations)
        G.close()
        G, R = H, Rn
    q.put(out)


@pytest.fixture(scope="module")
def oracle_full():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_oracle_chain, args=(q,))
    p.start()
    try:
        res = q.get(timeout=1800)
    finally:
        p.join(timeout=60)
    return res


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_fullsize_against_oracle(prdf, big, oracle_full, prec):
    g, _ = big
    tol = 1e-6 if prec == "f32" else 1e-9
    p = prdf.pr_params_default()
    if prec == "f32":
        p.precision = prdf.PR_F32
    s = synth.BatchStream(g, seed=1)
    with prdf.Graph(g.n, g.src, g.dst, p) as dg:
        st = dg.static()
        R_or, it_or = oracle_full["static"]
        assert st.converged
        assert np.max(np.abs(dg.ranks() - R_or)) <= tol
        for f in FULL_FRACS:
            b = s.next(f)
            R_prev, R_df, aff_or, it_df = oracle_full[f]
            dg.set_ranks(R_prev)
            dg.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            st = dg.frontier()
            R = dg.ranks()
            err = float(np.max(np.abs(R - R_df)))
            assert st.converged and err <= tol, (f, err)
            assert abs(st.iterations - it_df) <= 1, (f, st.iterations, it_df)
            got = np.sort(dg.affected().astype(np.int64))
            diff = np.setxor1d(got, aff_or.astype(np.int64)).shape[0]
            assert diff <= max(2, 0.01 * aff_or.shape[0]), (f, diff, aff_or.shape[0])


KMER_N = 20_000_000
KMER_FRACS = (1e-6, 1e-4)


def _oracle_kmer(q):
    """Oracle chain on the k-mer stand-in with 2e7 vertices (ranks near 5e-8, where the
    64-bit fixed point keeps about 37 significant bits)."""
    oracle.use_threads(oracle.host_cores())
    g = synth.kmer(KMER_N, seed=7)
    G = oracle.Graph.build(g.n, g.src, g.dst)
    R, st = oracle.static_pr(G)
    out = {"static": (R.copy(), st.iterations)}
    s = synth.BatchStream(g, seed=7)
    for f in KMER_FRACS:
        b = s.next(f)
        H, ed, ei = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        Rn, aff, st = oracle.df_sync(G, H, ed, ei, R)
        out[f] = (R.copy(), Rn.copy(), np.flatnonzero(aff).astype(np.uint32), st.iterations)
        G.close()
        G, R = H, Rn
    q.put(out)


def test_small_rank_magnitude_against_oracle(prdf):
    """64-bit mode where ranks are near 5e-8: absolute L-inf <= 1e-9 and a relative error
    per vertex <= 1e-6 against the oracle, for Static and two chained Dynamic Frontier
    updates; affected sets within 1%."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_oracle_kmer, args=(q,))
    p.start()
    try:
        res = q.get(timeout=1800)
    finally:
        p.join(timeout=60)
    g = synth.kmer(KMER_N, seed=7)
    s = synth.BatchStream(g, seed=7)
    with prdf.Graph(g.n, g.src, g.dst) as dg:
        st = dg.static()
        R_or, _ = res["static"]
        R = dg.ranks()
        assert st.converged and R_or.max() < 1e-6  # the small-rank regime
        assert np.max(np.abs(R - R_or)) <= 1e-9
        assert np.max(np.abs(R - R_or) / R_or) <= 1e-6
        for f in KMER_FRACS:
            b = s.next(f)
            R_prev, R_df, aff_or, it_df = res[f]
            dg.set_ranks(R_prev)
            dg.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            st = dg.frontier()
            R = dg.ranks()
            assert st.converged and abs(st.iterations - it_df) <= 1
            assert np.max(np.abs(R - R_df)) <= 1e-9, f
            assert np.max(np.abs(R - R_df) / R_df) <= 1e-6, f
            got = np.sort(dg.affected().astype(np.int64))
            diff = np.setxor1d(got, aff_or.astype(np.int64)).shape[0]
            assert diff <= max(2, 0.01 * aff_or.shape[0]), (f, diff, aff_or.shape[0])
