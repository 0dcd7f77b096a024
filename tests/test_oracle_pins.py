"""Pins for the FP64 oracle: each test ties it to something other than itself.

Closed forms (directed cycle, in-star, teleport star), an independent dense solve
(numpy on a matrix built here from Python sets), brute-force set semantics for graph
build and batch update, invariants (sum of ranks, empty batch), special cases that
reduce to another routine (DF with tau_f = 0 and every vertex affected is Naive-dynamic),
the paper's worked example (Figure 1) for the initial marking, and hop-by-hop frontier
growth that separates the synchronous and asynchronous readings of Algorithm 1.
"""
import json
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _brute_graph(n, pairs, self_loops=True):
    E = {(u, v) for u, v in pairs if u != v}
    if self_loops:
        E |= {(v, v) for v in range(n)}
    return E


def _csr_from_set(n, E, direction):
    rows = [[] for _ in range(n)]
    for u, v in E:
        if direction == 0:
            rows[u].append(v)
        else:
            rows[v].append(u)
    off = [0]
    col = []
    for r in rows:
        col.extend(sorted(r))
        off.append(len(col))
    return np.array(off, np.uint64), np.array(col, np.uint32)


def test_paper_constants():
    c = _golden("paper_constants.json")
    assert oracle.ALPHA == c["alpha"]
    assert oracle.TOL == c["tol"]
    assert oracle.FRONTIER_TOL == c["tol"] / c["frontier_tol_divisor"]
    assert oracle.MAX_ITER == c["max_iter"]
    p = oracle.Params()
    assert (p.alpha, p.tol, p.frontier_tol, p.max_iter) == (0.85, 1e-10, 1e-15, 500)


@pytest.mark.parametrize("self_loops", [True, False])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_build_matches_set_semantics(seed, self_loops):
    rng = random.Random(seed)
    n = rng.randint(1, 40)
    pairs = [(rng.randrange(n), rng.randrange(n)) for _ in range(rng.randint(0, 200))]
    pairs += pairs[: len(pairs) // 3]  # duplicates
    g = oracle.Graph.build(n, [p[0] for p in pairs], [p[1] for p in pairs], self_loops)
    E = _brute_graph(n, pairs, self_loops)
    assert g.m == len(E)
    for d in (0, 1):
        off, col = g.csr(d)
        eoff, ecol = _csr_from_set(n, E, d)
        assert np.array_equal(off, eoff)
        assert np.array_equal(col, ecol)


def test_build_rejects_bad_id():
    with pytest.raises(ValueError):
        oracle.Graph.build(4, [0, 4], [1, 2])


@pytest.mark.parametrize("seed", range(6))
def test_apply_matches_set_semantics(seed):
    rng = random.Random(100 + seed)
    n = rng.randint(2, 30)
    pairs = [(rng.randrange(n), rng.randrange(n)) for _ in range(rng.randint(0, 120))]
    E0 = {(u, v) for u, v in pairs if u != v}
    g = oracle.Graph.build(n, [p[0] for p in pairs], [p[1] for p in pairs])
    existing = sorted(E0)
    dels = [rng.choice(existing) for _ in range(min(len(existing), rng.randint(0, 10)))] if existing else []
    dels += [(rng.randrange(n), rng.randrange(n)) for _ in range(rng.randint(0, 5))]  # maybe absent
    ins = [(rng.randrange(n), rng.randrange(n)) for _ in range(rng.randint(0, 15))]
    ins += dels[:2]  # deleted and re-inserted in the same batch
    ins += [(0, 0), (1, 1)]  # self pairs are ignored
    dels += ins[:2]
    h, (eds, edd), (eis, eid) = g.apply([d[0] for d in dels], [d[1] for d in dels],
                                        [i[0] for i in ins], [i[1] for i in ins])
    D = {(u, v) for u, v in dels if u != v}
    I = {(u, v) for u, v in ins if u != v}
    E1 = (E0 - D) | I
    assert set(zip(eds.tolist(), edd.tolist())) == E0 - E1
    assert set(zip(eis.tolist(), eid.tolist())) == E1 - E0
    full = E1 | {(v, v) for v in range(n)}
    for d in (0, 1):
        off, col = h.csr(d)
        eoff, ecol = _csr_from_set(n, full, d)
        assert np.array_equal(off, eoff) and np.array_equal(col, ecol)
    # the old graph is untouched
    off, col = g.csr(0)
    eoff, ecol = _csr_from_set(n, E0 | {(v, v) for v in range(n)}, 0)
    assert np.array_equal(off, eoff) and np.array_equal(col, ecol)


def test_cycle_is_uniform():
    """Directed cycle with self-loops: every out-degree is 2 and R = 1/n is the fixed point."""
    n = 17
    g = oracle.Graph.build(n, list(range(n)), [(i + 1) % n for i in range(n)])
    R, st = oracle.static_pr(g)
    assert np.max(np.abs(R - 1.0 / n)) <= 4 * np.spacing(1.0 / n)
    assert st.iterations == 1 and st.converged


def test_complete_graph_is_uniform():
    n = 9
    src = [u for u in range(n) for v in range(n) if u != v]
    dst = [v for u in range(n) for v in range(n) if u != v]
    R, st = oracle.static_pr(oracle.Graph.build(n, src, dst))
    assert np.max(np.abs(R - 1.0 / n)) <= 4 * np.spacing(1.0 / n)
    assert st.iterations == 1


def test_in_star_closed_form():
    """k leaves -> centre with self-loops: r_leaf = 2(1-a)/(n(2-a)),
    r_centre = ((1-a)/n + a k r_leaf / 2) / (1-a), and they sum to 1."""
    k = 20
    n = k + 1
    a = Fraction(85, 100)
    r_leaf = 2 * (1 - a) / (n * (2 - a))
    r_c = ((1 - a) / n + a * k * r_leaf / 2) / (1 - a)
    assert r_c + k * r_leaf == 1
    g = oracle.Graph.build(n, list(range(1, n)), [0] * k)
    R, st = oracle.reference_static(g)
    assert abs(R[0] - float(r_c)) <= 1e-14
    assert np.max(np.abs(R[1:] - float(r_leaf))) <= 1e-15


def test_teleport_star_closed_form():
    """k leaves -> centre, no self-loops: the centre is a dead end whose rank is
    spread over all n vertices.  With t = (1-a)/n:
    r_leaf = t + a r_c / n and r_c = t(1 + a k) / (1 - a/n - a^2 k / n)."""
    k = 12
    n = k + 1
    a = Fraction(85, 100)
    t = (1 - a) / n
    r_c = t * (1 + a * k) / (1 - a / n - a * a * k / n)
    r_leaf = t + a * r_c / n
    assert r_c + k * r_leaf == 1
    g = oracle.Graph.build(n, list(range(1, n)), [0] * k, self_loops=False)
    R, _ = oracle.reference_static(g, dead_end=oracle.TELEPORT)
    assert abs(R[0] - float(r_c)) <= 1e-14
    assert np.max(np.abs(R[1:] - float(r_leaf))) <= 1e-15
    Rd = oracle.dense_solve(n, list(range(1, n)), [0] * k, self_loops=False)
    assert abs(Rd[0] - float(r_c)) <= 1e-15


def _numpy_dense(n, pairs, self_loops, alpha=0.85):
    E = _brute_graph(n, pairs, self_loops)
    outd = [0] * n
    for u, _ in E:
        outd[u] += 1
    A = np.eye(n)
    for u, v in E:
        A[v, u] -= alpha / outd[u]
    for u in range(n):
        if outd[u] == 0:
            A[:, u] -= alpha / n
    return np.linalg.solve(A, np.full(n, (1 - alpha) / n))


@pytest.mark.parametrize("self_loops", [True, False])
@pytest.mark.parametrize("seed", [3, 4, 5])
def test_dense_solve_and_static_agree_with_numpy(seed, self_loops):
    rng = random.Random(seed)
    n = rng.randint(2, 48)
    pairs = [(rng.randrange(n), rng.randrange(n)) for _ in range(rng.randint(1, 4 * n))]
    src = [p[0] for p in pairs]
    dst = [p[1] for p in pairs]
    ref = _numpy_dense(n, pairs, self_loops)
    Rd = oracle.dense_solve(n, src, dst, self_loops)
    assert np.max(np.abs(Rd - ref)) <= 1e-13
    g = oracle.Graph.build(n, src, dst, self_loops)
    mode = oracle.SELF_LOOPS if self_loops else oracle.TELEPORT
    Rs, _ = oracle.reference_static(g, dead_end=mode)
    assert np.max(np.abs(Rs - ref)) <= 1e-13
    Rt, st = oracle.static_pr(g, oracle.Params(dead_end=mode))
    assert st.converged and st.last_delta <= 1e-10
    # power iteration contracts by alpha per sweep: error <= tau * alpha / (1 - alpha)
    assert np.max(np.abs(Rt - ref)) <= 1e-10 * 0.85 / 0.15 + 1e-15


@pytest.mark.parametrize("mode", [oracle.SELF_LOOPS, oracle.TELEPORT])
def test_ranks_sum_to_one(mode):
    g = synth.rmat(10, 8, seed=7)
    G = oracle.Graph.build(g.n, g.src, g.dst, self_loops=(mode == oracle.SELF_LOOPS))
    R, st = oracle.static_pr(G, oracle.Params(dead_end=mode))
    assert abs(R.sum() - 1.0) <= 1e-12
    one = oracle.naive_pr(G, np.full(g.n, 1.0 / g.n), oracle.Params(max_iter=1, dead_end=mode))[0]
    assert abs(one.sum() - 1.0) <= 1e-12


def _stream_case(scale=10, ef=8, seed=1, frac=1e-3, batches=3):
    g = synth.rmat(scale, ef, seed=seed)
    G = oracle.Graph.build(g.n, g.src, g.dst)
    s = synth.BatchStream(g, seed=seed)
    return g, G, s, frac, batches


def test_empty_batch_leaves_ranks_bit_identical():
    g, G, s, _, _ = _stream_case()
    R0, _ = oracle.static_pr(G)
    H, ed, ei = G.apply([], [], [], [])
    R, aff, st = oracle.df_sync(G, H, ed, ei, R0)
    assert np.array_equal(R, R0)
    assert st.iterations == 1 and st.converged and st.affected_final == 0 and not aff.any()
    Ra, _, sta = oracle.df_async(G, H, ed, ei, R0)
    assert np.array_equal(Ra, R0) and sta.iterations == 1
    Rt, afft, stt = oracle.dt_sync(G, H, ed, ei, R0)
    assert np.array_equal(Rt, R0) and stt.iterations == 1 and not afft.any()


def test_df_with_everything_affected_and_zero_tau_f_is_naive():
    """A batch with a source at every vertex marks all of V (self-loops); with tau_f = 0
    Algorithm 1 then performs exactly the Naive-dynamic sweeps, bit for bit."""
    g = synth.rmat(9, 8, seed=11)
    n = g.n
    G = oracle.Graph.build(n, g.src, g.dst)
    R0, _ = oracle.static_pr(G)
    E = set(zip(g.src.tolist(), g.dst.tolist()))
    ins_src, ins_dst = [], []
    for u in range(n):
        v = next(w for w in range(n) if w != u and (u, w) not in E)
        ins_src.append(u)
        ins_dst.append(v)
    H, ed, ei = G.apply([], [], ins_src, ins_dst)
    assert sorted(ei[0].tolist()) == list(range(n))
    p = oracle.Params(frontier_tol=0.0)
    Rdf, aff, st = oracle.df_sync(G, H, ed, ei, R0, p)
    Rnv, stn = oracle.naive_pr(H, R0, p)
    assert aff.all()
    assert np.array_equal(Rdf, Rnv)
    assert st.iterations == stn.iterations


@pytest.mark.parametrize("self_loops,key", [(False, "initial_affected_no_self_loops"),
                                            (True, "initial_affected_with_self_loops")])
def test_paper_example_initial_marking(self_loops, key):
    ex = _golden("fig1_example.json")
    edges = ex["stated_edges"] + ex["filler_edges"]
    assert len(edges) == 25
    G = oracle.Graph.build(ex["n"], [e[0] for e in edges], [e[1] for e in edges], self_loops)
    dels, ins = ex["deletions"], ex["insertions"]
    H, ed, ei = G.apply([d[0] for d in dels], [d[1] for d in dels], [i[0] for i in ins], [i[1] for i in ins])
    assert ed[0].tolist() == [2] and ed[1].tolist() == [1]
    assert ei[0].tolist() == [4] and ei[1].tolist() == [12]
    mode = oracle.SELF_LOOPS if self_loops else oracle.TELEPORT
    R0 = np.full(ex["n"], 1.0 / ex["n"])
    for fn in (oracle.df_sync, oracle.df_async):
        _, aff, st = fn(G, H, ed, ei, R0, oracle.Params(max_iter=0, dead_end=mode))
        assert sorted(np.nonzero(aff)[0].tolist()) == ex[key]
        assert st.iterations == 0


def test_sync_frontier_grows_one_hop_per_iteration_async_sweeps_ahead():
    """Chain 0 -> 1 -> ... -> 9 with self-loops, insert (0, 5).  Initial marks are
    G^t.out(0) = {0, 1, 5}.  Synchronously the marks made in an iteration act in the
    next, so after one iteration the set is {0, 1, 2, 5, 6}; asynchronously a vertex
    marked ahead of the ascending sweep is processed at once, reaching the chain's end."""
    n = 10
    G = oracle.Graph.build(n, list(range(n - 1)), list(range(1, n)))
    R0, _ = oracle.static_pr(G)
    H, ed, ei = G.apply([], [], [0], [5])
    _, aff0, _ = oracle.df_sync(G, H, ed, ei, R0, oracle.Params(max_iter=0))
    assert sorted(np.nonzero(aff0)[0].tolist()) == [0, 1, 5]
    _, aff1, _ = oracle.df_sync(G, H, ed, ei, R0, oracle.Params(max_iter=1))
    assert sorted(np.nonzero(aff1)[0].tolist()) == [0, 1, 2, 5, 6]
    _, aff2, _ = oracle.df_sync(G, H, ed, ei, R0, oracle.Params(max_iter=2))
    assert sorted(np.nonzero(aff2)[0].tolist()) == [0, 1, 2, 3, 5, 6, 7]
    _, aa1, _ = oracle.df_async(G, H, ed, ei, R0, oracle.Params(max_iter=1))
    assert sorted(np.nonzero(aa1)[0].tolist()) == list(range(n))


def test_frontier_tolerance_is_strict():
    """A vertex whose rank change is not above tau_f does not expand: with tau_f huge,
    nothing beyond the initial marks is ever affected."""
    n = 10
    G = oracle.Graph.build(n, list(range(n - 1)), list(range(1, n)))
    R0, _ = oracle.static_pr(G)
    H, ed, ei = G.apply([], [], [0], [5])
    _, aff, st = oracle.df_sync(G, H, ed, ei, R0, oracle.Params(frontier_tol=1.0))
    assert sorted(np.nonzero(aff)[0].tolist()) == [0, 1, 5]
    assert st.converged


@pytest.mark.parametrize("mode", [oracle.SELF_LOOPS, oracle.TELEPORT])
def test_df_converges_near_exact_solution(mode):
    """DF ranks after successive batches stay within the error of a converged power
    iteration of the exact solution (dense solve), in both dead-end modes."""
    g = synth.rmat(9, 8, seed=5)
    n = g.n
    sl = mode == oracle.SELF_LOOPS
    p = oracle.Params(dead_end=mode)
    G = oracle.Graph.build(n, g.src, g.dst, sl)
    R, _ = oracle.static_pr(G, p)
    Ra = R.copy()
    s = synth.BatchStream(g, seed=5)
    for t in range(3):
        b = s.next(1e-2)
        H, ed, ei = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        R, _, st = oracle.df_sync(G, H, ed, ei, R, p)
        Ra, _, sta = oracle.df_async(G, H, ed, ei, Ra, p)
        assert st.converged and sta.converged
        cur = s.current()
        exact = oracle.dense_solve(n, cur.src, cur.dst, self_loops=sl)
        assert np.max(np.abs(R - exact)) <= 2e-9
        assert np.max(np.abs(Ra - exact)) <= 2e-9
        G = H
    assert abs(R.sum() - 1.0) <= 1e-8


def test_df_error_not_above_static_error():
    """Section 4.3 / 5.2: with tau_f = tau / 1e5, DF's L1 error against the reference
    Static PageRank is not above Static's at the same tau (checked on a seeded R-MAT)."""
    g = synth.rmat(11, 8, seed=1)
    G = oracle.Graph.build(g.n, g.src, g.dst)
    R, _ = oracle.static_pr(G)
    s = synth.BatchStream(g, seed=1)
    for t in range(3):
        b = s.next(1e-3)
        H, ed, ei = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        R, _, st = oracle.df_sync(G, H, ed, ei, R)
        ref, _ = oracle.reference_static(H)
        Rs, _ = oracle.static_pr(H)
        assert np.abs(R - ref).sum() <= np.abs(Rs - ref).sum()
        G = H


def test_dt_teleport_reaches_the_exact_solution():
    """Without self-loops a batch moves the dead-end mass D and with it the teleport share
    alpha D / n of every vertex, reached or not: Dynamic Traversal from the exact old ranks
    must still land on the exact new ranks (dense solve with teleport), which it can only
    do by taking every vertex as affected."""
    g = synth.rmat(8, 4, seed=9)
    n = g.n
    op = oracle.Params(tol=1e-14, dead_end=oracle.TELEPORT)
    G = oracle.Graph.build(n, g.src, g.dst, self_loops=False)
    R = oracle.dense_solve(n, g.src, g.dst, self_loops=False)
    s = synth.BatchStream(g, seed=9)
    for t in range(2):
        b = s.next(2e-2)
        H, ed, ei = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        R, aff, st = oracle.dt_sync(G, H, ed, ei, R, op)
        assert st.converged and st.affected_final == n
        cur = s.current()
        exact = oracle.dense_solve(n, cur.src, cur.dst, self_loops=False)
        assert np.max(np.abs(R - exact)) <= 1e-12
        G = H


def _union_reach(n, old_pairs, new_pairs, sources):
    """Brute force: vertices reachable from the sources in the union of both edge sets
    (self-loops added).  Every edge in only one graph starts at a source, so this is the
    set reachable from some source in G^{t-1} or in G^t."""
    adj = {v: {v} for v in range(n)}
    for u, v in list(old_pairs) + list(new_pairs):
        adj[u].add(v)
    seen, stack = set(), list(sources)
    while stack:
        x = stack.pop()
        if x in seen:
            continue
        seen.add(x)
        stack.extend(adj[x] - seen)
    return seen


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_dt_affected_set_is_reachability(seed):
    """Section 3.3.2: Dynamic Traversal marks exactly the vertices reachable from the
    sources of the effective changes in G^{t-1} or G^t (checked against a brute-force
    search), and that set contains everything Dynamic Frontier marks."""
    rng = random.Random(seed)
    n = 40
    pairs = {(rng.randrange(n), rng.randrange(n)) for _ in range(50)}
    pairs = {(u, v) for u, v in pairs if u != v}
    g = synth.from_pairs(n, sorted(pairs), "random")
    G = oracle.Graph.build(n, g.src, g.dst)
    R, _ = oracle.static_pr(G)
    dels = rng.sample(sorted(pairs), 3)
    ins = [(rng.randrange(n), rng.randrange(n)) for _ in range(3)]
    H, ed, ei = G.apply([u for u, _ in dels], [v for _, v in dels], [u for u, _ in ins], [v for _, v in ins])
    new_pairs = (pairs - set(dels)) | {(u, v) for u, v in ins if u != v}
    sources = set(ed[0].tolist()) | set(ei[0].tolist())
    Rt, aff_t, _ = oracle.dt_sync(G, H, ed, ei, R)
    Rf, aff_f, _ = oracle.df_sync(G, H, ed, ei, R)
    assert set(np.nonzero(aff_t)[0].tolist()) == _union_reach(n, pairs, new_pairs, sources)
    assert not np.any(aff_f & ~aff_t)


def test_dt_reaches_the_exact_solution():
    """Vertices no source reaches keep their in-rows and their in-neighbours' out-degrees,
    so their exact ranks do not change; Dynamic Traversal from the exact old ranks must
    therefore land on the exact new ranks (dense solve), up to the iteration tolerance."""
    g = synth.rmat(8, 4, seed=7)
    n = g.n
    G = oracle.Graph.build(n, g.src, g.dst)
    R = oracle.dense_solve(n, g.src, g.dst)
    s = synth.BatchStream(g, seed=7)
    p = oracle.Params(tol=1e-14)
    for t in range(3):
        b = s.next(2e-2)
        H, ed, ei = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        R, aff, st = oracle.dt_sync(G, H, ed, ei, R, p)
        assert st.converged and 0 < st.affected_final <= n
        cur = s.current()
        exact = oracle.dense_solve(n, cur.src, cur.dst)
        assert np.max(np.abs(R - exact)) <= 1e-12
        G = H
