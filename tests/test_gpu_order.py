"""The internal vertex numbering of single-graph handles is invisible at the boundary.

A handle created with vertex_order 2 or 3 renumbers its vertices breadth-first, from the
vertex of largest degree or from evenly spaced vertices; one created with
vertex_order 1 keeps the caller's ids; vertex_order 0 (the default) takes the better
internal numbering only where a model of the short rows' gathers finds it cheaper.  In
64-bit mode every in-edge sum is exact, so all must agree bit for bit: ranks after Static,
Naive-dynamic, Dynamic Traversal and Dynamic Frontier (Algorithm 1) calls, iteration
counts, the affected sets (a set of caller ids) and the exported CSR.  FP32 sums round in
another order, so there the two agree within the FP32 parity tolerance.  Graphs with vertices that no path reaches from the
first level (isolated vertices, several components, a chain longer than the level cap)
exercise the id-ordered tail.
"""
import numpy as np
import pytest

import __graft_entry__
import oracle
import synth

pytestmark = pytest.mark.gpu

TOL32 = 5e-6


@pytest.fixture(scope="module")
def prdf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    from paper_2401_03256_gb300 import prdf as mod

    mod.load()
    return mod


def _params(prdf, order, f32=False):
    p = prdf.pr_params_default()
    p.vertex_order = order
    p.precision = prdf.PR_F32 if f32 else prdf.PR_F64
    return p


def _two_islands():
    # two R-MAT graphs side by side plus isolated vertices at the end
    a, b = synth.rmat(10, 8, seed=3), synth.rmat(9, 8, seed=4)
    src = np.concatenate([a.src, b.src + a.n]).astype(np.uint32)
    dst = np.concatenate([a.dst, b.dst + a.n]).astype(np.uint32)
    return synth.from_pairs(a.n + b.n + 37, zip(src.tolist(), dst.tolist()), "two-islands")


def _graphs():
    # the k-mer-like chain needs more than the 1024-level cap from one seed
    return [synth.rmat(12, 8, seed=5), synth.grid(40, 30, seed=6), _two_islands(), synth.kmer(200_000, seed=9)]


@pytest.mark.parametrize("order", [2, 3, 0])
@pytest.mark.parametrize("gi", range(4))
def test_numbering_is_invisible_fp64(prdf, gi, order):
    g = _graphs()[gi]
    bs = synth.BatchStream(g, seed=7)
    batches = [bs.next(f) for f in (1e-4, 1e-3, 1e-2)]
    with prdf.Graph(g.n, g.src, g.dst, _params(prdf, order)) as A, \
            prdf.Graph(g.n, g.src, g.dst, _params(prdf, 1)) as B:
        sa, sb = A.static(), B.static()
        assert sa.iterations == sb.iterations
        assert np.array_equal(A.ranks(), B.ranks())
        for d in (0, 1):  # rows come out sorted in both
            oa, ca = A.csr(d)
            ob, cb = B.csr(d)
            assert np.array_equal(oa, ob) and np.array_equal(ca, cb)
        for k, b in enumerate(batches):
            for H in (A, B):
                H.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            mode = ("frontier", "traversal", "naive")[k % 3]
            sa, sb = getattr(A, mode)(), getattr(B, mode)()
            assert sa.iterations == sb.iterations, mode
            assert sa.affected_final == sb.affected_final, mode
            assert np.array_equal(A.ranks(), B.ranks()), mode
            if mode != "naive":
                assert np.array_equal(np.sort(A.affected()), np.sort(B.affected())), mode
        oa, ca = A.csr(1)
        ob, cb = B.csr(1)
        assert np.array_equal(oa, ob) and np.array_equal(ca, cb)


@pytest.mark.parametrize("order", [2, 3])
def test_numbering_set_ranks_round_trip(prdf, order):
    g = synth.rmat(11, 8, seed=8)
    rng = np.random.default_rng(9)
    r = rng.random(g.n)
    r /= r.sum() * 1.0001
    with prdf.Graph(g.n, g.src, g.dst, _params(prdf, order)) as A, \
            prdf.Graph(g.n, g.src, g.dst, _params(prdf, 1)) as B:
        A.set_ranks(r)
        B.set_ranks(r)
        assert np.array_equal(A.ranks(), B.ranks())
        b = synth.BatchStream(g, seed=10).next(1e-3)
        for H in (A, B):
            H.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        sa, sb = A.frontier(), B.frontier()
        assert sa.iterations == sb.iterations
        assert np.array_equal(A.ranks(), B.ranks())


@pytest.mark.parametrize("order", [2, 3])
def test_numbering_fp32_within_tolerance(prdf, order):
    g = synth.rmat(12, 8, seed=11)
    bs = synth.BatchStream(g, seed=12)
    b = bs.next(1e-3)
    h = bs.current()
    G = oracle.Graph.build(g.n, g.src, g.dst)
    with prdf.Graph(g.n, g.src, g.dst, _params(prdf, order, f32=True)) as A:
        A.static()
        assert np.max(np.abs(A.ranks() - oracle.static_pr(G)[0])) <= TOL32
        A.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        A.frontier()
        G2 = oracle.Graph.build(h.n, h.src, h.dst)
        assert np.max(np.abs(A.ranks() - oracle.static_pr(G2)[0])) <= TOL32


@pytest.mark.parametrize("order", [-1, 4])
def test_vertex_order_out_of_range_rejected(prdf, order):
    g = synth.rmat(8, 4, seed=13)
    with pytest.raises(prdf.PrdfError) as e:
        prdf.Graph(g.n, g.src, g.dst, _params(prdf, order))
    assert e.value.status == prdf.PR_ERR_INVALID_ARG


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("n", [1, 5])
def test_numbering_degenerate(prdf, n, order):
    # one vertex and no edges; five vertices, two edges, two of them unreached from the seed
    src = np.array([], np.uint32) if n == 1 else np.array([4, 0], np.uint32)
    dst = np.array([], np.uint32) if n == 1 else np.array([0, 3], np.uint32)
    with prdf.Graph(n, src, dst, _params(prdf, order)) as A, prdf.Graph(n, src, dst, _params(prdf, 1)) as B:
        A.static()
        B.static()
        assert np.array_equal(A.ranks(), B.ranks())


def _union(gs):
    firsts = np.cumsum([0] + [g.n for g in gs])
    src = np.concatenate([g.src.astype(np.uint64) + firsts[i] for i, g in enumerate(gs)]).astype(np.uint32)
    dst = np.concatenate([g.dst.astype(np.uint64) + firsts[i] for i, g in enumerate(gs)]).astype(np.uint32)
    return firsts, src, dst


@pytest.mark.parametrize("order", [2, 0])
def test_batched_numbering_is_invisible_fp64(prdf, order):
    # each graph numbered within its own id range; results bit-identical to the caller's ids
    gs = [synth.rmat(11, 8, seed=21), synth.grid(30, 20, seed=22), synth.rmat(9, 4, seed=23), _two_islands()]
    firsts, src, dst = _union(gs)
    sizes = [g.n for g in gs]
    bss = [synth.BatchStream(g, seed=24 + i) for i, g in enumerate(gs)]
    with prdf.Graph.batched(sizes, src, dst, _params(prdf, order)) as A, \
            prdf.Graph.batched(sizes, src, dst, _params(prdf, 1)) as B:
        A.static()
        B.static()
        assert np.array_equal(A.ranks(), B.ranks())
        for f in (1e-3, 1e-2):
            bs = [s.next(f) for s in bss]
            parts = [np.concatenate([(getattr(b, k).astype(np.uint64) + firsts[i]).astype(np.uint32)
                                     for i, b in enumerate(bs)]) for k in ("del_src", "del_dst", "ins_src", "ins_dst")]
            for H in (A, B):
                H.apply(*parts)
            A.frontier()
            B.frontier()
            assert np.array_equal(A.ranks(), B.ranks())
            assert np.array_equal(np.sort(A.affected()), np.sort(B.affected()))
            ca, cb = A.component_stats(), B.component_stats()
            assert [c.iterations for c in ca] == [c.iterations for c in cb]
        for d in (0, 1):
            oa, xa = A.csr(d)
            ob, xb = B.csr(d)
            assert np.array_equal(oa, ob) and np.array_equal(xa, xb)


def test_batched_rejects_seeded_numbering(prdf):
    gs = [synth.rmat(8, 4, seed=25), synth.rmat(8, 4, seed=26)]
    firsts, src, dst = _union(gs)
    with pytest.raises(prdf.PrdfError) as e:
        prdf.Graph.batched([g.n for g in gs], src, dst, _params(prdf, 3))
    assert e.value.status == prdf.PR_ERR_INVALID_ARG
