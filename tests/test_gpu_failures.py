"""Failure detection without a GPU fault (the failures are made on the host or by a wait
limit, never by a trap, a bad address or an endless loop).

* A grid barrier of the persistent launch waits at most its limit; with a 1 us limit the
  waits of a Static call run out, the blocks end the launch, and the call returns
  PR_ERR_DEVICE_TIMEOUT.  The context stays usable: with the default limit the next call
  matches the oracle.
* A device allocation failure (injected on the host) in a batch update returns
  PR_ERR_OUT_OF_MEMORY and leaves the graph as it was; the same batch then applies.
"""
import numpy as np
import pytest

import __graft_entry__
import oracle
import synth

pytestmark = pytest.mark.gpu

PR_ERR_OUT_OF_MEMORY = 3
PR_ERR_DEVICE_TIMEOUT = 5


@pytest.fixture(scope="module")
def prdf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    from paper_2401_03256_gb300 import prdf as mod

    mod.load()
    return mod


def test_barrier_wait_runs_out_and_the_handle_recovers(prdf):
    # teleport mode: Static runs in the persistent launch, one grid barrier per iteration
    g = synth.rmat(14, 8, seed=31)
    p = prdf.pr_params_default()
    p.dead_end = prdf.PR_DEADEND_TELEPORT
    G = oracle.Graph.build(g.n, g.src, g.dst, self_loops=False)
    R_or, _ = oracle.static_pr(G, oracle.Params(dead_end=oracle.TELEPORT))
    with prdf.Graph(g.n, g.src, g.dst, p) as dg:
        t = dg.tuning()
        dg.set_tuning(t.bin_lo, t.bin_hi, t.dense_div, t.blocks_per_sm, t.df_split, barrier_us=1)
        assert dg.tuning().barrier_us == 1
        timed_out = 0
        for _ in range(5):
            try:
                dg.static()
            except prdf.PrdfError as e:
                assert e.status == PR_ERR_DEVICE_TIMEOUT
                timed_out += 1
        assert timed_out > 0
        dg.set_tuning(t.bin_lo, t.bin_hi, t.dense_div, t.blocks_per_sm, t.df_split, barrier_us=0)
        st = dg.static()
        assert st.converged and np.max(np.abs(dg.ranks() - R_or)) <= 1e-9


def test_allocation_failure_leaves_the_graph_unchanged(prdf):
    g = synth.rmat(13, 8, seed=32)
    s = synth.BatchStream(g, seed=32)
    small, big = s.next(1e-3), s.next(2e-1)  # the second needs more batch scratch
    with prdf.Graph(g.n, g.src, g.dst) as dg:
        dg.apply(small.del_src, small.del_dst, small.ins_src, small.ins_dst)
        before = [dg.csr(d) for d in (0, 1)]
        prdf.pr_inject_alloc_failure(0)
        try:
            with pytest.raises(prdf.PrdfError) as ei:
                dg.apply(big.del_src, big.del_dst, big.ins_src, big.ins_dst)
        finally:
            prdf.pr_inject_alloc_failure(-1)
        assert ei.value.status == PR_ERR_OUT_OF_MEMORY
        after = [dg.csr(d) for d in (0, 1)]
        for (o0, c0), (o1, c1) in zip(before, after):
            assert np.array_equal(o0, o1) and np.array_equal(c0, c1)
        # the pending marks of the small batch survived: the update still matches the oracle
        G = oracle.Graph.build(g.n, g.src, g.dst)
        R0, _ = oracle.static_pr(G)
        H, ed, ei2 = G.apply(small.del_src, small.del_dst, small.ins_src, small.ins_dst)
        dg.set_ranks(R0)
        dg.frontier()
        R_df, _, _ = oracle.df_sync(G, H, ed, ei2, R0)
        assert np.max(np.abs(dg.ranks() - R_df)) <= 1e-9
        dg.apply(big.del_src, big.del_dst, big.ins_src, big.ins_dst)
        H2, _, _ = H.apply(big.del_src, big.del_dst, big.ins_src, big.ins_dst)
        for d in (0, 1):
            off, col = dg.csr(d)
            eoff, ecol = H2.csr(d)
            assert np.array_equal(off, eoff) and np.array_equal(col, ecol)


@pytest.mark.parametrize("order", [0, 2])
def test_creation_out_of_memory_is_reported(prdf, order):
    # every graph allocation fails: the numbering's transient build (vertex_order 0 falls
    # back to the caller's numbering) and then the handle's own build report it
    g = synth.rmat(12, 8, seed=34)
    p = prdf.pr_params_default()
    p.vertex_order = order
    prdf.pr_inject_alloc_failure(0)
    try:
        with pytest.raises(prdf.PrdfError) as ei:
            prdf.Graph(g.n, g.src, g.dst, p)
    finally:
        prdf.pr_inject_alloc_failure(-1)
    assert ei.value.status == PR_ERR_OUT_OF_MEMORY
    with prdf.Graph(g.n, g.src, g.dst, p) as dg:  # nothing left behind
        assert dg.static().converged


def test_set_ranks_rejects_what_is_not_a_distribution(prdf):
    torch = pytest.importorskip("torch")
    g = synth.rmat(10, 8, seed=33)
    with prdf.Graph(g.n, g.src, g.dst) as dg:
        dg.static()
        R = dg.ranks().copy()
        bads = []
        for k, x in ((3, np.nan), (5, -1e-3), (7, np.inf), (9, 2.5)):
            b = R.copy()
            b[k] = x
            bads.append(b)
        bads.append(np.full(g.n, 3.0 / g.n))  # mass 3
        for b in bads:
            for arr in (b, torch.from_numpy(b).cuda()):  # host and device arrays
                with pytest.raises(prdf.PrdfError) as ei:
                    dg.set_ranks(arr)
                assert ei.value.status == 1  # PR_ERR_INVALID_ARG
                assert np.array_equal(dg.ranks(), R)  # unchanged
        # the drift of chained approximate updates is accepted (mass up to 2)
        dg.set_ranks(R * 1.5)
        assert np.allclose(dg.ranks(), R * 1.5, rtol=0, atol=1e-15)
