"""The -fopenmp build of the oracle equals the sequential build bit for bit.

The threaded build (the same C source; its vertex loops carry OpenMP annotations with the
paper's schedule(dynamic, 2048), Section 5.1.2) times the oracle on all host cores and
computes the expected values of the largest workloads.  Each vertex's sum is still taken
by one thread in in-edge order, the L-inf maximum is exact and marking only sets flags, so
every rank, flag and counter must come out identical.  The threaded run happens in a
spawned process (the build is fixed per process).
"""
import multiprocessing as mp

import numpy as np

import oracle
import synth


def _workload(threads):
    """Static, Naive-dynamic, Dynamic Frontier (both readings' sync form) and Dynamic
    Traversal over a chain of batches on an R-MAT graph and a grid, in both dead-end
    modes; returns every result."""
    if threads > 1:
        assert oracle.use_threads(threads) == threads
    out = []
    for g, self_loops in ((synth.rmat(14, 8, seed=5), True), (synth.grid(40, 50, seed=6), True),
                          (synth.rmat(11, 4, seed=7), False)):
        G = oracle.Graph.build(g.n, g.src, g.dst, self_loops=self_loops)
        p = oracle.Params(dead_end=oracle.SELF_LOOPS if self_loops else oracle.TELEPORT)
        R, st = oracle.static_pr(G, p)
        out.append((R, st))
        bs = synth.BatchStream(g, seed=8)
        for f in (1e-3, 1e-2):
            b = bs.next(f)
            H, ed, ei = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            Rn, stn = oracle.naive_pr(H, R, p)
            Rd, ad, std = oracle.df_sync(G, H, ed, ei, R, p)
            Rt, at, stt = oracle.dt_sync(G, H, ed, ei, R, p)
            out.extend([(Rn, stn), (Rd, ad, std), (Rt, at, stt)])
            G, R = H, Rd
    return out


def _child(threads, q):
    res = _workload(threads)
    q.put((oracle.threads(), res))


def test_threaded_build_is_bit_identical():
    seq = _workload(1)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_child, args=(4, q))
    p.start()
    used, par = q.get(timeout=600)
    p.join(timeout=60)
    assert used == 4
    assert len(par) == len(seq)
    for a, b in zip(seq, par):
        assert len(a) == len(b)
        for x, y in zip(a, b):
            if isinstance(x, np.ndarray):
                assert x.dtype == y.dtype and np.array_equal(x, y)
            else:
                assert x == y
