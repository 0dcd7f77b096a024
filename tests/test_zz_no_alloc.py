"""pr_static_noalloc: Static PageRank for callers that must not allocate device memory.

Such callers (code that takes all of its device memory from a host application's own pool,
latency-critical code that cannot take the device-wide synchronisation of cudaMalloc, or
plugins handed buffers without the right to allocate) pass the graph and the output in
device memory, and the library works in a fixed array of its own.  The ranks must match
the allocating entry point's (pr_static on a graph handle) and the FP64 oracle's within the
tolerance of the other tests, on consecutive calls that share that array, up to the
largest accepted size.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import __graft_entry__
import oracle
import synth

pytestmark = pytest.mark.gpu

TOL64 = 1e-9


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()
    from paper_2401_03256_gb300 import prdf

    prdf.load()
    return prdf, torch


def _reference(prdf, g):
    """Ranks and iteration count of the allocating path, and the stored in-edge CSR."""
    with prdf.Graph(g.n, g.src, g.dst) as A:
        st = A.static()
        off, col = A.csr(1)
        return A.ranks().copy(), st.iterations, off, col


def _call(prdf, torch, n, off_d, col_d, out):
    """One call through the C ABI; returns (status, stats)."""
    s = prdf.pr_stats()
    torch.cuda.synchronize()
    st = prdf.load().pr_static_noalloc(n, int(col_d.numel()), off_d.data_ptr(), col_d.data_ptr(), None,
                                       torch.cuda.current_stream().cuda_stream, out.data_ptr(), ctypes.byref(s))
    return st, s


def _device_csr(torch, off, col):
    off_d = torch.from_numpy(np.asarray(off, dtype=np.int64)).cuda()
    col_d = torch.from_numpy(np.asarray(col, dtype=np.uint32).view(np.int32)).cuda()
    return off_d, col_d


def test_matches_allocating_static_on_consecutive_calls(env):
    prdf, torch = env
    # the largest accepted size (the last bytes of the array in use), a smaller graph, and
    # the largest again: each call must start clean although the shared array keeps the
    # previous call's contents
    graphs = [synth.rmat(18, 8, seed=60), synth.rmat(14, 8, seed=61), synth.rmat(11, 16, seed=62)]
    assert graphs[0].n == prdf.PR_NOALLOC_MAX_VERTICES
    refs = [_reference(prdf, g) for g in graphs]
    ors = []
    for g in graphs:
        G = oracle.Graph.build(g.n, g.src, g.dst)
        ors.append(oracle.static_pr(G)[0])
        G.close()
    for k, gi in enumerate([0, 1, 2, 0]):
        g = graphs[gi]
        R_ref, it_ref, off, col = refs[gi]
        off_d, col_d = _device_csr(torch, off, col)
        out = torch.full((g.n,), -1.0, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st, s = _call(prdf, torch, g.n, off_d, col_d, out)
        torch.cuda.synchronize()
        assert st == prdf.PR_OK, k
        R = out.cpu().numpy()
        assert np.max(np.abs(R - R_ref)) <= TOL64, k  # the allocating entry point
        assert np.max(np.abs(R - ors[gi])) <= TOL64, k  # the oracle
        assert s.converged == 1 and abs(s.iterations - it_ref) <= 1, (k, s.iterations, it_ref)
        assert abs(R.sum() - 1.0) <= 1e-9
        if k >= 1:
            # after the first call on the device nothing more is allocated
            assert torch.cuda.mem_get_info()[0] == free_before, k


def test_rejects_oversized_and_malformed_input(env):
    prdf, torch = env
    lib = prdf.load()
    n_big = prdf.PR_NOALLOC_MAX_VERTICES + 1
    assert lib.pr_static_noalloc(n_big, 0, None, None, None, None, None, None) == prdf.PR_ERR_CAPACITY
    g = synth.rmat(8, 8, seed=63)
    _, _, off, col = _reference(prdf, g)
    out = torch.zeros(g.n, dtype=torch.float64, device="cuda")
    # a column id >= n
    bad_col = np.array(col, dtype=np.uint32)
    bad_col[5] = g.n
    off_d, col_d = _device_csr(torch, off, bad_col)
    st, _ = _call(prdf, torch, g.n, off_d, col_d, out)
    assert st == prdf.PR_ERR_VERTEX_RANGE
    # decreasing offsets
    bad_off = np.array(off, dtype=np.int64)
    bad_off[3], bad_off[4] = bad_off[4], bad_off[3] - 1
    off_d, col_d = _device_csr(torch, bad_off, col)
    st, _ = _call(prdf, torch, g.n, off_d, col_d, out)
    assert st == prdf.PR_ERR_INVALID_ARG
    assert torch.count_nonzero(out).item() == 0  # nothing written on rejection
    # host memory is refused
    off_h = np.asarray(off, dtype=np.uint64)
    assert lib.pr_static_noalloc(g.n, len(col), off_h.ctypes.data, col_d.data_ptr(), None, None,
                                 out.data_ptr(), None) == prdf.PR_ERR_INVALID_ARG
    # a valid call still works afterwards
    off_d, col_d = _device_csr(torch, off, col)
    st, s = _call(prdf, torch, g.n, off_d, col_d, out)
    assert st == prdf.PR_OK and s.converged == 1
