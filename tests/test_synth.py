"""The seeded input generators: structure the recipes promise (no method arithmetic)."""
import numpy as np

import synth


def _sorted_unique_no_self(g):
    k = g.keys()
    assert np.all(k[1:] > k[:-1])
    assert not np.any(g.src == g.dst)
    assert g.src.max() < g.n and g.dst.max() < g.n


def test_kmer_like_structure():
    g = synth.kmer(200_000, seed=3)
    _sorted_unique_no_self(g)
    rev = np.sort((g.dst.astype(np.uint64) << np.uint64(32)) | g.src.astype(np.uint64))
    assert np.array_equal(rev, g.keys())  # symmetric, like the k-mer graphs
    deg = np.bincount(g.src, minlength=g.n)
    assert 2.0 <= g.m / g.n <= 2.2  # 3.0-3.2 with self-loops
    assert (deg == 0).sum() <= 70 and deg.max() <= 8  # isolated only where a jump passes the end
    assert np.array_equal(synth.kmer(200_000, seed=3).keys(), g.keys())
    assert not np.array_equal(synth.kmer(200_000, seed=4).keys(), g.keys())


def test_kmer_like_tiny_and_chain_only():
    assert synth.kmer(1, seed=1).m == 0
    g = synth.kmer(2, mean_chain=1e9, branch_frac=0.0, seed=1)
    assert sorted(zip(g.src.tolist(), g.dst.tolist())) == [(0, 1), (1, 0)]
    g = synth.kmer(1000, mean_chain=1e9, branch_frac=0.0, seed=2)
    assert g.m == 2 * 999  # one symmetric path through all vertices
    deg = np.bincount(g.src, minlength=g.n)
    assert np.bincount(deg).tolist() == [0, 2, 998]


def test_batches_of_each_mix():
    g = synth.rmat(10, 8, seed=1)
    s = synth.BatchStream(g, seed=2)
    for share, f in ((1.0, 1e-2), (0.0, 1e-2), (0.8, 1e-2)):
        b = s.next(f, ins_share=share)
        k = max(1, round(f * g.m))
        assert b.size == k
        assert b.ins_src.shape[0] == round(share * k)
    ek = set(s.current().keys().tolist())
    b = s.next(1e-2, apply=False)
    assert all(((int(u) << 32) | int(v)) in ek for u, v in zip(b.del_src, b.del_dst))
    assert not any(((int(u) << 32) | int(v)) in ek for u, v in zip(b.ins_src, b.ins_dst))
