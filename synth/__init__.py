"""Seeded synthetic inputs for Dynamic Frontier PageRank (graphs and batch updates).

Inputs only: this package holds none of the method's arithmetic.  Both the oracle
(``oracle/``) and the CUDA library consume what it produces; it imports neither.

Recipes (the paper's datasets, Table 1, are not available; these stand in for them):

* R-MAT / Kronecker: 2^scale vertices, round(ef * 2^scale) sampled pairs, quadrant
  probabilities (a, b, c, d) = (0.57, 0.19, 0.19, 0.05), one seeded vertex relabelling,
  self-pairs and duplicates removed.  Stands in for the web and social graphs.
* Grid: rows x cols, arcs to the four grid neighbours, plus 1% uniformly random
  long-range arcs.  Stands in for the road networks (average degree about 4).
* k-mer-like: symmetric chains over a random vertex order (mean length 24), a cut joining
  a vertex 2..65 places further along instead, 5% more such short branches: one long
  component with local shortcuts only; average out-degree about 2.1, 3.1 with
  self-loops.  Stands in for the protein k-mer graphs (171-214 M vertices).
* Batches (Section 5.1.4): k = max(1, round(f |E|)) edges of the original graph's
  |E|; 80% insertions of uniform random absent pairs, 20% deletions of existing edges
  drawn uniformly without replacement.  Successive batches are drawn against the
  updated edge set.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile libsynth.so beside its source with gcc (OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    lib.synth_rmat.restype = ctypes.c_void_p
    lib.synth_rmat.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, ctypes.c_uint64, ctypes.c_int, u64p]
    lib.synth_grid.restype = ctypes.c_void_p
    lib.synth_grid.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, ctypes.c_uint64, u64p]
    lib.synth_kmer.restype = ctypes.c_void_p
    lib.synth_kmer.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_double, ctypes.c_uint64, u64p]
    lib.synth_free.argtypes = [ctypes.c_void_p]
    lib.synth_free.restype = None
    lib.synth_stream_create.restype = ctypes.c_void_p
    lib.synth_stream_create.argtypes = [ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint64,
                                        ctypes.c_uint64, ctypes.c_uint64]
    lib.synth_stream_destroy.argtypes = [ctypes.c_void_p]
    lib.synth_stream_destroy.restype = None
    lib.synth_stream_m.restype = ctypes.c_uint64
    lib.synth_stream_m.argtypes = [ctypes.c_void_p]
    lib.synth_stream_keys.restype = ctypes.c_void_p
    lib.synth_stream_keys.argtypes = [ctypes.c_void_p]
    lib.synth_batch_sizes.restype = None
    lib.synth_batch_sizes.argtypes = [ctypes.c_uint64, ctypes.c_double, ctypes.c_double, u64p, u64p]
    lib.synth_stream_next.restype = ctypes.c_int
    lib.synth_stream_next.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    _lib = lib
    return lib


@dataclass
class EdgeList:
    """A directed graph as sorted unique (src, dst) arrays without self-pairs."""
    n: int
    src: np.ndarray  # uint32
    dst: np.ndarray  # uint32
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.src.shape[0])

    def keys(self) -> np.ndarray:
        return (self.src.astype(np.uint64) << np.uint64(32)) | self.dst.astype(np.uint64)


def _take_keys(ptr: int, m: int) -> np.ndarray:
    lib = _load()
    if not ptr:
        raise MemoryError("synth: allocation failed")
    buf = (ctypes.c_uint64 * max(m, 1)).from_address(ptr)
    keys = np.frombuffer(buf, dtype=np.uint64, count=m).copy()
    lib.synth_free(ptr)
    return keys


def _from_keys(n: int, keys: np.ndarray, name: str) -> EdgeList:
    src = (keys >> np.uint64(32)).astype(np.uint32)
    dst = (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    return EdgeList(n, src, dst, name)


def rmat(scale: int, ef: float, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, permute: bool = True) -> EdgeList:
    """R-MAT graph with 2^scale vertices and round(ef 2^scale) samples (deduplicated)."""
    lib = _load()
    m = ctypes.c_uint64(0)
    ptr = lib.synth_rmat(scale, ef, a, b, c, seed, 1 if permute else 0, ctypes.byref(m))
    keys = _take_keys(ptr, m.value)
    return _from_keys(1 << scale, keys, f"rmat-s{scale}-ef{ef:g}")


def grid(rows: int, cols: int, longrange_frac: float = 0.01, seed: int = 1) -> EdgeList:
    """Directed 2D grid (4-neighbour arcs) with a fraction of random long-range arcs."""
    lib = _load()
    m = ctypes.c_uint64(0)
    ptr = lib.synth_grid(rows, cols, longrange_frac, seed, ctypes.byref(m))
    keys = _take_keys(ptr, m.value)
    return _from_keys(rows * cols, keys, f"grid-{rows}x{cols}")


def kmer(n: int, mean_chain: float = 24.0, branch_frac: float = 0.05, seed: int = 1) -> EdgeList:
    """Low-degree stand-in for the protein k-mer graphs: symmetric chains over a random
    vertex order, local junctions where a chain is cut, a few short branches."""
    lib = _load()
    m = ctypes.c_uint64(0)
    ptr = lib.synth_kmer(n, mean_chain, branch_frac, seed, ctypes.byref(m))
    keys = _take_keys(ptr, m.value)
    return _from_keys(n, keys, f"kmer-{n}")


def from_pairs(n: int, pairs, name: str = "") -> EdgeList:
    """EdgeList from explicit (u, v) pairs: sorted, unique, self-pairs removed."""
    arr = np.asarray(list(pairs), dtype=np.uint64).reshape(-1, 2)
    keys = (arr[:, 0] << np.uint64(32)) | arr[:, 1]
    keys = np.unique(keys)
    keys = keys[(keys >> np.uint64(32)) != (keys & np.uint64(0xFFFFFFFF))]
    return _from_keys(n, keys, name)


def batch_sizes(base_m: int, frac: float, ins_share: float = 0.8):
    """(k_ins, k_del) for a batch of fraction `frac` of base_m edges."""
    lib = _load()
    ki = ctypes.c_uint64(0)
    kd = ctypes.c_uint64(0)
    lib.synth_batch_sizes(base_m, frac, ins_share, ctypes.byref(ki), ctypes.byref(kd))
    return ki.value, kd.value


@dataclass
class Batch:
    """One batch update: deletions and insertions as uint32 arrays."""
    del_src: np.ndarray
    del_dst: np.ndarray
    ins_src: np.ndarray
    ins_dst: np.ndarray

    @property
    def size(self) -> int:
        return int(self.del_src.shape[0] + self.ins_src.shape[0])


class BatchStream:
    """Successive random 80/20 batches against an evolving copy of the edge set."""

    def __init__(self, g: EdgeList, seed: int = 1, base_m: int | None = None):
        lib = _load()
        self.n = g.n
        self.base_m = g.m if base_m is None else int(base_m)
        keys = np.ascontiguousarray(g.keys())
        self._h = lib.synth_stream_create(g.n, keys.ctypes.data, keys.shape[0], self.base_m, seed)
        if not self._h:
            raise MemoryError("synth: stream allocation failed")

    def next(self, frac: float, ins_share: float = 0.8, apply: bool = True) -> Batch:
        lib = _load()
        ki, kd = batch_sizes(self.base_m, frac, ins_share)
        ds = np.empty(kd, np.uint32)
        dd = np.empty(kd, np.uint32)
        is_ = np.empty(ki, np.uint32)
        id_ = np.empty(ki, np.uint32)
        rc = lib.synth_stream_next(self._h, frac, ins_share, 1 if apply else 0,
                                   ds.ctypes.data, dd.ctypes.data, is_.ctypes.data, id_.ctypes.data)
        if rc != 0:
            raise ValueError("synth: batch request cannot be met on this graph")
        return Batch(ds, dd, is_, id_)

    def current(self) -> EdgeList:
        """The stream's current edge set (after the batches it applied)."""
        lib = _load()
        m = lib.synth_stream_m(self._h)
        ptr = lib.synth_stream_keys(self._h)
        buf = (ctypes.c_uint64 * max(m, 1)).from_address(ptr)
        keys = np.frombuffer(buf, dtype=np.uint64, count=m).copy()
        return _from_keys(self.n, keys, "stream")

    def close(self):
        if getattr(self, "_h", None):
            _load().synth_stream_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
