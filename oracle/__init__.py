"""FP64 sequential oracle for Dynamic Frontier PageRank (arXiv 2401.03256).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The product library never loads
it, and it shares no code with the CUDA path (it is plain C compiled with gcc, wrapped
here with ctypes).

Functions and the passages they follow:

* ``Graph.build``      Section 3.1 / 5.1.4: deduplicated pairs, self-loops added.
* ``Graph.apply``      Section 3.2: E^t = (E^{t-1} minus D) union I, effective deltas.
* ``static_pr``        Section 3.1, Eq. 1: power iteration from 1/n.
* ``naive_pr``         Section 3.3.1: power iteration from the previous ranks.
* ``df_sync``          Algorithm 1, synchronous reading (Section 4.2).
* ``df_async``         Algorithm 1, asynchronous reading (Section 4.2).
* ``reference_static`` Section 5.1.5: Static PageRank at tau = 1e-100, 500 iterations.
* ``dense_solve``      (I - alpha P^T) r = (1 - alpha)/n with dead-end teleport.

Every function is pinned by ``tests/test_oracle_pins.py``; only the later iterations of
the paper's worked example (Figure 1, whose drawing is missing) are parity unpinned.

``use_threads(k)`` switches a process to the -fopenmp build of the same C source (its
vertex loops are annotated with schedule(dynamic, 2048), the paper's CPU schedule); its
results equal the sequential build's bit for bit (``tests/test_oracle_threads.py``).  It
times the oracle on all host cores and computes the expected values of the largest
workloads; the default is the sequential build.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prdf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lib = None
_want_threads = 1

# Section 5.1.2 and Section 4.3 constants.
ALPHA = 0.85
TOL = 1e-10
FRONTIER_TOL = TOL / 1e5
MAX_ITER = 500
SELF_LOOPS = 0
TELEPORT = 1


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile liboracle.so with gcc (IEEE double, no contraction, no fast-math), or with
    openmp=True the same source with -fopenmp as liboracle_omp.so."""
    lib = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
               "-std=c11", *(["-fopenmp"] if openmp else []), _SRC, "-o", lib + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(lib + ".tmp", lib)
    return lib


def host_cores() -> int:
    """Host cores this process may run on (sched_getaffinity)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def use_threads(k: int) -> int:
    """Run this process's oracle on k threads (k > 1: the -fopenmp build of the same
    source, whose results equal the sequential build's bit for bit).  The build is chosen
    by the first oracle call of the process; returns the threads in effect."""
    global _want_threads
    k = max(1, int(k))
    if _lib is None:
        _want_threads = k
    elif (k > 1) != (_want_threads > 1):
        raise RuntimeError("oracle: the sequential or threaded build is fixed once loaded")
    return int(_load().or_threads(k if k > 1 else 0))


def threads() -> int:
    """Threads the loaded oracle runs its vertex loops on."""
    return int(_load().or_threads(0))


class _Params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("tol", ctypes.c_double),
                ("frontier_tol", ctypes.c_double), ("max_iter", ctypes.c_int32),
                ("dead_end", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("affected_final", ctypes.c_int64), ("vertices_processed", ctypes.c_int64),
                ("edges_processed", ctypes.c_int64), ("last_delta", ctypes.c_double)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    par = _want_threads > 1
    lib = ctypes.CDLL(build(openmp=par))
    vp = ctypes.c_void_p
    u64 = ctypes.c_uint64
    lib.or_threads.restype = ctypes.c_int
    lib.or_threads.argtypes = [ctypes.c_int]
    if par:
        lib.or_threads(_want_threads)
    lib.or_graph_build.restype = vp
    lib.or_graph_build.argtypes = [ctypes.c_uint32, u64, vp, vp, ctypes.c_int]
    lib.or_graph_free.restype = None
    lib.or_graph_free.argtypes = [vp]
    lib.or_graph_n.restype = ctypes.c_uint32
    lib.or_graph_n.argtypes = [vp]
    lib.or_graph_m.restype = u64
    lib.or_graph_m.argtypes = [vp]
    lib.or_graph_export.restype = None
    lib.or_graph_export.argtypes = [vp, ctypes.c_int, vp, vp]
    lib.or_apply_batch.restype = vp
    lib.or_apply_batch.argtypes = [vp, u64, vp, vp, u64, vp, vp, vp, vp, vp, vp, vp, vp]
    for name in ("or_static", "or_naive"):
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        f.argtypes = [vp, ctypes.POINTER(_Params), vp, ctypes.POINTER(_Stats)]
    for name in ("or_df_sync", "or_df_async", "or_dt_sync"):
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        f.argtypes = [vp, vp, ctypes.POINTER(_Params), u64, vp, vp, u64, vp, vp, vp, vp,
                      ctypes.POINTER(_Stats)]
    lib.or_dense_solve.restype = ctypes.c_int
    lib.or_dense_solve.argtypes = [ctypes.c_uint32, u64, vp, vp, ctypes.c_int, ctypes.c_double, vp]
    _lib = lib
    return lib


@dataclass
class Params:
    alpha: float = ALPHA
    tol: float = TOL
    frontier_tol: float = FRONTIER_TOL
    max_iter: int = MAX_ITER
    dead_end: int = SELF_LOOPS

    def _c(self) -> _Params:
        return _Params(self.alpha, self.tol, self.frontier_tol, self.max_iter, self.dead_end)


@dataclass
class Stats:
    iterations: int
    converged: bool
    affected_final: int
    vertices_processed: int
    edges_processed: int
    last_delta: float


def _stats(s: _Stats) -> Stats:
    return Stats(s.iterations, bool(s.converged), s.affected_final, s.vertices_processed,
                 s.edges_processed, s.last_delta)


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


class Graph:
    """Paired out/in adjacency held by the C oracle (immutable; apply returns a new one)."""

    def __init__(self, handle, self_loops: bool):
        self._h = handle
        self.self_loops = self_loops

    @classmethod
    def build(cls, n: int, src, dst, self_loops: bool = True) -> "Graph":
        lib = _load()
        s, d = _u32(src), _u32(dst)
        h = lib.or_graph_build(n, s.shape[0], s.ctypes.data, d.ctypes.data, 1 if self_loops else 0)
        if not h:
            raise ValueError("oracle: vertex id out of range")
        return cls(h, self_loops)

    @property
    def n(self) -> int:
        return int(_load().or_graph_n(self._h))

    @property
    def m(self) -> int:
        return int(_load().or_graph_m(self._h))

    def csr(self, direction: int):
        """(offsets uint64[n+1], columns uint32[m]); direction 0 = out, 1 = in."""
        off = np.empty(self.n + 1, np.uint64)
        col = np.empty(self.m, np.uint32)
        _load().or_graph_export(self._h, direction, off.ctypes.data, col.ctypes.data)
        return off, col

    def apply(self, del_src, del_dst, ins_src, ins_dst):
        """(new graph, (eff_del_src, eff_del_dst), (eff_ins_src, eff_ins_dst))."""
        lib = _load()
        ds, dd, is_, id_ = _u32(del_src), _u32(del_dst), _u32(ins_src), _u32(ins_dst)
        nd, ni = ds.shape[0], is_.shape[0]
        eds = np.empty(max(nd, 1), np.uint32)
        edd = np.empty(max(nd, 1), np.uint32)
        eis = np.empty(max(ni, 1), np.uint32)
        eid = np.empty(max(ni, 1), np.uint32)
        ned = ctypes.c_uint64(0)
        nei = ctypes.c_uint64(0)
        h = lib.or_apply_batch(self._h, nd, ds.ctypes.data, dd.ctypes.data, ni, is_.ctypes.data,
                               id_.ctypes.data, ctypes.addressof(ned), eds.ctypes.data,
                               edd.ctypes.data, ctypes.addressof(nei), eis.ctypes.data, eid.ctypes.data)
        if not h:
            raise ValueError("oracle: vertex id out of range")
        a, b = ned.value, nei.value
        return Graph(h, self.self_loops), (eds[:a].copy(), edd[:a].copy()), (eis[:b].copy(), eid[:b].copy())

    def close(self):
        if getattr(self, "_h", None):
            _load().or_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def static_pr(g: Graph, params: Params | None = None):
    """Static PageRank: (ranks float64[n], Stats)."""
    p = (params or Params())._c()
    R = np.empty(g.n, np.float64)
    st = _Stats()
    _load().or_static(g._h, ctypes.byref(p), R.ctypes.data, ctypes.byref(st))
    return R, _stats(st)


def naive_pr(g: Graph, R_prev, params: Params | None = None):
    """Naive-dynamic PageRank from R_prev: (ranks, Stats)."""
    p = (params or Params())._c()
    R = np.array(R_prev, dtype=np.float64, copy=True)
    st = _Stats()
    _load().or_naive(g._h, ctypes.byref(p), R.ctypes.data, ctypes.byref(st))
    return R, _stats(st)


def _df(fn, g_old: Graph, g_new: Graph, eff_del, eff_ins, R_prev, params):
    p = (params or Params())._c()
    ds, dd = _u32(eff_del[0]), _u32(eff_del[1])
    is_, id_ = _u32(eff_ins[0]), _u32(eff_ins[1])
    R = np.array(R_prev, dtype=np.float64, copy=True)
    aff = np.zeros(g_new.n, np.uint8)
    st = _Stats()
    fn(g_old._h, g_new._h, ctypes.byref(p), ds.shape[0], ds.ctypes.data, dd.ctypes.data,
       is_.shape[0], is_.ctypes.data, id_.ctypes.data, R.ctypes.data, aff.ctypes.data, ctypes.byref(st))
    return R, aff.astype(bool), _stats(st)


def df_sync(g_old: Graph, g_new: Graph, eff_del, eff_ins, R_prev, params: Params | None = None):
    """Dynamic Frontier, synchronous: (ranks, affected flags, Stats)."""
    return _df(_load().or_df_sync, g_old, g_new, eff_del, eff_ins, R_prev, params)


def df_async(g_old: Graph, g_new: Graph, eff_del, eff_ins, R_prev, params: Params | None = None):
    """Dynamic Frontier, asynchronous (paper's CPU form): (ranks, affected flags, Stats)."""
    return _df(_load().or_df_async, g_old, g_new, eff_del, eff_ins, R_prev, params)


def dt_sync(g_old: Graph, g_new: Graph, eff_del, eff_ins, R_prev, params: Params | None = None):
    """Dynamic Traversal (Section 3.3.2): (ranks, affected flags, Stats)."""
    return _df(_load().or_dt_sync, g_old, g_new, eff_del, eff_ins, R_prev, params)


def reference_static(g: Graph, dead_end: int = SELF_LOOPS):
    """Section 5.1.5 reference: Static PageRank at tau = 1e-100 capped at 500 iterations."""
    return static_pr(g, Params(tol=1e-100, max_iter=500, dead_end=dead_end))


def dense_solve(n: int, src, dst, self_loops: bool = True, alpha: float = ALPHA) -> np.ndarray:
    """Exact ranks of a small graph (n <= 4096) by Gaussian elimination."""
    s, d = _u32(src), _u32(dst)
    r = np.empty(n, np.float64)
    rc = _load().or_dense_solve(n, s.shape[0], s.ctypes.data, d.ctypes.data,
                                1 if self_loops else 0, alpha, r.ctypes.data)
    if rc != 0:
        raise ValueError("oracle: dense solve failed")
    return r
