"""Thin ctypes binding of libprdf.so (include/prdf.h); argument marshalling only.

Every function here has the name of the C entry point it calls.  Arrays may be numpy
arrays (host) or torch tensors (host or CUDA); they are passed as raw pointers and the
library copies what it needs.  A non-OK status raises PrdfError with pr_last_error's
message.  There is no fallback: if the CUDA library is missing this module fails to
import its functions with an OSError.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libprdf.so")

PR_OK = 0
PR_ERR_INVALID_ARG = 1
PR_ERR_VERTEX_RANGE = 2
PR_ERR_OUT_OF_MEMORY = 3
PR_ERR_CUDA = 4
PR_ERR_DEVICE_TIMEOUT = 5
PR_ERR_CAPACITY = 6
PR_F64 = 0
PR_F32 = 1
PR_DEADEND_SELFLOOP = 0
PR_DEADEND_TELEPORT = 1

EXPORTED = (
    "pr_params_default", "pr_graph_create", "pr_graph_destroy", "pr_apply_batch", "pr_apply_batches", "pr_static",
    "pr_naive_dynamic", "pr_dynamic_frontier", "pr_dynamic_traversal", "pr_dynamic_frontier_async",
    "pr_get_ranks", "pr_set_ranks", "pr_graph_info",
    "pr_get_csr", "pr_get_affected", "pr_get_trace", "pr_kernel_launches", "pr_last_error", "pr_status_string",
    "pr_graph_create_batched", "pr_get_component_stats", "pr_set_tuning", "pr_get_tuning", "pr_autotune",
    "pr_set_graph_launch", "pr_server_config_default", "pr_server_create", "pr_server_add_graph",
    "pr_server_submit", "pr_server_wait", "pr_server_drain", "pr_server_destroy", "pr_static_noalloc",
    "pr_inject_alloc_failure",
)

PR_NOALLOC_MAX_VERTICES = 1 << 18


class pr_params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("tol", ctypes.c_double), ("frontier_tol", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("precision", ctypes.c_int32), ("dead_end", ctypes.c_int32),
                ("bin_lo", ctypes.c_int32), ("bin_hi", ctypes.c_int32), ("vertex_order", ctypes.c_int32)]


class pr_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("affected_final", ctypes.c_int64), ("vertices_processed", ctypes.c_int64),
                ("edges_processed", ctypes.c_int64), ("bytes_algorithmic", ctypes.c_double),
                ("last_delta", ctypes.c_double), ("ms_apply", ctypes.c_double), ("ms_rank", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class pr_tuning(ctypes.Structure):
    _fields_ = [("bin_lo", ctypes.c_int32), ("bin_hi", ctypes.c_int32), ("dense_div", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("df_split", ctypes.c_int32), ("barrier_us", ctypes.c_int32),
                ("chunk_len", ctypes.c_int32), ("group_max", ctypes.c_int32),
                ("ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class pr_server_config(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("max_coalesce", ctypes.c_int32), ("hbm_reserve_bytes", ctypes.c_uint64)]


class pr_request_result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("graph", ctypes.c_int32), ("status", ctypes.c_int32),
                ("t_submit_ms", ctypes.c_double), ("t_start_ms", ctypes.c_double), ("t_done_ms", ctypes.c_double),
                ("coalesced", ctypes.c_int32), ("reserved", ctypes.c_int32), ("stats", pr_stats)]


class pr_server_info(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("waited_for_memory", ctypes.c_int64), ("elapsed_ms", ctypes.c_double)]


class PrdfError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_status_name(status)}: {message}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Loads libprdf.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libprdf.so not found at {path}; build it with paper_2401_03256_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, u32, i32, i64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int32, ctypes.c_int64
    lib.pr_params_default.restype = None
    lib.pr_params_default.argtypes = [ctypes.POINTER(pr_params)]
    lib.pr_graph_create.restype = ctypes.c_int
    lib.pr_graph_create.argtypes = [u32, i64, vp, vp, ctypes.POINTER(pr_params), vp, ctypes.POINTER(vp)]
    lib.pr_graph_destroy.restype = ctypes.c_int
    lib.pr_graph_destroy.argtypes = [vp]
    lib.pr_apply_batch.restype = ctypes.c_int
    lib.pr_apply_batch.argtypes = [vp, i64, vp, vp, i64, vp, vp]
    lib.pr_static_noalloc.restype = ctypes.c_int
    lib.pr_static_noalloc.argtypes = [ctypes.c_uint32, i64, vp, vp, vp, vp, vp, vp]
    lib.pr_apply_batches.restype = ctypes.c_int
    lib.pr_apply_batches.argtypes = [vp, ctypes.c_int32, vp, vp, vp, vp, vp, vp]
    for name in ("pr_static", "pr_naive_dynamic", "pr_dynamic_frontier", "pr_dynamic_traversal",
                 "pr_dynamic_frontier_async"):
        f = getattr(lib, name)
        f.restype = ctypes.c_int
        f.argtypes = [vp, ctypes.POINTER(pr_stats)]
    lib.pr_get_ranks.restype = ctypes.c_int
    lib.pr_get_ranks.argtypes = [vp, vp, u32]
    lib.pr_set_ranks.restype = ctypes.c_int
    lib.pr_set_ranks.argtypes = [vp, vp, u32]
    lib.pr_graph_info.restype = ctypes.c_int
    lib.pr_graph_info.argtypes = [vp, ctypes.POINTER(u32), ctypes.POINTER(i64)]
    lib.pr_get_csr.restype = ctypes.c_int
    lib.pr_get_csr.argtypes = [vp, i32, vp, vp]
    lib.pr_get_affected.restype = ctypes.c_int
    lib.pr_get_affected.argtypes = [vp, vp, i64, ctypes.POINTER(i64)]
    lib.pr_graph_create_batched.restype = ctypes.c_int
    lib.pr_graph_create_batched.argtypes = [i32, vp, i64, vp, vp, ctypes.POINTER(pr_params), vp, ctypes.POINTER(vp)]
    lib.pr_get_component_stats.restype = ctypes.c_int
    lib.pr_get_component_stats.argtypes = [vp, ctypes.POINTER(pr_stats), i32]
    lib.pr_set_tuning.restype = ctypes.c_int
    lib.pr_set_tuning.argtypes = [vp, ctypes.POINTER(pr_tuning)]
    lib.pr_get_tuning.restype = ctypes.c_int
    lib.pr_get_tuning.argtypes = [vp, ctypes.POINTER(pr_tuning)]
    lib.pr_autotune.restype = ctypes.c_int
    lib.pr_autotune.argtypes = [vp, i32, ctypes.POINTER(pr_tuning)]
    lib.pr_set_graph_launch.restype = ctypes.c_int
    lib.pr_set_graph_launch.argtypes = [vp, i32]
    lib.pr_server_config_default.restype = None
    lib.pr_server_config_default.argtypes = [ctypes.POINTER(pr_server_config)]
    lib.pr_server_create.restype = ctypes.c_int
    lib.pr_server_create.argtypes = [ctypes.POINTER(pr_server_config), ctypes.POINTER(vp)]
    lib.pr_server_add_graph.restype = ctypes.c_int
    lib.pr_server_add_graph.argtypes = [vp, vp, ctypes.POINTER(i32)]
    lib.pr_server_submit.restype = ctypes.c_int
    lib.pr_server_submit.argtypes = [vp, i32, i64, vp, vp, i64, vp, vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.pr_server_wait.restype = ctypes.c_int
    lib.pr_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(pr_request_result)]
    lib.pr_server_drain.restype = ctypes.c_int
    lib.pr_server_drain.argtypes = [vp, ctypes.POINTER(pr_server_info)]
    lib.pr_server_destroy.restype = ctypes.c_int
    lib.pr_server_destroy.argtypes = [vp]
    lib.pr_get_trace.restype = ctypes.c_int
    lib.pr_get_trace.argtypes = [vp, i32, vp, vp, vp, vp, ctypes.POINTER(i32)]
    lib.pr_kernel_launches.restype = ctypes.c_uint64
    lib.pr_kernel_launches.argtypes = []
    lib.pr_inject_alloc_failure.restype = None
    lib.pr_inject_alloc_failure.argtypes = [i32]
    lib.pr_last_error.restype = ctypes.c_char_p
    lib.pr_last_error.argtypes = [vp]
    lib.pr_status_string.restype = ctypes.c_char_p
    lib.pr_status_string.argtypes = [ctypes.c_int]
    _lib = lib
    return lib


def _status_name(status: int) -> str:
    try:
        return load().pr_status_string(status).decode()
    except OSError:
        return str(status)


def _check(status: int, handle=None):
    if status != PR_OK:
        msg = load().pr_last_error(handle)
        raise PrdfError(status, msg.decode() if msg else "")


def _ptr(a):
    """Raw pointer and length of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None, 0
    if hasattr(a, "data_ptr"):  # torch tensor
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), int(a.numel())
    if not isinstance(a, np.ndarray) or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous numpy array or a torch tensor")
    return a.ctypes.data, int(a.size)


def _u32(a):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


def pr_params_default() -> pr_params:
    p = pr_params()
    load().pr_params_default(ctypes.byref(p))
    return p


def pr_graph_create(n: int, src, dst, params: pr_params | None = None, stream: int | None = None) -> int:
    """Returns the opaque handle (an int)."""
    src, dst = _u32(src), _u32(dst)
    ps, ms = _ptr(src)
    pd, md = _ptr(dst)
    if ms != md:
        raise ValueError("src and dst differ in length")
    h = ctypes.c_void_p()
    st = load().pr_graph_create(n, ms, ps, pd, ctypes.byref(params) if params is not None else None,
                                stream, ctypes.byref(h))
    _check(st, None)
    return h.value


def pr_graph_create_batched(comp_n, src, dst, params: pr_params | None = None, stream: int | None = None) -> int:
    """Batched handle of len(comp_n) graphs; src/dst use global ids (graph c owns
    [sum(comp_n[:c]), sum(comp_n[:c+1])))."""
    cn = np.ascontiguousarray(np.asarray(comp_n, dtype=np.uint32))
    src, dst = _u32(src), _u32(dst)
    ps, ms = _ptr(src)
    pd, md = _ptr(dst)
    if ms != md:
        raise ValueError("src and dst differ in length")
    h = ctypes.c_void_p()
    st = load().pr_graph_create_batched(cn.shape[0], cn.ctypes.data, ms, ps, pd,
                                        ctypes.byref(params) if params is not None else None, stream,
                                        ctypes.byref(h))
    _check(st, None)
    return h.value


def pr_get_component_stats(h: int, ncomp: int):
    arr = (pr_stats * ncomp)()
    _check(load().pr_get_component_stats(h, arr, ncomp), h)
    return [arr[i] for i in range(ncomp)]


def pr_set_tuning(h: int, bin_lo: int, bin_hi: int, dense_div: int, blocks_per_sm: int, df_split: int = 1,
                  barrier_us: int = 0, chunk_len: int = 512, group_max: int = 64) -> None:
    t = pr_tuning(bin_lo, bin_hi, dense_div, blocks_per_sm, df_split, barrier_us, chunk_len, group_max, 0.0)
    _check(load().pr_set_tuning(h, ctypes.byref(t)), h)


def pr_get_tuning(h: int) -> pr_tuning:
    t = pr_tuning()
    _check(load().pr_get_tuning(h, ctypes.byref(t)), h)
    return t


def pr_autotune(h: int, sweep_iters: int = 8) -> pr_tuning:
    t = pr_tuning()
    _check(load().pr_autotune(h, sweep_iters, ctypes.byref(t)), h)
    return t


def pr_set_graph_launch(h: int, enable: bool) -> None:
    _check(load().pr_set_graph_launch(h, 1 if enable else 0), h)


def pr_graph_destroy(h: int) -> None:
    _check(load().pr_graph_destroy(h), None)


def pr_apply_batch(h: int, del_src, del_dst, ins_src, ins_dst) -> None:
    del_src, del_dst, ins_src, ins_dst = _u32(del_src), _u32(del_dst), _u32(ins_src), _u32(ins_dst)
    a, na = _ptr(del_src)
    b, nb = _ptr(del_dst)
    c, nc = _ptr(ins_src)
    d, nd = _ptr(ins_dst)
    if na != nb or nc != nd:
        raise ValueError("source and target arrays differ in length")
    _check(load().pr_apply_batch(h, na, a, b, nc, c, d), h)


def pr_apply_batches(h: int, batches) -> None:
    """batches: a sequence of (del_src, del_dst, ins_src, ins_dst) host arrays, applied in
    order by one library call."""
    parts = [[], [], [], []]
    doff, ioff = [0], [0]
    for bt in batches:
        arrs = [np.asarray(x, dtype=np.uint32).ravel() for x in bt]
        if arrs[0].size != arrs[1].size or arrs[2].size != arrs[3].size:
            raise ValueError("source and target arrays differ in length")
        for k in range(4):
            parts[k].append(arrs[k])
        doff.append(doff[-1] + arrs[0].size)
        ioff.append(ioff[-1] + arrs[2].size)
    if not doff[1:]:
        return
    cat = [np.ascontiguousarray(np.concatenate(p) if p else np.zeros(0, np.uint32), dtype=np.uint32) for p in parts]
    do = np.asarray(doff, dtype=np.int64)
    io = np.asarray(ioff, dtype=np.int64)
    _check(load().pr_apply_batches(h, len(doff) - 1, do.ctypes.data, cat[0].ctypes.data, cat[1].ctypes.data,
                                   io.ctypes.data, cat[2].ctypes.data, cat[3].ctypes.data), h)


def pr_static_noalloc(n: int, in_off, in_col, ranks, params: pr_params | None = None,
                      stream: int | None = None) -> pr_stats:
    """Allocation-free Static PageRank of an in-edge CSR held in device memory (torch
    tensors: in_off int64 [n + 1], in_col int32 [m], ranks float64 [n], all on the current
    device); the library allocates no device memory for it."""
    s = pr_stats()
    st = load().pr_static_noalloc(n, int(in_col.numel()), in_off.data_ptr(), in_col.data_ptr(),
                                  ctypes.byref(params) if params is not None else None, stream,
                                  ranks.data_ptr(), ctypes.byref(s))
    if st != PR_OK:
        raise PrdfError(st, load().pr_status_string(st).decode())
    return s


def _rank(fn, h: int) -> pr_stats:
    s = pr_stats()
    _check(fn(h, ctypes.byref(s)), h)
    return s


def pr_static(h: int) -> pr_stats:
    return _rank(load().pr_static, h)


def pr_naive_dynamic(h: int) -> pr_stats:
    return _rank(load().pr_naive_dynamic, h)


def pr_dynamic_frontier(h: int) -> pr_stats:
    return _rank(load().pr_dynamic_frontier, h)


def pr_dynamic_traversal(h: int) -> pr_stats:
    return _rank(load().pr_dynamic_traversal, h)


def pr_dynamic_frontier_async(h: int) -> pr_stats:
    return _rank(load().pr_dynamic_frontier_async, h)


def pr_graph_info(h: int):
    n = ctypes.c_uint32()
    m = ctypes.c_int64()
    _check(load().pr_graph_info(h, ctypes.byref(n), ctypes.byref(m)), h)
    return n.value, m.value


def pr_get_ranks(h: int, out=None):
    """Ranks as float64; into `out` (numpy or CUDA tensor) if given, else a new numpy array."""
    n, _ = pr_graph_info(h)
    if out is None:
        out = np.empty(n, np.float64)
    p, k = _ptr(out)
    if k != n:
        raise ValueError("out must hold n values")
    _check(load().pr_get_ranks(h, p, n), h)
    return out


def pr_set_ranks(h: int, ranks) -> None:
    n, _ = pr_graph_info(h)
    if not hasattr(ranks, "data_ptr"):
        ranks = np.ascontiguousarray(np.asarray(ranks, dtype=np.float64))
    p, k = _ptr(ranks)
    if k != n:
        raise ValueError("ranks must hold n values")
    _check(load().pr_set_ranks(h, p, n), h)


def pr_get_csr(h: int, direction: int):
    """(offsets uint64[n+1], columns uint32[m]) of the out (0) or in (1) adjacency."""
    n, m = pr_graph_info(h)
    off = np.empty(n + 1, np.uint64)
    col = np.empty(max(m, 1), np.uint32)
    _check(load().pr_get_csr(h, direction, off.ctypes.data, col.ctypes.data), h)
    return off, col[:m]


def pr_get_trace(h: int) -> dict:
    """Device-clock trace of the last rank call: phase-0 ms and per-iteration ms, affected
    counts and kinds (0 lists, 1 dense reused, 2 dense compacted, 3 all vertices, 4 all items
    with stamp checks, 5 continuation of a split call)."""
    cnt = ctypes.c_int32()
    _check(load().pr_get_trace(h, 0, None, None, None, None, ctypes.byref(cnt)), h)
    k = cnt.value
    ph = ctypes.c_double()
    ms = np.zeros(max(k, 1), np.float64)
    aff = np.zeros(max(k, 1), np.int64)
    kind = np.zeros(max(k, 1), np.int32)
    _check(load().pr_get_trace(h, k, ctypes.byref(ph), ms.ctypes.data, aff.ctypes.data, kind.ctypes.data,
                               ctypes.byref(cnt)), h)
    return {"phase_ms": ph.value, "iter_ms": ms[:k], "affected": aff[:k], "kind": kind[:k]}


def pr_kernel_launches() -> int:
    """Kernels launched by libprdf.so in this process so far."""
    return int(load().pr_kernel_launches())


def pr_inject_alloc_failure(after: int) -> None:
    """Host-side fault injection: the next `after` allocations succeed, later ones fail
    (negative: off)."""
    load().pr_inject_alloc_failure(int(after))


def pr_get_affected(h: int) -> np.ndarray:
    """Vertices marked affected by the last Dynamic Frontier or Traversal call (unordered)."""
    cnt = ctypes.c_int64()
    _check(load().pr_get_affected(h, None, 0, ctypes.byref(cnt)), h)
    out = np.empty(max(cnt.value, 1), np.uint32)
    _check(load().pr_get_affected(h, out.ctypes.data, cnt.value, ctypes.byref(cnt)), h)
    return out[: cnt.value]


class Graph:
    """Owning wrapper of a handle: ``with Graph(n, src, dst) as g: g.static()``.
    ``Graph.batched(comp_n, src, dst)`` builds a batched handle."""

    def __init__(self, n: int, src, dst, params: pr_params | None = None, stream: int | None = None,
                 _handle: int | None = None):
        self.h = _handle if _handle is not None else pr_graph_create(n, src, dst, params, stream)
        self.ncomp = 1

    @classmethod
    def batched(cls, comp_n, src, dst, params: pr_params | None = None, stream: int | None = None) -> "Graph":
        g = cls(0, None, None, _handle=pr_graph_create_batched(comp_n, src, dst, params, stream))
        g.ncomp = len(comp_n)
        return g

    def component_stats(self):
        return pr_get_component_stats(self.h, self.ncomp)

    def autotune(self, sweep_iters: int = 8) -> pr_tuning:
        return pr_autotune(self.h, sweep_iters)

    def tuning(self) -> pr_tuning:
        return pr_get_tuning(self.h)

    def set_tuning(self, bin_lo: int, bin_hi: int, dense_div: int, blocks_per_sm: int, df_split: int = 1,
                   barrier_us: int = 0, chunk_len: int = 512, group_max: int = 64):
        pr_set_tuning(self.h, bin_lo, bin_hi, dense_div, blocks_per_sm, df_split, barrier_us, chunk_len, group_max)

    def set_graph_launch(self, enable: bool):
        pr_set_graph_launch(self.h, enable)

    def apply(self, del_src, del_dst, ins_src, ins_dst):
        pr_apply_batch(self.h, del_src, del_dst, ins_src, ins_dst)

    def apply_batches(self, batches):
        pr_apply_batches(self.h, batches)

    def static(self) -> pr_stats:
        return pr_static(self.h)

    def naive(self) -> pr_stats:
        return pr_naive_dynamic(self.h)

    def frontier(self) -> pr_stats:
        return pr_dynamic_frontier(self.h)

    def traversal(self) -> pr_stats:
        return pr_dynamic_traversal(self.h)

    def frontier_async(self) -> pr_stats:
        return pr_dynamic_frontier_async(self.h)

    def ranks(self, out=None):
        return pr_get_ranks(self.h, out)

    def set_ranks(self, r):
        pr_set_ranks(self.h, r)

    def csr(self, direction: int):
        return pr_get_csr(self.h, direction)

    def affected(self):
        return pr_get_affected(self.h)

    def trace(self):
        return pr_get_trace(self.h)

    def info(self):
        return pr_graph_info(self.h)

    def close(self):
        if getattr(self, "h", None):
            pr_graph_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pr_server_config_default() -> pr_server_config:
    c = pr_server_config()
    load().pr_server_config_default(ctypes.byref(c))
    return c


class Server:
    """Serving form: ``srv = Server(slots=2); gi = srv.add(graph); t = srv.submit(gi, batch...)``.
    Attached graphs must outlive the server and are not used directly while attached."""

    def __init__(self, slots: int = 2, max_coalesce: int = 256, hbm_reserve_bytes: int = 1 << 30):
        c = pr_server_config(slots, max_coalesce, hbm_reserve_bytes)
        h = ctypes.c_void_p()
        _check(load().pr_server_create(ctypes.byref(c), ctypes.byref(h)), None)
        self.h = h.value

    def add(self, graph: "Graph") -> int:
        idx = ctypes.c_int32()
        _check(load().pr_server_add_graph(self.h, graph.h, ctypes.byref(idx)), None)
        return idx.value

    def submit(self, gi: int, del_src, del_dst, ins_src, ins_dst) -> int:
        del_src, del_dst, ins_src, ins_dst = _u32(del_src), _u32(del_dst), _u32(ins_src), _u32(ins_dst)
        a, na = _ptr(del_src)
        b, nb = _ptr(del_dst)
        c, nc = _ptr(ins_src)
        d, nd = _ptr(ins_dst)
        if na != nb or nc != nd:
            raise ValueError("source and target arrays differ in length")
        t = ctypes.c_uint64()
        _check(load().pr_server_submit(self.h, gi, na, a, b, nc, c, d, ctypes.byref(t)), None)
        return t.value

    def wait(self, ticket: int) -> pr_request_result:
        r = pr_request_result()
        _check(load().pr_server_wait(self.h, ticket, ctypes.byref(r)), None)
        return r

    def drain(self) -> pr_server_info:
        info = pr_server_info()
        _check(load().pr_server_drain(self.h, ctypes.byref(info)), None)
        return info

    def close(self):
        if getattr(self, "h", None):
            load().pr_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
