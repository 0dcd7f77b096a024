#!/usr/bin/env python3
"""Dynamic Frontier PageRank benchmark on one GB300 (or N replicas, one per GPU).

Workload: directed R-MAT scale 22, edge factor 16 (a, b, c, d = 0.57, 0.19, 0.19,
0.05, duplicates removed, self-loops added), 64-bit ranks, and a batch-size sweep of
uniformly random 80/20 insertion/deletion batches of 1e-7 ... 1e-3 |E| (Section 5.1.4).

One step = for every batch size f: apply one batch to the device-resident graph, bring
the ranks up to date with Dynamic Frontier (the measured update), then recompute the
same snapshot with Naive-dynamic (from the previous ranks) and Static (from 1/n) as the
paper's comparators (Section 5.2), then continue the chain from the DF ranks.

value = geometric mean over f of the mean DF update time (CUDA events on the library's
stream around the rank computation: marking, iterations and convergence detection, as
timed in Section 5.1.5; graph update excluded and reported as apply_ms).  e2e = the same
per update measured on the host around the public C-ABI calls with pinned host buffers:
pr_apply_batch (host batch -> device), pr_dynamic_frontier, pr_get_ranks (all n ranks
device -> host).  L2 is flushed (256 MB write) before every timed call.

The default run adds, after the timed region: the FP32 chain; the oracle (FP64, Algorithm
1) timed on all host cores and on one core (cpu_baseline), with the GPU replaying its
updates from its own previous ranks (parity: L-inf per f, 64-bit and FP32); the serving
form at the configured and at a lower offered rate; the batched form; the precision form
(config 3) against the oracle.  --no-legs keeps the headline, FP32 chain and parity only.

--impl reference times the oracle (FP64, Algorithm 1, synchronous) on the host cores on
the same workload, one update per step.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DF update ms & processed-edge GB/s vs GPU Static/Naive; serving p50/p99 ms"
FRACS = [1e-7, 1e-6, 1e-5, 1e-4, 1e-3]
FALLBACK_HBM_GBS = 6800.0


def geomean(xs):
    xs = [x for x in xs if x > 0]
    return math.exp(sum(math.log(x) for x in xs) / len(xs)) if xs else None


def source_digest(names) -> str:
    """sha256 of the kernel sources with comments and blank space removed (a capture stays
    valid across comment edits, not across code changes)."""
    import hashlib
    import re

    h = hashlib.sha256()
    for name in names:
        text = open(os.path.join(ROOT, "paper_2401_03256_gb300", "csrc", name)).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------------ clocks ----

class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, name in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# ------------------------------------------------------------ CPU baseline ----
# The oracle (plain FP64 C of Algorithm 1) runs in spawned processes while the GPU works:
# first its -fopenmp build on every host core (the timed CPU baseline, and the expected
# values of the parity leg), then, side by side, its sequential build on one core (a
# one-update sample) and the expected values of the precision form on the other cores.

PREC_FRACS = [1e-5, 1e-3]


def precision_shapes(rank: int):
    """Config 3's graphs: (name, generator) pairs."""
    import synth

    return [("kronecker s24 ef16", lambda: synth.rmat(24, 16, seed=11 + rank)),
            ("grid 4900x4900 + 1% long-range", lambda: synth.grid(4900, 4900, 0.01, seed=12 + rank))]


def _oracle_part(kind, scale, ef, seed, fracs, rank, cores, tmpdir, q):
    """One oracle job in its own process (the build, sequential or threaded, is per process)."""
    import numpy as np

    import oracle
    import synth

    try:
        threads = oracle.use_threads(cores)
        if kind == "headline":
            t0 = time.perf_counter()
            g = synth.rmat(scale, ef, seed=seed)
            G = oracle.Graph.build(g.n, g.src, g.dst)
            t1 = time.perf_counter()
            R, st = oracle.static_pr(G)
            static_ms = (time.perf_counter() - t1) * 1e3
            np.save(os.path.join(tmpdir, "R_static.npy"), R)
            s = synth.BatchStream(g, seed=seed)
            per, its, aff = {}, {}, {}
            for k, f in enumerate(fracs):
                b = s.next(f)
                H, ed, ei = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
                t = time.perf_counter()
                Rn, a, st = oracle.df_sync(G, H, ed, ei, R)
                per[f] = (time.perf_counter() - t) * 1e3
                its[f] = st.iterations
                np.save(os.path.join(tmpdir, f"R_df_{k}.npy"), Rn)
                np.save(os.path.join(tmpdir, f"aff_{k}.npy"), np.flatnonzero(a).astype(np.uint32))
                aff[f] = int(a.sum())
                G.close()
                G, R = H, Rn
            q.put(("headline", {"per_frac_ms": per, "iterations": its, "affected": aff, "static_ms": static_ms,
                                "setup_s": t1 - t0, "threads": threads}))
        elif kind == "sequential":
            g = synth.rmat(scale, ef, seed=seed)
            G = oracle.Graph.build(g.n, g.src, g.dst)
            R = np.load(os.path.join(tmpdir, "R_static.npy"))
            b = synth.BatchStream(g, seed=seed).next(fracs[0])
            H, ed, ei = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            t = time.perf_counter()
            oracle.df_sync(G, H, ed, ei, R)
            q.put(("sequential", {"f": fracs[0], "ms": (time.perf_counter() - t) * 1e3, "threads": threads}))
        elif kind == "precision":
            out = {}
            for si, (name, make) in enumerate(precision_shapes(rank)):
                g = make()
                G = oracle.Graph.build(g.n, g.src, g.dst)
                del g
                R, _ = oracle.static_pr(G)
                np.save(os.path.join(tmpdir, f"p{si}_static.npy"), R)
                g = make()
                s = synth.BatchStream(g, seed=13 + rank)
                del g
                its = {}
                for k, f in enumerate(PREC_FRACS):
                    b = s.next(f)
                    H, ed, ei = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
                    Rn, _, st = oracle.df_sync(G, H, ed, ei, R)
                    its[f] = st.iterations
                    np.save(os.path.join(tmpdir, f"p{si}_df_{k}.npy"), Rn)
                    G.close()
                    G, R = H, Rn
                G.close()
                out[name] = {"iterations": its}
            q.put(("precision", {"shapes": out, "threads": threads}))
    except Exception as e:  # reported, not fatal
        q.put((kind, {"error": repr(e)}))


def _oracle_chain(scale, ef, seed, fracs, rank, jobs, tmpdir, q):
    """The threaded headline job on every core, then the sequential sample on one core
    beside the precision job on the rest (jobs: which of the three to run)."""
    ctx = mp.get_context("spawn")
    import oracle

    cores = oracle.host_cores()
    if "headline" in jobs:
        pa = ctx.Process(target=_oracle_part, args=("headline", scale, ef, seed, fracs, rank, cores, tmpdir, q))
        pa.start()
        pa.join()
    both = "sequential" in jobs and "precision" in jobs
    procs = []
    if "sequential" in jobs:
        procs.append(ctx.Process(target=_oracle_part, args=("sequential", scale, ef, seed, fracs, rank, 1, tmpdir, q)))
    if "precision" in jobs:
        procs.append(ctx.Process(target=_oracle_part, args=("precision", scale, ef, seed, fracs, rank,
                                                             max(1, cores - 1) if both else cores, tmpdir, q)))
    for j in procs:
        j.start()
    for j in procs:
        j.join()
    q.put(("done", None))


def start_oracle(args, rank, jobs):
    """Spawns the oracle chain (before the first GPU call); returns its results handle."""
    ctx = mp.get_context("spawn")
    tmpdir = tempfile.mkdtemp(prefix="prdf_oracle_")
    q = ctx.Queue()
    proc = ctx.Process(target=_oracle_chain, args=(args.scale, args.ef, 1, FRACS, rank, jobs, tmpdir, q))
    proc.start()
    return OracleResults(q, proc, tmpdir)


class OracleResults:
    """Messages of the oracle chain, collected as they arrive."""

    def __init__(self, q, proc, tmpdir):
        self.q, self.proc, self.dir, self.res = q, proc, tmpdir, {}

    def wait(self, kind, timeout):
        t_end = time.time() + timeout
        while kind not in self.res and "done" not in self.res:
            try:
                k, v = self.q.get(timeout=max(0.1, t_end - time.time()))
            except Exception:
                break
            self.res[k] = v
        return self.res.get(kind)

    def close(self):
        import shutil

        if self.proc is not None:
            self.proc.join(timeout=5)
            if self.proc.is_alive():
                self.proc.terminate()
        shutil.rmtree(self.dir, ignore_errors=True)


# --------------------------------------------------------- multi-GPU runs ----
# Replicas only: every rank updates its own copy of the workload (seed 1 + rank) with no
# data-path exchange; the ranks meet only at the barriers around the timed region and in
# this reduction of the timings.

def replica_seed(rank: int) -> int:
    return 1 + rank


def max_over_ranks(values, device):
    """The job's figure for each time-like value: the slowest rank's."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


# ------------------------------------------------------------- legs ----
# Each leg returns a dict for the default line (and serves its --config run).

def _leg(fn, *a, **kw):
    """A leg of the default run; a failure is reported in its key, not fatal to the line."""
    try:
        return fn(*a, **kw)
    except Exception as e:
        import traceback

        traceback.print_exc()
        return {"error": repr(e)}


def parity_leg(args, g, dev, stream, res, tmpdir):
    """The oracle's chain of updates replayed on the GPU from the oracle's own previous
    ranks (64-bit and FP32 handles): L-inf of the ranks and the affected-set difference per
    f, after Static from 1/n."""
    import numpy as np
    import torch

    import synth
    from paper_2401_03256_gb300 import prdf

    out = {"linf_vs_oracle": {}, "fp32_linf_vs_oracle": {}, "affected_symdiff": {}, "affected_oracle": {},
           "iterations": {}, "iterations_oracle": {}}
    R0 = np.load(os.path.join(tmpdir, "R_static.npy"))
    p32 = prdf.pr_params_default()
    p32.precision = prdf.PR_F32
    with torch.cuda.stream(stream):
        A = prdf.Graph(g.n, g.src, g.dst, None, stream.cuda_stream)
        F = prdf.Graph(g.n, g.src, g.dst, p32, stream.cuda_stream)
        A.static()
        F.static()
        out["static_linf_vs_oracle"] = float(np.max(np.abs(A.ranks() - R0)))
        out["fp32_static_linf_vs_oracle"] = float(np.max(np.abs(F.ranks() - R0)))
        s = synth.BatchStream(g, seed=1)
        R_prev = R0
        for k, f in enumerate(FRACS):
            b = s.next(f)
            R_df = np.load(os.path.join(tmpdir, f"R_df_{k}.npy"))
            aff = np.load(os.path.join(tmpdir, f"aff_{k}.npy")).astype(np.int64)
            for h in (A, F):
                h.set_ranks(R_prev)
                h.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
            st = A.frontier()
            F.frontier()
            key = f"{f:g}"
            out["linf_vs_oracle"][key] = float(np.max(np.abs(A.ranks() - R_df)))
            out["fp32_linf_vs_oracle"][key] = float(np.max(np.abs(F.ranks() - R_df)))
            out["affected_symdiff"][key] = int(np.setxor1d(A.affected().astype(np.int64), aff).shape[0])
            out["affected_oracle"][key] = int(aff.shape[0])
            out["iterations"][key] = st.iterations
            out["iterations_oracle"][key] = res["iterations"][f]
            R_prev = R_df
        A.close()
        F.close()
    out["bound"] = {"fp64_mode": 1e-9, "fp32": 1e-6}
    return out


def serving_leg(args, dev, g22, rank, rates, duration=None, gcache=None):
    """Serving form (config 5): 8 resident R-MAT graphs (scales 18, 18, 19, 20, 21, 22, 23,
    24, edge factor 16, FP32 ranks), Poisson arrivals, target graph uniform, batch f ~
    log-uniform [1e-7, 1e-3] of that graph's edges (80/20), admission by slots and free
    HBM, continuous batching of each graph's queue.  One run per offered rate: the
    configured rate (queueing once the largest graphs saturate) and a rate below it, where
    latency is service time."""
    import numpy as np
    import torch

    import synth
    from paper_2401_03256_gb300 import prdf

    duration = duration or args.serve_duration
    scales = [int(x) for x in args.serve_scales.split(",")]
    gcache = {} if gcache is None else gcache

    def make(i, s):
        if s == 22 and g22 is not None and g22.n == 1 << 22:
            return g22  # the headline graph
        if s == 24:  # the precision form's Kronecker graph, generated once for both
            if "kron24" not in gcache:
                gcache["kron24"] = precision_shapes(rank)[0][1]()
            return gcache["kron24"]
        return synth.rmat(s, 16, seed=500 + 10 * rank + i)

    gs = [make(i, s) for i, s in enumerate(scales)]
    params = prdf.pr_params_default()
    params.precision = prdf.PR_F32
    streams = [torch.cuda.Stream(device=dev) for _ in gs]
    hs = [prdf.Graph(g.n, g.src, g.dst, params, st.cuda_stream) for g, st in zip(gs, streams)]
    for h in hs:
        h.static()
    out = {"config": {"graphs": [f"R-MAT s{s} ef16" for s in scales], "slots": args.slots,
                      "max_coalesce": args.coalesce, "precision": "fp32", "duration_s": duration,
                      "batch": "f ~ logU[1e-7, 1e-3] of the target graph's edges, 80/20"}}
    for ri, rate in enumerate(rates):
        rng = np.random.default_rng(1 + rank + 7 * ri)
        bstreams = [synth.BatchStream(g, seed=900 + 31 * ri + i) for i, g in enumerate(gs)]
        nreq = max(1, int(rate * duration))
        warm = 2 * len(gs)
        targets = rng.integers(0, len(gs), nreq + warm)
        fr = np.exp(rng.uniform(np.log(1e-7), np.log(1e-3), nreq + warm))
        batches = [bstreams[t].next(float(f), apply=False) for t, f in zip(targets, fr)]
        gaps = rng.exponential(1.0 / rate, nreq)
        srv = prdf.Server(slots=args.slots, max_coalesce=args.coalesce, hbm_reserve_bytes=1 << 30)
        idx = [srv.add(h) for h in hs]
        for k in range(warm):
            b = batches[k]
            srv.submit(idx[targets[k]], b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        srv.drain()
        tickets = []
        t0 = time.perf_counter()
        due = t0
        for k in range(nreq):
            due += gaps[k]
            while True:
                now = time.perf_counter()
                if now >= due:
                    break
                if due - now > 2e-4:
                    time.sleep((due - now) * 0.5)
            b = batches[warm + k]
            tickets.append(srv.submit(idx[targets[warm + k]], b.del_src, b.del_dst, b.ins_src, b.ins_dst))
        info = srv.drain()
        res = [srv.wait(t) for t in tickets]
        srv.close()
        lat = np.array([r.t_done_ms - r.t_submit_ms for r in res])
        svc = np.array([r.t_done_ms - r.t_start_ms for r in res])
        span_ms = max(r.t_done_ms for r in res) - min(r.t_submit_ms for r in res)
        out[f"rate_{rate:g}"] = {
            "offered_per_s": rate, "requests": nreq, "ok": sum(1 for r in res if r.status == prdf.PR_OK),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "service_p50_ms": float(np.percentile(svc, 50)), "service_p99_ms": float(np.percentile(svc, 99)),
            "updates_per_s": nreq / (span_ms * 1e-3), "coalesced_mean": float(np.mean([r.coalesced for r in res])),
            "waited_for_memory": info.waited_for_memory}
    for h in hs:
        h.close()
    first = out[f"rate_{rates[0]:g}"]
    out["p50_ms"], out["p99_ms"], out["updates_per_s"] = first["p50_ms"], first["p99_ms"], first["updates_per_s"]
    return out


def batched_leg(args, dev, rank, W=1, K=2, graphs=None):
    """Batched form (config 4): 256 independent R-MAT graphs (scales uniform in 10..18, edge
    factor 8), each with its own 80/20 batch of f ~ log-uniform [1e-4, 1e-2] of its edges;
    one pr_apply_batch for all graphs and one Dynamic Frontier launch (CUDA-graph replay,
    autotuned bins), FP32 ranks; against the same updates through standalone handles called
    one after another."""
    import numpy as np
    import torch

    import synth
    from paper_2401_03256_gb300 import prdf

    rng = np.random.default_rng(1 + rank)
    Gn = graphs or args.graphs
    scales = rng.integers(10, 19, Gn)
    gs = [synth.rmat(int(s), 8, seed=1000 * (1 + rank) + i) for i, s in enumerate(scales)]
    fr = np.exp(rng.uniform(np.log(1e-4), np.log(1e-2), Gn))
    firsts = np.cumsum([0] + [g.n for g in gs])
    src = np.concatenate([g.src.astype(np.uint64) + firsts[i] for i, g in enumerate(gs)]).astype(np.uint32)
    dst = np.concatenate([g.dst.astype(np.uint64) + firsts[i] for i, g in enumerate(gs)]).astype(np.uint32)
    params = prdf.pr_params_default()
    params.precision = prdf.PR_F32 if args.precision != "fp64" or args.config == "plain" else prdf.PR_F64
    streams = [synth.BatchStream(g, seed=77 + i) for i, g in enumerate(gs)]
    steps = []
    for _ in range(W + K):
        bs = [s.next(float(fr[i])) for i, s in enumerate(streams)]
        off = lambda a, i: (a.astype(np.uint64) + firsts[i]).astype(np.uint32)
        comb = [np.concatenate([off(getattr(b, k), i) for i, b in enumerate(bs)])
                for k in ("del_src", "del_dst", "ins_src", "ins_dst")]
        steps.append((bs, comb))
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        B = prdf.Graph.batched([g.n for g in gs], src, dst, params, stream.cuda_stream)
        tune = B.autotune(6)
        B.set_graph_launch(True)
        B.static()
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
        times, dfms, apms, iters = [], [], [], []
        l0 = None
        for i in range(W + K):
            if i == W:
                torch.cuda.synchronize(dev)
                l0 = prdf.pr_kernel_launches()
            flush.zero_()
            torch.cuda.synchronize(dev)
            t = time.perf_counter()
            B.apply(*steps[i][1])
            st = B.frontier()
            torch.cuda.synchronize(dev)
            if i >= W:
                times.append((time.perf_counter() - t) * 1e3)
                dfms.append(st.ms_rank)
                apms.append(st.ms_apply)
                iters.append(max(c.iterations for c in B.component_stats()))
        launches = prdf.pr_kernel_launches() - l0
        B.close()
        As = [prdf.Graph(g.n, g.src, g.dst, params, stream.cuda_stream) for g in gs]
        for A in As:
            A.static()
        seq = []
        for i in range(W + K):
            flush.zero_()
            torch.cuda.synchronize(dev)
            t = time.perf_counter()
            for j, A in enumerate(As):
                b = steps[i][0][j]
                A.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
                A.frontier()
            torch.cuda.synchronize(dev)
            if i >= W:
                seq.append((time.perf_counter() - t) * 1e3)
        for A in As:
            A.close()
    value = statistics.median(times)
    return {"ms": value, "df_ms": statistics.median(dfms), "apply_ms": statistics.median(apms),
            "sequential_ms": statistics.median(seq), "speedup_vs_sequential": statistics.median(seq) / value,
            "max_graph_iterations": max(iters), "gpu_launches": launches, "steps": K, "warmup": W,
            "config": {"workload": f"{Gn} R-MAT graphs, scales U{{10..18}}, edge factor 8, own 80/20 batch of "
                                   f"f ~ logU[1e-4, 1e-2] each", "vertices": int(firsts[-1]), "edges": int(src.size),
                       "precision": "fp32" if params.precision == prdf.PR_F32 else "fp64",
                       "launch": "CUDA graph replay", "tuning": tune.as_dict()}}


def precision_leg(args, dev, rank, orc=None, gcache=None):
    """Precision form (config 3): FP32 ranks and contributions (FP64 compensated dead-end
    mass) on a Kronecker scale-24 graph (edge factor 16) and on a 4900 x 4900 directed grid
    with 1% random long-range arcs; one 80/20 batch of 1e-5 |E|, then one of 1e-3 |E|,
    chained.  Every update starts from the oracle's previous ranks (when the oracle ran) in
    an FP32 and a 64-bit handle; errors are L-inf against the oracle's result."""
    import numpy as np
    import torch

    import synth
    from paper_2401_03256_gb300 import prdf

    ores = orc.wait("precision", args.cpu_timeout) if orc is not None else None
    have = bool(ores) and "shapes" in ores
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    out = {"error_reference": "FP64 oracle (Algorithm 1), same previous ranks" if have else "64-bit path",
           "oracle_note": None if have else (ores or {}).get("error", "oracle not run")}
    gcache = {} if gcache is None else gcache
    for si, (name, make) in enumerate(precision_shapes(rank)):
        g = gcache.pop("kron24", None) if si == 0 else None
        g = g if g is not None else make()
        p32 = prdf.pr_params_default()
        p32.precision = prdf.PR_F32
        with torch.cuda.stream(stream):
            A = prdf.Graph(g.n, g.src, g.dst, p32, stream.cuda_stream)
            B = prdf.Graph(g.n, g.src, g.dst, None, stream.cuda_stream)
            n, m = A.info()
            st32 = A.static()
            st64 = B.static()
            R32, R64 = A.ranks(), B.ranks()
            entry = {"n": n, "m_with_self_loops": m, "static_fp32_ms": st32.ms_rank, "static_fp64_ms": st64.ms_rank,
                     "per_frac": {}}
            if have:
                R0 = np.load(os.path.join(orc.dir, f"p{si}_static.npy"))
                entry["static_fp32_linf_vs_oracle"] = float(np.max(np.abs(R32 - R0)))
                entry["static_fp64_linf_vs_oracle"] = float(np.max(np.abs(R64 - R0)))
                R_prev = R0
            else:
                entry["static_fp32_linf_vs_fp64"] = float(np.max(np.abs(R32 - R64)))
                R_prev = R64
            s = synth.BatchStream(g, seed=13 + rank)
            for k, f in enumerate(PREC_FRACS):
                b = s.next(f)
                for h in (A, B):
                    h.set_ranks(R_prev)
                    h.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
                flush.zero_()
                s32 = A.frontier()
                flush.zero_()
                s64 = B.frontier()
                r32, r64 = A.ranks(), B.ranks()
                ref = np.load(os.path.join(orc.dir, f"p{si}_df_{k}.npy")) if have else r64
                A.set_ranks(R_prev)
                flush.zero_()
                sn = A.naive()
                flush.zero_()
                ss = A.static()
                e = {"df_fp32_ms": s32.ms_rank, "df_fp64_ms": s64.ms_rank, "naive_fp32_ms": sn.ms_rank,
                     "static_fp32_ms": ss.ms_rank, "speedup_vs_naive": sn.ms_rank / s32.ms_rank,
                     "speedup_vs_static": ss.ms_rank / s32.ms_rank, "df_fp32_iterations": s32.iterations,
                     "df_fp64_iterations": s64.iterations, "df_affected": s32.affected_final,
                     "fp32_linf": float(np.max(np.abs(r32 - ref)))}
                if have:
                    e["fp64_linf_vs_oracle"] = float(np.max(np.abs(r64 - ref)))
                    e["oracle_iterations"] = ores["shapes"][name]["iterations"][f]
                entry["per_frac"][f"{f:g}"] = e
                R_prev = ref
            A.close()
            B.close()
        out[name] = entry
        del g
    return out


# ------------------------------------------------------------- GPU arm ----

def run_ours(args, rank: int, world: int, local_rank: int):
    orc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # started before the first GPU call; the oracle runs on the host cores while the
        # GPU works (its expected values feed the parity and precision legs)
        orc = start_oracle(args, rank, ["headline", "sequential"] + ([] if args.no_legs else ["precision"]))

    import numpy as np
    import torch

    import synth
    from paper_2401_03256_gb300 import build as libbuild

    libbuild.build()
    from paper_2401_03256_gb300 import prdf

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    seed = replica_seed(rank)
    g = synth.rmat(args.scale, args.ef, seed=seed)
    params = prdf.pr_params_default()
    params.precision = prdf.PR_F32 if args.precision == "fp32" else prdf.PR_F64
    stream = torch.cuda.Stream(device=dev)
    W, K = args.warmup, args.steps
    with torch.cuda.stream(stream):
        G = prdf.Graph(g.n, g.src, g.dst, params, stream.cuda_stream)
        n, m = G.info()
        G.static()
        # Dynamic Traversal and asynchronous DF consume pending marks too: each runs on a
        # handle of its own that receives the same batches and starts from the same ranks
        G_dt = prdf.Graph(g.n, g.src, g.dst, params, stream.cuda_stream)
        G_as = prdf.Graph(g.n, g.src, g.dst, params, stream.cuda_stream)
        bs = synth.BatchStream(g, seed=seed)
        batches = [[bs.next(f) for f in FRACS] for _ in range(W + K)]
        e2e_batches = [[bs.next(f) for f in FRACS] for _ in range(K)]
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
        R_prev = torch.empty(n, dtype=torch.float64, device=dev)
        R_cur = torch.empty(n, dtype=torch.float64, device=dev)
        rec = {f: {"df": [], "naive": [], "static": [], "apply": [], "df_iters": [], "df_affected": [],
                   "df_bytes": [], "naive_iters": [], "static_iters": [], "static_bytes": [], "naive_bytes": [],
                   "df_edges": [], "dt": [], "dt_iters": [], "dt_affected": [], "dfa": [], "dfa_iters": []} for f in FRACS}

        def call(name, fn):
            if not args.nvtx:
                return fn()
            torch.cuda.nvtx.range_push(name)
            try:
                return fn()
            finally:
                torch.cuda.nvtx.range_pop()

        def step(i, record):
            for fi, f in enumerate(FRACS):
                b = batches[i][fi]
                G.ranks(R_prev)
                G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
                flush.zero_()
                sd = call("df", G.frontier)
                G.ranks(R_cur)
                G.set_ranks(R_prev)
                G_dt.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
                G_dt.set_ranks(R_prev)
                flush.zero_()
                st = call("dt", G_dt.traversal)
                G_as.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
                G_as.set_ranks(R_prev)
                flush.zero_()
                sa = call("df_async", G_as.frontier_async)
                flush.zero_()
                sn = call("naive", G.naive)
                flush.zero_()
                ss = call("static", G.static)
                G.set_ranks(R_cur)
                if record:
                    r = rec[f]
                    r["df"].append(sd.ms_rank)
                    r["apply"].append(sd.ms_apply)
                    r["naive"].append(sn.ms_rank)
                    r["static"].append(ss.ms_rank)
                    r["df_iters"].append(sd.iterations)
                    r["df_affected"].append(sd.affected_final)
                    r["df_bytes"].append(sd.bytes_algorithmic)
                    r["df_edges"].append(sd.edges_processed)
                    r["naive_iters"].append(sn.iterations)
                    r["static_iters"].append(ss.iterations)
                    r["static_bytes"].append(ss.bytes_algorithmic)
                    r["naive_bytes"].append(sn.bytes_algorithmic)
                    r["dt"].append(st.ms_rank)
                    r["dt_iters"].append(st.iterations)
                    r["dt_affected"].append(st.affected_final)
                    r["dfa"].append(sa.ms_rank)
                    r["dfa_iters"].append(sa.iterations)

        for i in range(W):
            step(i, False)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        clocks = ClockSampler(local_rank)
        clocks.start()
        l0 = prdf.pr_kernel_launches()
        t0 = time.perf_counter()
        for i in range(K):
            step(W + i, True)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        t1 = time.perf_counter()
        launches = prdf.pr_kernel_launches() - l0
        clk = clocks.stop()
        R_final64 = R_cur.clone()

        # the same chain of updates with FP32 ranks (untimed by the step clock; its own events)
        fp32 = None
        if args.precision == "fp64" and not args.no_fp32:
            p32 = prdf.pr_params_default()
            p32.precision = prdf.PR_F32
            G32 = prdf.Graph(g.n, g.src, g.dst, p32, stream.cuda_stream)
            G32.static()
            rec32 = {f: {"df": [], "naive": [], "static": []} for f in FRACS}
            P = torch.empty(n, dtype=torch.float64, device=dev)
            Q = torch.empty(n, dtype=torch.float64, device=dev)
            for i in range(W + K):
                for fi, f in enumerate(FRACS):
                    b = batches[i][fi]
                    G32.ranks(P)
                    G32.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
                    flush.zero_()
                    sd = G32.frontier()
                    G32.ranks(Q)
                    G32.set_ranks(P)
                    flush.zero_()
                    sn = G32.naive()
                    flush.zero_()
                    ss = G32.static()
                    G32.set_ranks(Q)
                    if i >= W:
                        rec32[f]["df"].append(sd.ms_rank)
                        rec32[f]["naive"].append(sn.ms_rank)
                        rec32[f]["static"].append(ss.ms_rank)
            G32.ranks(Q)
            err = float((Q - R_final64).abs().max())
            G32.close()
            avg = lambda xs: sum(xs) / len(xs)
            fp32 = {"value": geomean([avg(rec32[f]["df"]) for f in FRACS]), "unit": "ms",
                    "linf_vs_fp64_after_chain": err,
                    "per_frac": {f"{f:g}": {"df_ms": avg(rec32[f]["df"]), "naive_ms": avg(rec32[f]["naive"]),
                                           "static_ms": avg(rec32[f]["static"])} for f in FRACS},
                    "note": "same batches, FP32 ranks and contributions; error = L-inf between the FP32 "
                            "and FP64 chains' ranks after all updates"}

        # end to end through the C ABI with pinned host buffers
        out_h = torch.empty(n, dtype=torch.float64, pin_memory=True)
        e2e = {f: [] for f in FRACS}
        h2d = 0
        pinned = []
        for i in range(K):
            row = []
            for fi in range(len(FRACS)):
                b = e2e_batches[i][fi]
                row.append([torch.from_numpy(a.astype(np.int32)).pin_memory() for a in
                            (b.del_src, b.del_dst, b.ins_src, b.ins_dst)])
            pinned.append(row)
        for i in range(K):
            for fi, f in enumerate(FRACS):
                ds, dd, is_, id_ = pinned[i][fi]
                h2d += 4 * (ds.numel() + dd.numel() + is_.numel() + id_.numel())
                flush.zero_()
                torch.cuda.synchronize(dev)
                t = time.perf_counter()
                G.apply(ds, dd, is_, id_)
                G.frontier()
                G.ranks(out_h)
                e2e[f].append((time.perf_counter() - t) * 1e3)
        G.close()
        G_dt.close()
        G_as.close()

    def mean(xs):
        return sum(xs) / len(xs) if xs else float("nan")

    df_ms = {f: mean(rec[f]["df"]) for f in FRACS}
    value = geomean(df_ms.values())
    static_bytes = sum(sum(rec[f]["static_bytes"]) for f in FRACS)
    static_ms = sum(sum(rec[f]["static"]) for f in FRACS)
    static_launches = sum(len(rec[f]["static"]) for f in FRACS)
    all_bytes = static_bytes + sum(sum(rec[f]["naive_bytes"]) + sum(rec[f]["df_bytes"]) for f in FRACS)
    all_ms = static_ms + sum(sum(rec[f]["naive"]) + sum(rec[f]["df"]) for f in FRACS)
    peak, peak_kind = hbm_peak()
    # the Static call is one k_full_init, one full-sweep k_sweep launch per iteration and one
    # writeback, timed by CUDA events on its stream: the time per iteration bounds a sweep
    # launch's duration from above (it includes the init and writeback and the loop's node
    # switches), so `achieved` is a lower bound
    static_iters = sum(sum(rec[f]["static_iters"]) for f in FRACS)
    launch_bytes = static_bytes / static_iters
    launch_ms = static_ms / static_iters
    achieved = launch_bytes / (launch_ms * 1e-3) / 1e9
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "k_sweep_traffic.json")
    try:
        with open(tr_path) as f:
            tr = json.load(f)
        if tr.get("sources_code_sha256") == source_digest(tr.get("sources", [])) and tr.get("precision") == args.precision:
            traffic = tr.get("launch_dram_bytes_full_size")
    except Exception:
        traffic = None

    per_f = {}
    for f in FRACS:
        r = rec[f]
        per_f[f"{f:g}"] = {
            "df_ms": df_ms[f], "naive_ms": mean(r["naive"]), "static_ms": mean(r["static"]),
            "apply_ms": mean(r["apply"]), "speedup_vs_static": mean(r["static"]) / df_ms[f],
            "speedup_vs_naive": mean(r["naive"]) / df_ms[f], "df_iterations": mean(r["df_iters"]),
            "naive_iterations": mean(r["naive_iters"]), "static_iterations": mean(r["static_iters"]),
            "df_affected": mean(r["df_affected"]),
            "dt_ms": mean(r["dt"]), "dt_iterations": mean(r["dt_iters"]), "dt_affected": mean(r["dt_affected"]),
            "speedup_vs_dt": mean(r["dt"]) / df_ms[f],
            "df_async_ms": mean(r["dfa"]), "df_async_iterations": mean(r["dfa_iters"]),
            "df_gbs": (sum(r["df_bytes"]) / (sum(r["df"]) * 1e-3) / 1e9) if sum(r["df"]) > 0 else None,
            "e2e_ms": mean(e2e[f]),
        }
    e2e_value = geomean([mean(e2e[f]) for f in FRACS])
    ms_per_step = (t1 - t0) / K * 1e3

    if dist:
        value, e2e_value, ms_per_step = max_over_ranks([value, e2e_value, ms_per_step], dev)

    cpu = None
    legs = {}
    if orc is not None:
        res = orc.wait("headline", args.cpu_timeout)
        if res and "per_frac_ms" in res:
            cpu_val = geomean(res["per_frac_ms"].values())
            seq = orc.wait("sequential", args.cpu_timeout)
            cpu = {"value": cpu_val, "unit": "ms", "cores": res["threads"], "kind": "oracle",
                   "sample": (f"FP64 oracle (Algorithm 1, synchronous), its -fopenmp build with schedule(dynamic, "
                              f"2048) on {res['threads']} host cores (sched_getaffinity), one 80/20 batch per f in "
                              f"{[f'{x:g}' for x in FRACS]} on the same R-MAT s{args.scale} ef{args.ef} graph, chained "
                              f"from its own Static ranks (graph build {res['setup_s']:.0f} s and Static "
                              f"{res['static_ms'] / 1e3:.1f} s untimed)"),
                   "per_frac_ms": {f"{k:g}": v for k, v in res["per_frac_ms"].items()},
                   "iterations": {f"{k:g}": v for k, v in res["iterations"].items()}}
            if seq and "ms" in seq:
                cpu["sequential_1core"] = {"value": seq["ms"], "unit": "ms", "cores": 1, "f": seq["f"],
                                           "sample": "the sequential build of the same source, one update at this f"}
            legs["parity"] = _leg(parity_leg, args, g, dev, stream, res, orc.dir)
        else:
            cpu = {"value": None, "unit": "ms", "cores": None, "kind": "oracle",
                   "sample": (res or {}).get("error", "timed out")}
    if not args.no_legs and rank == 0:
        gcache = {}
        legs["serving"] = _leg(serving_leg, args, dev, g, rank, rates=(args.rate, args.sub_rate), gcache=gcache)
        legs["batched"] = _leg(batched_leg, args, dev, rank)
        legs["precision"] = _leg(precision_leg, args, dev, rank, orc, gcache=gcache)
        gcache.clear()
    if orc is not None:
        orc.close()

    line = {
        "metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "i64", "data": "synthetic",
        "config": {"workload": f"R-MAT scale {args.scale} edge factor {args.ef}, 80/20 batches f=1e-7..1e-3 |E|, "
                               f"Dynamic Frontier vs Static vs Naive-dynamic",
                   "n": n, "m_with_self_loops": m, "batch_fracs": FRACS,
                   "precision": args.precision, "l2": "flushed (256 MB write) before every timed call",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "e2e": {"value": e2e_value, "unit": "ms", "h2d_bytes_per_step": h2d // K,
                "d2h_bytes_per_step": 8 * n * len(FRACS)},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": "k_sweep<64-bit, full sweep> (one launch per Static iteration)",
                     "launch_bytes_algorithmic": launch_bytes, "launch_ms": launch_ms,
                     "all_rank_calls_gbs": all_bytes / (all_ms * 1e-3) / 1e9},
        "per_frac": per_f,
        "fp32": fp32,
        "speedup_vs_static_geomean": geomean([per_f[k]["speedup_vs_static"] for k in per_f]),
        "speedup_vs_naive_geomean": geomean([per_f[k]["speedup_vs_naive"] for k in per_f]),
        "clocks": clk,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    line.update(legs)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------- single-form configs ----

def _setup_device(local_rank):
    import torch

    from paper_2401_03256_gb300 import build as libbuild

    libbuild.build()
    torch.cuda.set_device(local_rank)
    return torch.device("cuda", local_rank)


def _form_line(metric, value, world, steps, warmup, dtype, config, extra, clk=None):
    line = {"metric": metric, "value": value, "unit": "ms", "n_gpus": world, "steps": steps, "warmup": warmup,
            "ms_per_step": value, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic", "config": config}
    line.update(extra)
    if clk is not None:
        line["clocks"] = clk
    return line


def run_batched(args, rank: int, world: int, local_rank: int):
    """--config batched: the batched form alone (batched_leg), K timed updates."""
    dev = _setup_device(local_rank)
    clocks = ClockSampler(local_rank)
    clocks.start()
    r = batched_leg(args, dev, rank, W=args.warmup, K=args.steps)
    clk = clocks.stop()
    line = _form_line("batched form: ms per update of all graphs (apply + Dynamic Frontier, one launch)", r["ms"],
                      world, args.steps, args.warmup, r["config"]["precision"], r.pop("config"), r, clk)
    if rank == 0:
        print(json.dumps(line))


def run_serving(args, rank: int, world: int, local_rank: int):
    """--config serving: the serving form alone (serving_leg) at --rate for --duration s."""
    dev = _setup_device(local_rank)
    clocks = ClockSampler(local_rank)
    clocks.start()
    r = serving_leg(args, dev, None, rank, rates=(args.rate,), duration=args.duration)
    clk = clocks.stop()
    line = _form_line("serving p50/p99 ms", r["p99_ms"], world, r[f"rate_{args.rate:g}"]["requests"], 0, "f32",
                      r.pop("config"), r, clk)
    if rank == 0:
        print(json.dumps(line))


def run_precision(args, rank: int, world: int, local_rank: int):
    """--config precision: the precision form alone (precision_leg), errors against the
    FP64 oracle run on the host cores meanwhile."""
    orc = start_oracle(args, rank, ["precision"]) if rank == 0 and world == 1 and not args.no_cpu_baseline else None
    dev = _setup_device(local_rank)
    clocks = ClockSampler(local_rank)
    clocks.start()
    r = precision_leg(args, dev, rank, orc)
    clk = clocks.stop()
    if orc is not None:
        orc.close()
    dfs = [e["df_fp32_ms"] for k, v in r.items() if isinstance(v, dict) and "per_frac" in v
           for e in v["per_frac"].values()]
    line = _form_line("precision form: FP32 Dynamic Frontier update ms (geomean over shapes and batch sizes)",
                      geomean(dfs), world, len(dfs), 0, "f32",
                      {"workload": "Kronecker s24 ef16 and 4900x4900 grid + 1% long-range, 80/20 batches 1e-5 then "
                                   "1e-3 |E|, FP32 ranks/contributions, FP64 compensated dead-end mass",
                       "l2": "flushed (256 MB write) before every timed call"}, {"shapes": r}, clk)
    if rank == 0:
        print(json.dumps(line))


def run_mixes(args, rank: int, world: int, local_rank: int):
    """Update mixes and frontier tolerance (Sections 5.1.3, 5.2): insertion-only,
    deletion-only and 80/20 batches of 1e-7 ... 1e-3 |E| on R-MAT (scale --scale, edge
    factor --ef) and on a 2048 x 2048 grid with 1% long-range arcs.  Static, Naive-dynamic,
    Dynamic Traversal and Dynamic Frontier (synchronous and asynchronous) each run on a
    handle of their own that receives the same batches and continues from its own ranks, as
    in the paper's runs; after every update each result's L1 distance to a reference Static
    PageRank (tau = 1e-100, 500 iterations) on the same graph is taken.  On insertion-only
    batches Dynamic Frontier also runs with tau_f = tau / 10^k, k = 0 ... 4 (k = 5 is the
    default).  value = geometric mean of the Dynamic Frontier times."""
    import torch

    import synth
    from paper_2401_03256_gb300 import build as libbuild

    libbuild.build()
    from paper_2401_03256_gb300 import prdf

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    W, K = args.warmup, args.steps
    shapes = [(f"R-MAT s{args.scale} ef{args.ef}", lambda: synth.rmat(args.scale, args.ef, seed=41 + rank)),
              ("grid 2048x2048 + 1% long-range", lambda: synth.grid(2048, 2048, 0.01, seed=42 + rank))]
    mixes = [("insert-only", 1.0), ("delete-only", 0.0), ("80/20", 0.8)]
    methods = ["static", "naive", "dt", "df", "df_async"]
    tauf_k = [0, 1, 2, 3, 4]
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    mean = lambda xs: sum(xs) / len(xs) if xs else float("nan")
    out, dfs = {}, []
    launches = 0
    clocks = ClockSampler(local_rank)
    clocks.start()
    t_start = time.perf_counter()
    for sname, make in shapes:
        g = make()
        out[sname] = {}
        for mname, share in mixes:
            with torch.cuda.stream(stream):
                pref = prdf.pr_params_default()
                pref.tol = 1e-100
                pref.max_iter = 500
                H = {m: prdf.Graph(g.n, g.src, g.dst, None, stream.cuda_stream) for m in methods}
                ref = prdf.Graph(g.n, g.src, g.dst, pref, stream.cuda_stream)
                sweep = {}
                if share == 1.0:
                    for k in tauf_k:
                        pk = prdf.pr_params_default()
                        pk.frontier_tol = pk.tol / 10 ** k
                        sweep[k] = prdf.Graph(g.n, g.src, g.dst, pk, stream.cuda_stream)
                n, m = ref.info()
                H["static"].static()
                R0 = torch.empty(n, dtype=torch.float64, device=dev)
                H["static"].ranks(R0)
                for h in list(H.values()) + list(sweep.values()):
                    h.set_ranks(R0)
                Rr = torch.empty(n, dtype=torch.float64, device=dev)
                Rm = torch.empty(n, dtype=torch.float64, device=dev)
                bs = synth.BatchStream(g, seed=43 + rank)
                rec = {f: {"ms": {x: [] for x in methods}, "err": {x: [] for x in methods},
                           "it": {x: [] for x in methods}, "aff_df": [], "aff_dt": [],
                           "sweep_ms": {k: [] for k in tauf_k}, "sweep_err": {k: [] for k in tauf_k},
                           "sweep_aff": {k: [] for k in tauf_k}} for f in FRACS}
                l0 = prdf.pr_kernel_launches()
                calls = {"static": lambda h: h.static(), "naive": lambda h: h.naive(),
                         "dt": lambda h: h.traversal(), "df": lambda h: h.frontier(),
                         "df_async": lambda h: h.frontier_async()}
                for i in range(W + K):
                    for f in FRACS:
                        b = bs.next(f, ins_share=share)
                        for h in [ref] + list(H.values()) + list(sweep.values()):
                            h.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
                        res = {}
                        for x in methods:
                            flush.zero_()
                            res[x] = calls[x](H[x])
                        sres = {}
                        for k, h in sweep.items():
                            flush.zero_()
                            sres[k] = h.frontier()
                        if i < W:
                            continue
                        ref.static()
                        ref.ranks(Rr)
                        r = rec[f]
                        for x in methods:
                            H[x].ranks(Rm)
                            r["ms"][x].append(res[x].ms_rank)
                            r["err"][x].append(float((Rm - Rr).abs().sum()))
                            r["it"][x].append(res[x].iterations)
                        r["aff_df"].append(res["df"].affected_final)
                        r["aff_dt"].append(res["dt"].affected_final)
                        for k, h in sweep.items():
                            h.ranks(Rm)
                            r["sweep_ms"][k].append(sres[k].ms_rank)
                            r["sweep_err"][k].append(float((Rm - Rr).abs().sum()))
                            r["sweep_aff"][k].append(sres[k].affected_final)
                torch.cuda.synchronize(dev)
                launches += prdf.pr_kernel_launches() - l0
                for h in [ref] + list(H.values()) + list(sweep.values()):
                    h.close()
            per = {}
            for f in FRACS:
                r = rec[f]
                per[f"{f:g}"] = {
                    **{f"{x}_ms": mean(r["ms"][x]) for x in methods},
                    **{f"{x}_l1_err": mean(r["err"][x]) for x in methods},
                    **{f"{x}_iterations": mean(r["it"][x]) for x in methods},
                    "df_affected": mean(r["aff_df"]), "dt_affected": mean(r["aff_dt"]),
                }
                dfs.append(mean(r["ms"]["df"]))
            gm = lambda x: geomean([mean(rec[f]["ms"][x]) for f in FRACS])
            entry = {"n": n, "m_with_self_loops": m, "per_frac": per,
                     "df_speedup_geomean": {x: gm(x) / gm("df") for x in methods if x != "df"}}
            if sweep:
                entry["tau_f_sweep"] = {
                    f"tau/1e{k}": {"df_ms_geomean": geomean([mean(rec[f]["sweep_ms"][k]) for f in FRACS]),
                                   "l1_err_mean": mean([mean(rec[f]["sweep_err"][k]) for f in FRACS]),
                                   "affected_mean": mean([mean(rec[f]["sweep_aff"][k]) for f in FRACS])}
                    for k in tauf_k}
                entry["tau_f_sweep"]["tau/1e5"] = {
                    "df_ms_geomean": gm("df"),
                    "l1_err_mean": mean([mean(rec[f]["err"]["df"]) for f in FRACS]),
                    "affected_mean": mean([mean(rec[f]["aff_df"]) for f in FRACS])}
                entry["static_l1_err_mean"] = mean([mean(rec[f]["err"]["static"]) for f in FRACS])
            out[sname][mname] = entry
        del g
    t_end = time.perf_counter()
    clk = clocks.stop()
    line = {
        "metric": "update mixes: Dynamic Frontier update ms (geomean over graphs, mixes and batch sizes)",
        "value": geomean(dfs), "unit": "ms", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": (t_end - t_start) * 1e3 / (K + W), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "i64", "data": "synthetic",
        "config": {"workload": f"R-MAT s{args.scale} ef{args.ef} and 2048x2048 grid + 1% long-range; "
                               "insertion-only, deletion-only and 80/20 batches 1e-7..1e-3 |E|; tau_f sweep "
                               "tau..tau/1e5 on insertion-only batches",
                   "l2": "flushed (256 MB write) before every timed call",
                   "error_reference": "Static PageRank, tau = 1e-100, 500 iterations, same graph"},
        "graphs": out, "gpu_launches": launches, "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line))


def run_kmer(args, rank: int, world: int, local_rank: int):
    """Low-degree huge graph (the protein k-mer graphs of Table 1: 171-214 M vertices,
    average degree 3.1 with self-loops): synth.kmer with --kmer-n vertices, one long
    symmetric component with local shortcuts under a random numbering.  80/20 batches of
    1e-7 ... 1e-3 |E| drawn against the original edge set (the generator's copy of the
    ~420 M edges is not re-merged on the host after every batch; an absent deletion or a
    present insertion is a no-op).  Per batch: Dynamic Frontier on the chained handle,
    then Naive-dynamic and Static from the same previous ranks, and Dynamic Traversal on
    a second handle given the same batch and ranks.  value = geometric mean of the
    Dynamic Frontier times."""
    import torch

    import synth
    from paper_2401_03256_gb300 import build as libbuild

    libbuild.build()
    from paper_2401_03256_gb300 import prdf

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    W, K = args.warmup, args.steps
    t_gen = time.perf_counter()
    g = synth.kmer(args.kmer_n, seed=51 + rank)
    t_gen = time.perf_counter() - t_gen
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    mean = lambda xs: sum(xs) / len(xs) if xs else float("nan")
    free0 = torch.cuda.mem_get_info(dev)[0]
    with torch.cuda.stream(stream):
        G = prdf.Graph(g.n, g.src, g.dst, None, stream.cuda_stream)
        torch.cuda.synchronize(dev)
        handle_bytes = free0 - torch.cuda.mem_get_info(dev)[0]
        T = prdf.Graph(g.n, g.src, g.dst, None, stream.cuda_stream)
        n, m = G.info()
        st0 = G.static()
        bs = synth.BatchStream(g, seed=53 + rank)
        batches = [[bs.next(f, apply=False) for f in FRACS] for _ in range(W + K)]
        bs.close()
        del g
        R_prev = torch.empty(n, dtype=torch.float64, device=dev)
        R_cur = torch.empty(n, dtype=torch.float64, device=dev)
        rec = {f: {x: [] for x in ("df", "naive", "static", "dt", "df_it", "dt_it", "st_it", "df_aff", "dt_aff",
                                   "apply", "df_bytes")} for f in FRACS}
        clocks = ClockSampler(local_rank)
        clocks.start()
        l0 = prdf.pr_kernel_launches()
        t0 = time.perf_counter()
        for i in range(W + K):
            for fi, f in enumerate(FRACS):
                b = batches[i][fi]
                G.ranks(R_prev)
                G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
                T.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
                flush.zero_()
                sd = G.frontier()
                G.ranks(R_cur)
                T.set_ranks(R_prev)
                flush.zero_()
                st = T.traversal()
                G.set_ranks(R_prev)
                flush.zero_()
                sn = G.naive()
                flush.zero_()
                ss = G.static()
                G.set_ranks(R_cur)
                if i >= W:
                    r = rec[f]
                    for key, val in (("df", sd.ms_rank), ("naive", sn.ms_rank), ("static", ss.ms_rank),
                                     ("dt", st.ms_rank), ("df_it", sd.iterations), ("dt_it", st.iterations),
                                     ("st_it", ss.iterations), ("df_aff", sd.affected_final),
                                     ("dt_aff", st.affected_final), ("apply", sd.ms_apply),
                                     ("df_bytes", sd.bytes_algorithmic)):
                        r[key].append(val)
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        launches = prdf.pr_kernel_launches() - l0
        clk = clocks.stop()
        G.close()
        T.close()
    per = {}
    for f in FRACS:
        r = rec[f]
        per[f"{f:g}"] = {
            "df_ms": mean(r["df"]), "naive_ms": mean(r["naive"]), "static_ms": mean(r["static"]),
            "dt_ms": mean(r["dt"]), "apply_ms": mean(r["apply"]),
            "speedup_vs_static": mean(r["static"]) / mean(r["df"]),
            "speedup_vs_naive": mean(r["naive"]) / mean(r["df"]), "speedup_vs_dt": mean(r["dt"]) / mean(r["df"]),
            "df_iterations": mean(r["df_it"]), "dt_iterations": mean(r["dt_it"]),
            "static_iterations": mean(r["st_it"]), "df_affected": mean(r["df_aff"]),
            "dt_affected": mean(r["dt_aff"]),
            "df_gbs": sum(r["df_bytes"]) / (sum(r["df"]) * 1e-3) / 1e9 if sum(r["df"]) > 0 else None,
        }
    line = {
        "metric": "k-mer stand-in: Dynamic Frontier update ms (geomean over batch sizes)",
        "value": geomean([per[f"{f:g}"]["df_ms"] for f in FRACS]), "unit": "ms", "n_gpus": world,
        "steps": K, "warmup": W, "ms_per_step": (t1 - t0) * 1e3 / (W + K), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "i64", "data": "synthetic",
        "config": {"workload": f"k-mer-like graph, {n} vertices, {m} stored edges with self-loops, "
                               "80/20 batches 1e-7..1e-3 |E|",
                   "l2": "flushed (256 MB write) before every timed call",
                   "generator_s": t_gen, "device_bytes_per_handle": handle_bytes,
                   "static_ms_first": st0.ms_rank, "static_iterations_first": st0.iterations},
        "per_frac": per, "gpu_launches": launches, "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line))


# -------------------------------------------------------- reference arm ----

def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    import oracle
    import synth

    cores = oracle.use_threads(oracle.host_cores())
    g = synth.rmat(args.scale, args.ef, seed=1)
    G = oracle.Graph.build(g.n, g.src, g.dst)
    R, _ = oracle.static_pr(G)
    s = synth.BatchStream(g, seed=1)
    W, K = args.warmup, args.steps
    times = {f: [] for f in FRACS}
    for i in range(W + K):
        f = FRACS[i % len(FRACS)]
        b = s.next(f)
        H, ed, ei = G.apply(b.del_src, b.del_dst, b.ins_src, b.ins_dst)
        t = time.perf_counter()
        R, _, st = oracle.df_sync(G, H, ed, ei, R)
        dt = (time.perf_counter() - t) * 1e3
        if i >= W:
            times[f].append(dt)
        G = H
    means = [sum(v) / len(v) for v in times.values() if v]
    value = geomean(means)
    all_t = [x for v in times.values() for x in v]
    sample = (f"FP64 oracle (Algorithm 1, synchronous), its -fopenmp build on {cores} host cores, on R-MAT "
              f"s{args.scale} ef{args.ef}; step i updates one 80/20 batch of f = FRACS[i mod 5]; {K} timed steps "
              f"after {W} warm-up steps")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": sum(all_t) / len(all_t) if all_t else None, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"R-MAT scale {args.scale} edge factor {args.ef}, 80/20 batches f=1e-7..1e-3 |E|, "
                               f"Dynamic Frontier vs Static vs Naive-dynamic", "batch_fracs": FRACS,
                   "precision": "fp64"},
        "cpu_baseline": {"value": value, "unit": "ms", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "per_frac_ms": {f"{f:g}": (sum(v) / len(v) if v else None) for f, v in times.items()},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scale", type=int, default=22)
    ap.add_argument("--ef", type=int, default=16)
    ap.add_argument("--precision", choices=["fp64", "fp32"], default=None,
                    help="default fp64 for the plain workload, fp32 for the batched form")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true", help="plain workload: skip the FP32 leg")
    ap.add_argument("--cpu-timeout", type=float, default=600.0)
    ap.add_argument("--config", choices=["plain", "precision", "batched", "serving", "mixes", "kmer"], default="plain",
                    help="plain: the headline workload (R-MAT s22 sweep); precision / batched / serving: "
                         "those forms; mixes: insertion-only / deletion-only / 80/20 batches and the tau_f "
                         "sweep, with L1 errors against a reference Static PageRank; kmer: the low-degree huge "
                         "graph (k-mer stand-in)")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: Poisson arrivals per second")
    ap.add_argument("--sub-rate", type=float, default=50.0,
                    help="serving leg of the default run: a second, lower offered rate")
    ap.add_argument("--duration", type=float, default=2.0, help="serving: seconds of arrivals")
    ap.add_argument("--serve-duration", type=float, default=1.0,
                    help="serving leg of the default run: seconds of arrivals per rate")
    ap.add_argument("--nvtx", action="store_true",
                    help="mark each timed rank call with an NVTX range named after it (static, naive, df, dt, "
                         "df_async), so that a profiler can select one call")
    ap.add_argument("--no-legs", action="store_true",
                    help="default run: skip the serving, batched and precision legs (and the precision oracle)")
    ap.add_argument("--slots", type=int, default=2, help="serving: concurrent updates")
    ap.add_argument("--coalesce", type=int, default=256, help="serving: requests per coalesced update")
    ap.add_argument("--serve-scales", default="18,18,19,20,21,22,23,24", help="serving: R-MAT scales")
    ap.add_argument("--graphs", type=int, default=256, help="graphs of the batched form")
    ap.add_argument("--kmer-n", type=int, default=200_000_000, help="kmer: vertices of the k-mer stand-in")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.precision is None:
        args.precision = "fp32" if args.config in ("batched", "serving") else "fp64"
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.config == "precision":
        run_precision(args, rank, world, local_rank)
    elif args.config == "batched":
        run_batched(args, rank, world, local_rank)
    elif args.config == "serving":
        run_serving(args, rank, world, local_rank)
    elif args.config == "mixes":
        run_mixes(args, rank, world, local_rank)
    elif args.config == "kmer":
        run_kmer(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
