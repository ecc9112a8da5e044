#!/usr/bin/env python3
"""Benchmark of the GleanVec eager multi-step search on GB300.

One step = one pass of the whole hot path over one batch of queries with device-resident
inputs:  glv_project_queries -> glv_score_candidates -> glv_topk -> glv_rerank.
Default workload: 1M x 768 database, d = 160, C = 32 clusters, 10,000 OOD queries, 2,048
random candidate ids per query (graph-search-like gathers), kappa = 100 re-ranked to
k = 10, reduced rows stored in BF16 (the FP32 store is timed beside it).

Prints ONE JSON line (rank 0).  Multi-GPU (torchrun): every rank holds a replica of the
database and searches its own query set (queries are independent, so there is no data
collective); value = all ranks' queries / max-over-ranks time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl glv|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import signal
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "queries/s at 10-recall@10>=0.9 vs oracle (low-prec vs FP32); gather-score HBM GB/s"
UNIT = "queries/s"
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="glv", choices=["glv", "reference"])
    p.add_argument("--workload", default="graph-1M-d160")
    p.add_argument("--store", default="bf16", choices=["f32", "bf16", "fp8"])
    p.add_argument("--compare-stores", default="fp8,f32", help="comma list of other stores to time too")
    p.add_argument("--cpu-sample", type=int, default=256, help="queries in the CPU-baseline sample")
    p.add_argument("--recall-sample", type=int, default=256)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--ref-queries-per-step", type=int, default=256)
    p.add_argument("--no-autotune", action="store_true", help="keep the library's default scoring configuration")
    p.add_argument("--graph", action="store_true", help="time the step as a captured CUDA graph")
    p.add_argument("--queries", default="ood", choices=["ood", "id"], help="query distribution")
    p.add_argument("--lazy", action="store_true",
                   help="also time the lazy inner product (Algorithm 3) against the eager path")
    p.add_argument("--score-error", action="store_true",
                   help="report each store's score error against the FP64 oracle on the recall sample")
    p.add_argument("--per-query", type=int, default=0,
                   help="also time the per-query launch path on this many queries (batching comparison)")
    p.add_argument("--override", nargs="*", default=[],
                   help="workload fields to override, e.g. nq=2000 D=256 (smaller profiling cases)")
    a = p.parse_args()
    a.overrides = {}
    for kv in a.override:
        k, v = kv.split("=", 1)
        a.overrides[k] = int(v)
    return a


# ---------------------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------------------

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float) -> float:
    """Max of a per-rank float over the process group (identity without one).  Used for the
    step time: the job is as slow as its slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(per_rank_units: int, world: int, max_ms: float) -> float:
    """Whole-job units per second: every rank processed per_rank_units in at most max_ms."""
    return world * per_rank_units / (max_ms / 1e3)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            mp = json.load(f)
        return float(mp["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        # wait for the first sample, so nvidia-smi's start-up is over before timing starts
        t0 = time.time()
        while self.proc is not None and time.time() - t0 < 10:
            if os.path.getsize(self.tmp.name) > 0:
                break
            time.sleep(0.05)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        self.tmp.flush()
        rows = []
        try:
            with open(self.tmp.name) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        finally:
            os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [num(r[3]) for r in rows if num(r[3]) is not None]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


def source_sha(*rel):
    h = hashlib.sha256()
    for r in rel:
        with open(os.path.join(ROOT, r), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


KERNEL_SOURCES = tuple("paper_2410_22347_gb300/csrc/" + f for f in (
    "score_variants.cuh", "score_dev.cuh", "score_launch.cuh", "score_bulk.cuh", "topk_dev.cuh", "common.cuh",
    "kernels.cuh", "score.cu", "score_bf16_fused.cu", "score_fp8_fused.cu", "score_f32_fused.cu"))


def recorded_traffic(workload: str, store: str):
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, valid
    only while the kernel source still has the hash the counters were taken with."""
    path = os.path.join(ROOT, "profiles", "score_topk_traffic.md")
    if not os.path.exists(path):
        return None
    sha = source_sha(*KERNEL_SOURCES)
    with open(path) as f:
        for line in f:
            m = re.match(r"\s*traffic\s+(\S+)\s+(\S+)\s+([0-9a-f]+)\s+([0-9.eE+]+)", line)
            if m and m.group(1) == workload and m.group(2) == store and m.group(3) == sha:
                return float(m.group(4))
    return None


# ---------------------------------------------------------------------------------------
# oracle (CPU baseline / reference arm / recall check) on a bounded sample
# ---------------------------------------------------------------------------------------

def oracle_subproblem(X, Q, mu, A, B, off, ids, qsel):
    """Restrict the problem to the database rows the selected queries touch (a valid
    GleanVec problem on its own: tags and reduced rows are per row).  numpy inputs."""
    import numpy as np
    import oracle
    lists = [ids[off[j]:off[j + 1]] for j in qsel]
    cat = np.concatenate(lists) if lists else np.zeros(0, np.int32)
    uniq = np.unique(cat)
    loff = np.zeros(len(qsel) + 1, np.int64)
    loff[1:] = np.cumsum([len(l) for l in lists])
    lids = np.searchsorted(uniq, cat).astype(np.int32)
    Xs = np.ascontiguousarray(X[uniq])
    t0 = time.perf_counter()
    tags = oracle.assign_tags(Xs, mu)
    Xr = oracle.build_reduced(Xs, tags, B)
    prep = time.perf_counter() - t0
    return dict(X=Xs, Q=np.ascontiguousarray(Q[qsel]), A=A, tags=tags, Xr=Xr, off=loff, ids=lids, uniq=uniq,
                prep_s=prep)


def oracle_search_timed(sp, kappa, k, repeats=1):
    import oracle
    best = None
    out = None
    for _ in range(repeats):
        t0 = time.perf_counter()
        out = oracle.search(sp["X"], sp["Xr"], sp["tags"], sp["A"], sp["Q"], sp["off"], sp["ids"], kappa, k)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    s, i = out
    import numpy as np
    gid = np.where(i >= 0, sp["uniq"][np.clip(i, 0, None)], -1)
    return best, s, gid


# ---------------------------------------------------------------------------------------
# reference arm: the oracle, timed on the host cores
# ---------------------------------------------------------------------------------------

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import torch
    import oracle
    from paper_2410_22347_gb300 import synth

    oracle.set_threads(os.cpu_count() or 1)
    w = synth.workload(args.workload, device="cpu", queries=args.queries, **args.overrides)
    X, Q, mu, A, B = (t.numpy() for t in (w.X, w.Q, w.mu, w.A, w.B))
    off, ids = w.off.numpy(), w.ids.numpy()
    nq = Q.shape[0]
    per = min(args.ref_queries_per_step, nq)
    nsteps = args.warmup + args.steps
    sels = [np.arange(s * per, s * per + per) % nq for s in range(nsteps)]
    allq = np.unique(np.concatenate(sels))
    sp = oracle_subproblem(X, Q, mu, A, B, off, ids, allq)
    pos = {int(q): t for t, q in enumerate(allq)}
    times = []
    for s in range(nsteps):
        loc = np.array([pos[int(q)] for q in sels[s]])
        sub = dict(sp)
        sub["Q"] = sp["Q"][loc]
        lo = sp["off"]
        lists = [sp["ids"][lo[t]:lo[t + 1]] for t in loc]
        sub["off"] = np.zeros(len(loc) + 1, np.int64)
        sub["off"][1:] = np.cumsum([len(l) for l in lists])
        sub["ids"] = np.concatenate(lists).astype(np.int32)
        dt, _, _ = oracle_search_timed(sub, w.kappa, w.k)
        if s >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = per * len(times) / total
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": args.workload, "queries_per_step": per, "candidates_per_query": 2048,
                   "kappa": w.kappa, "k": w.k},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                         "sample": f"{per} queries per step, reduced rows precomputed for the "
                                   f"{len(sp['uniq'])} rows they touch ({sp['prep_s']:.1f} s, untimed)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------

def run_glv(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    from paper_2410_22347_gb300 import build_lib
    build_lib.build()
    from paper_2410_22347_gb300 import glv, synth
    from paper_2410_22347_gb300.index import GleanVecIndex

    w = synth.workload(args.workload, device=dev, replica=rank, queries=args.queries, **args.overrides)
    nq, D = w.Q.shape
    C, d, _ = w.A.shape
    total = int(w.off[-1])
    stores = [args.store] + [s for s in args.compare_stores.split(",") if s and s not in (args.store, "none")]
    idx = {}
    for st in stores:
        idx[st] = GleanVecIndex(w.X, w.A, w.B, mu=w.mu if not idx else None,
                                tags=None if not idx else next(iter(idx.values())).tags, store=st)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2

    def step(ix, ev=None):
        b = ix._buffers(nq, total, w.kappa, w.k)
        if ev:
            ev[0].record()
        glv.glv_project_queries(w.Q, ix.A, ix.compute, Qp=b["Qp"], workspace=b["pws"], d_status=ix.status)
        if ev:
            ev[1].record()
        glv.glv_score_topk(b["Qp"], ix.Xred, ix.row_stride, ix.scales, ix.dt, ix.tags, w.off, w.ids, w.kappa,
                           scores_scratch=b["scores"], workspace=b["tws"], out_s=b["ts"], out_id=b["ti"], d_status=ix.status)
        if ev:
            ev[2].record()
        glv.glv_rerank(w.X, w.Q, b["ti"], w.k, out_s=b["fs"], out_id=b["fi"], d_status=ix.status)
        if ev:
            ev[3].record()
        return b["fs"], b["fi"]

    # projection: 2 operand-prep launches + GEMM; (work plan +) fused score+top-k; re-rank
    launches_per_step = 3 + 2
    results = {}
    tuned = {}
    clocks = None
    for si, st in enumerate(stores):
        ix = idx[st]
        if not args.no_autotune:  # untimed set-up: pick the scoring configuration for this store
            from paper_2410_22347_gb300.autotune import tune_score
            G, mode, carve, sched, table = tune_score(ix, w.Q, w.off, w.ids, w.kappa, use_cache=False)
            tuned[st] = {"lanes_per_candidate": G, "gather_mode": mode, "smem_carveout_kb": carve,
                         "schedule": sched, "ms_by_config(G/mode/carveout_kb/schedule)": table}
        for _ in range(args.warmup):
            step(ix)
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if si == 0 else None
        if sampler:
            sampler.__enter__()
        t0 = time.perf_counter()
        torch.cuda.nvtx.range_push(f"timed_{st}")  # lets a profiler select the timed launches
        for s in range(args.steps):
            flush.zero_()  # evict L2 between timed steps (not inside the timed events)
            step(ix, evs[s])
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if sampler:
            sampler.__exit__()
            clocks = sampler.summary()
        if world > 1:
            dist.barrier()
        per_step = [evs[s][0].elapsed_time(evs[s][3]) for s in range(args.steps)]
        kern = [[evs[s][t].elapsed_time(evs[s][t + 1]) for s in range(args.steps)] for t in range(3)]
        tot_ms = max_over_ranks(sum(per_step))
        assert ix.device_status() == 0, "device reported an error during the bench"
        results[st] = dict(ms_per_step=tot_ms / args.steps,
                           value=job_throughput(nq * args.steps, world, tot_ms),
                           kernels_ms={n: statistics.mean(v) for n, v in
                                       zip(("project", "score_topk", "rerank"), kern)},
                           wall_s=wall)

    # ---- batching: the step as one CUDA graph, and the per-query launch path ----
    batching = {}
    if args.graph or args.per_query:
        ix = idx[args.store]
        if args.graph:
            g = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                step(ix)  # warm the buffers on the capture stream
            torch.cuda.current_stream().wait_stream(side)
            torch.cuda.synchronize()
            with torch.cuda.graph(g):
                step(ix)
            g.replay()
            torch.cuda.synchronize()
            gms = []
            for _ in range(max(5, min(args.steps, 50))):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                g.replay()
                e1.record()
                e1.synchronize()
                gms.append(e0.elapsed_time(e1))
            gms_max = max_over_ranks(sum(gms) / len(gms))
            batching["graph"] = {"ms_per_step": gms_max, "value": job_throughput(nq, world, gms_max)}
        if args.per_query:
            nsub = min(args.per_query, nq)
            b = ix._buffers(nq, total, w.kappa, w.k)
            fsz, isz = 4, 4
            Qp1 = torch.empty(1, C, d, dtype=torch.float32, device=dev)
            pws1 = torch.empty(max(glv.project_workspace_bytes(1, D, C, d, ix.compute), 1), dtype=torch.uint8,
                               device=dev)
            lib = glv.lib()
            stv = glv._stream(None)

            def one(j):
                # every query on its own: projection, scoring + top-kappa, re-rank (pointer offsets)
                lib.glv_project_queries(w.Q.data_ptr() + j * D * 4, 1, D, ix.A.data_ptr(), C, d, ix.compute,
                                        Qp1.data_ptr(), pws1.data_ptr(), None, stv)
                lib.glv_score_topk(Qp1.data_ptr(), 1, C, d, ix.Xred.data_ptr(), ix.row_stride,
                                   None if ix.scales is None else ix.scales.data_ptr(), ix.dt, ix.tags.data_ptr(),
                                   ix.N, w.off.data_ptr() + j * 8, w.ids.data_ptr(), total, w.kappa,
                                   b["scores"].data_ptr(), b["tws"].data_ptr(), b["ts"].data_ptr() + j * w.kappa * fsz,
                                   b["ti"].data_ptr() + j * w.kappa * isz, None, stv)
                lib.glv_rerank(w.X.data_ptr(), ix.N, D, w.Q.data_ptr() + j * D * 4, 1,
                               b["ti"].data_ptr() + j * w.kappa * isz, w.kappa, w.k,
                               b["fs"].data_ptr() + j * w.k * fsz, b["fi"].data_ptr() + j * w.k * isz, None, stv)
            for j in range(min(8, nsub)):
                one(j)
            torch.cuda.synchronize()
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for j in range(nsub):
                one(j)
            e1.record()
            e1.synchronize()
            pms = max_over_ranks(e0.elapsed_time(e1))
            batching["per_query_launches"] = {"queries": nsub, "ms": pms,
                                              "value": job_throughput(nsub, world, pms)}

    # ---- lazy (Algorithm 3) vs eager (Algorithm 4) scoring + top-kappa ----
    lazy = None
    if args.lazy:
        ix = idx[args.store]
        b = ix._buffers(nq, total, w.kappa, w.k)
        vis = torch.empty(nq, dtype=torch.int32, device=dev)

        def lazy_step():
            glv.glv_score_lazy(w.Q, ix.A, ix.Xred, ix.row_stride, ix.scales, ix.dt, ix.tags, w.off, w.ids,
                               scores=b["scores"], visited=vis)
            glv.glv_topk(b["scores"], w.off, w.ids, w.kappa, out_s=b["ts"], out_id=b["ti"])

        def eager_step():
            glv.glv_project_queries(w.Q, ix.A, ix.compute, Qp=b["Qp"], workspace=b["pws"])
            glv.glv_score_topk(b["Qp"], ix.Xred, ix.row_stride, ix.scales, ix.dt, ix.tags, w.off, w.ids, w.kappa,
                               scores_scratch=b["scores"], workspace=b["tws"], out_s=b["ts"], out_id=b["ti"])

        def timed(fn, reps=10):
            fn()
            torch.cuda.synchronize()
            ms = []
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                fn()
                e1.record()
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            return sum(ms) / len(ms)
        le, ee = timed(lazy_step), timed(eager_step)
        v = vis.float()
        lazy = {"lazy_ms": le, "eager_ms": ee, "visited_clusters_mean": float(v.mean()),
                "visited_clusters_max": int(vis.max()), "clusters": C}

    # ---- gather ceiling: the same rows for the same candidate ids, read with no arithmetic ----
    ixc = idx[args.store]
    gout = torch.empty(total, dtype=torch.float32, device=dev)
    for _ in range(3):
        glv.glv_gather_rows(ixc.Xred, ixc.row_stride, w.ids, out=gout)
    torch.cuda.synchronize()
    g_ms = []
    for _ in range(10):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        glv.glv_gather_rows(ixc.Xred, ixc.row_stride, w.ids, out=gout)
        e1.record()
        e1.synchronize()
        g_ms.append(e0.elapsed_time(e1))
    gather_ms = sum(g_ms) / len(g_ms)
    del gout


    # Every step copies its queries and candidate lists from pinned host memory and reads
    # its top-k back; steps stream through HostSearchPipeline, so step s+1's copies overlap
    # step s's search.  The serial figure is one batch alone (copy in, search, copy out).
    from paper_2410_22347_gb300.index import HostSearchPipeline
    ix = idx[args.store]
    Qh = w.Q.cpu().pin_memory()
    offh = w.off.cpu().pin_memory()
    idsh = w.ids.cpu().pin_memory()
    outs = torch.empty(nq, w.k, dtype=torch.float32, pin_memory=True)
    outi = torch.empty(nq, w.k, dtype=torch.int32, pin_memory=True)
    for _ in range(max(1, args.warmup)):
        ix.search_host(Qh, offh, idsh, w.kappa, w.k, outs, outi)
    torch.cuda.synchronize()
    e2e_steps = max(5, min(args.steps, 20))
    e_ms = []
    for _ in range(e2e_steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        ix.search_host(Qh, offh, idsh, w.kappa, w.k, outs, outi)
        e1.record()
        e1.synchronize()
        e_ms.append(e0.elapsed_time(e1))
    serial_ms = max_over_ranks(sum(e_ms) / len(e_ms))
    pipe = HostSearchPipeline(ix, w.kappa, w.k)
    for _ in range(max(3, args.warmup)):
        pipe.submit(Qh, offh, idsh, outs, outi)
    pipe.synchronize()
    pipe_steps = max(10, min(args.steps, 50))
    flush.zero_()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    pipe.begin()
    for _ in range(pipe_steps):
        pipe.submit(Qh, offh, idsh, outs, outi)
    e1.record()
    e1.synchronize()
    pipe.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / pipe_steps)
    h2d = Qh.numel() * 4 + offh.numel() * 8 + idsh.numel() * 4
    d2h = outs.numel() * 4 + outi.numel() * 4

    # ---- recall vs the FP64 oracle (rank 0, bounded sample) and CPU baseline ----
    line_extra = {}
    if rank == 0:
        import oracle
        oracle.set_threads(os.cpu_count() or 1)
        Xn = w.X.cpu().numpy()
        Qn = w.Q.cpu().numpy()
        mun, An, Bn = w.mu.cpu().numpy(), w.A.cpu().numpy(), w.B.cpu().numpy()
        offn, idsn = w.off.cpu().numpy(), w.ids.cpu().numpy()
        rng = np.random.default_rng(12345)
        qsel = np.sort(rng.choice(nq, size=min(args.recall_sample, nq), replace=False))
        sp = oracle_subproblem(Xn, Qn, mun, An, Bn, offn, idsn, qsel)
        ot, os_, oid = oracle_search_timed(sp, w.kappa, w.k)
        recall = {}
        for st in stores:
            fs, fi = step(idx[st])
            torch.cuda.synchronize()
            recall[st] = oracle.recall(fi.cpu().numpy()[qsel], oid)
        line_extra["recall_10at10_vs_oracle"] = recall
        if args.score_error:
            # reduced-space scores of the sample, each store against the unquantised FP64 oracle
            # (rows whose GPU tag differs from the oracle's near-tie decision are left out)
            import oracle as orc
            red, _ = orc.score(orc.project(sp["Q"], sp["A"]), sp["Xr"], sp["tags"], sp["off"], sp["ids"])
            gtags = idx[args.store].tags.cpu().numpy()
            rows = sp["uniq"][sp["ids"]]
            same = gtags[rows] == sp["tags"][sp["ids"]]
            qn = np.linalg.norm(orc.project(sp["Q"], sp["A"]), axis=2)
            xn = np.linalg.norm(sp["Xr"], axis=1)
            cj = np.repeat(np.arange(len(qsel)), np.diff(sp["off"]))
            scale = np.maximum(np.abs(red), qn[cj, sp["tags"][sp["ids"]]] * xn[sp["ids"]])
            errs = {}
            for st in stores:
                ix = idx[st]
                b = ix._buffers(nq, total, w.kappa, w.k)
                glv.glv_project_queries(w.Q, ix.A, ix.compute, Qp=b["Qp"], workspace=b["pws"])
                sc = glv.glv_score_candidates(b["Qp"], ix.Xred, ix.row_stride, ix.scales, ix.dt, ix.tags, w.off,
                                              w.ids)
                allsc = sc.cpu().numpy()
                got = np.concatenate([allsc[offn[j]:offn[j + 1]] for j in qsel])
                rel = np.abs(got - red)[same] / scale[same]
                errs[st] = {"max_rel": float(rel.max()), "mean_rel": float(rel.mean()),
                            "p99_rel": float(np.quantile(rel, 0.99))}
            line_extra["score_error_vs_fp64_oracle"] = errs
        line_extra["recall_sample"] = f"{len(qsel)} random queries; oracle restricted to the rows they touch"
        if not args.no_cpu_baseline:
            csel = qsel if args.cpu_sample == len(qsel) else np.sort(
                rng.choice(nq, size=min(args.cpu_sample, nq), replace=False))
            cp = sp if csel is qsel else oracle_subproblem(Xn, Qn, mun, An, Bn, offn, idsn, csel)
            ctime, _, _ = oracle_search_timed(cp, w.kappa, w.k, repeats=3)
            line_extra["cpu_baseline"] = {
                "value": len(csel) / ctime, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                "sample": f"{len(csel)} of the {nq} queries (all {w.ids.shape[0] // nq} candidates each); "
                          f"reduced rows precomputed untimed for the {len(cp['uniq'])} rows they touch; best of 3"}

    if world > 1:
        dist.barrier()
    if rank != 0:
        return 0

    head = results[args.store]
    hbm, peak_kind = measured_peaks()
    eb = glv.elem_bytes(glv.DTYPES[args.store])
    bytes_per_cand = d * eb + (4 if args.store == "fp8" else 0) + 4
    alg_bytes = total * bytes_per_cand
    score_ms = head["kernels_ms"]["score_topk"]
    achieved = alg_bytes / (score_ms / 1e3) / 1e9
    traffic = recorded_traffic(args.workload, args.store)
    rec = line_extra.get("recall_10at10_vs_oracle", {}).get(args.store)
    line = {
        "metric": METRIC,
        "value": head["value"],
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": head["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": args.store,
        "data": "synthetic",
        "config": {"workload": args.workload, "overrides": args.overrides or None, "N": int(w.X.shape[0]), "D": D, "d": d, "C": C,
                   "queries_per_gpu": nq, "candidates_per_query": total // nq, "kappa": w.kappa, "k": w.k,
                   "reduced_row_store": args.store, "accumulate": "f32",
                   "projection": {0: "f32 (tcgen05 3xTF32)", 1: "bf16 (tcgen05)"}[idx[args.store].compute],
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}"},
        "roofline": {"kernel": "glv_score_topk (score_topk_kernel)", "bound": "hbm", "achieved": achieved, "peak": hbm,
                     "unit": "GB/s", "frac": achieved / hbm, "peak_source": f"{peak_kind} hbm_gbs",
                     "traffic": traffic, "algorithmic_bytes_per_launch": alg_bytes,
                     "bytes_per_candidate": bytes_per_cand, "kernel_ms": score_ms,
                     "gather_ceiling": {
                         "kernel": "glv_gather_rows (same rows, same ids, no arithmetic)",
                         "ms": gather_ms,
                         "achieved_GBs": total * (ixc.row_stride + 8) / (gather_ms / 1e3) / 1e9,
                         "frac_of_copy_peak": total * (ixc.row_stride + 8) / (gather_ms / 1e3) / 1e9 / hbm,
                         "score_topk_frac_of_ceiling": gather_ms / score_ms}},
        "kernels_ms": head["kernels_ms"],
        "e2e": {"value": job_throughput(nq, world, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "path": f"HostSearchPipeline, {pipe_steps} steps streamed (copies of step s+1 overlap the "
                        f"search of step s); inputs larger than L2 (reduced store + re-rank rows)",
                "serial_ms_per_batch": serial_ms},
        "gpu_launches": (launches_per_step + (1 if (tuned.get(args.store) or {}).get("schedule", 1) == 1 else 0))
                        * args.steps,
        "clocks": clocks,
        "modes": {st: {"value": r["value"], "ms_per_step": r["ms_per_step"], "kernels_ms": r["kernels_ms"]}
                  for st, r in results.items()},
        "autotune": tuned or None,
        "batching": batching or None,
        "lazy_vs_eager": lazy,
    }
    line.update(line_extra)
    if rec is not None and rec < 0.9:
        line["warning"] = f"{args.store} recall {rec:.3f} below 0.9"
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_learn(args):
    """Differentiation workload: 200k database + 20k OOD learning queries, D = 768, d = 128,
    C = 16.  Times the FP64 second moments, the LeanVec-Sphering initialisation (host
    eigendecompositions) and refinement minibatches of 4096 pairs (forward + backward +
    Adam), and checks one minibatch gradient against the FP64 oracle."""
    import numpy as np
    import torch
    from paper_2410_22347_gb300 import build_lib
    build_lib.build()
    from paper_2410_22347_gb300 import glv, learn, synth
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    kw = dict(N=200_000, D=768, d=128, C=16, nq=20_000, K_db=32, cands=1, kappa=0, k=1, cfg=4)
    kw.update(args.overrides)
    w = synth.make_workload(device=dev, name="refine-200k-d128", **kw)
    n, D = w.X.shape
    C, d, _ = w.A.shape
    tags = glv.glv_assign_tags(w.X, w.mu)
    torch.cuda.synchronize()

    def timed(fn, reps=1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / reps, out

    ms_kx, KX = timed(lambda: learn.glv_second_moments(w.X, tags, C))
    ms_kq, KQ = timed(lambda: learn.glv_second_moments(w.Q))
    fp64_flops = (n + w.Q.shape[0]) * D * (D + 1)  # multiply-adds of the symmetric halves, x2
    t0 = time.perf_counter()
    A0, B0 = learn.sphering_init(w.Q, w.X, tags, C, d)
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t0
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    P = 4096
    A = A0.clone().requires_grad_(True)
    B = B0.clone().requires_grad_(True)
    opt = torch.optim.Adam([A, B], lr=1e-4)

    def minibatch():
        qi = torch.randint(0, w.Q.shape[0], (P,), generator=g, device=dev, dtype=torch.int32)
        xi = torch.randint(0, n, (P,), generator=g, device=dev, dtype=torch.int32)
        opt.zero_grad(set_to_none=True)
        loss = learn.pair_loss(A, B, w.Q, w.X, tags, qi, xi)
        loss.backward()
        opt.step()
        return loss
    for _ in range(args.warmup):
        minibatch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        minibatch()
    e1.record()
    e1.synchronize()
    ms_step = e0.elapsed_time(e1) / args.steps
    # one minibatch gradient against the FP64 oracle (relative to the gradient's max entry)
    import oracle
    qi = torch.randint(0, w.Q.shape[0], (P,), generator=g, device=dev, dtype=torch.int32)
    xi = torch.randint(0, n, (P,), generator=g, device=dev, dtype=torch.int32)
    Ad, Bd = A.detach(), B.detach()
    s, t, u, v = learn.glv_pair_forward(w.Q, w.X, tags, Ad, Bd, qi, xi)
    dA, dB = learn.glv_pair_backward(w.Q, w.X, tags, C, qi, xi, u, v, -2.0 * (t - s))
    qn, xn = qi.cpu().numpy(), xi.cpu().numpy()
    sub_q, sub_x = np.unique(qn), np.unique(xn)
    Qs, Xs = w.Q.cpu().numpy()[sub_q], w.X.cpu().numpy()[sub_x]
    _, gA, gB = oracle.pair_loss_grad(Qs, Xs, tags.cpu().numpy()[sub_x], Ad.cpu().numpy(), Bd.cpu().numpy(),
                                      np.searchsorted(sub_q, qn), np.searchsorted(sub_x, xn))
    rel = max(float(np.abs(dA.cpu().numpy() - gA).max() / np.abs(gA).max()),
              float(np.abs(dB.cpu().numpy() - gB).max() / np.abs(gB).max()))
    line = {"metric": "refinement minibatches/s (4096 pairs: forward + backward + Adam)",
            "value": 1e3 / ms_step, "unit": "minibatches/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (moments f64)", "data": "synthetic",
            "config": {"workload": "refine-200k-d128", "N": n, "nq": int(w.Q.shape[0]), "D": D, "d": d, "C": C,
                       "pairs_per_minibatch": P},
            "second_moments": {"ms_database_per_cluster": ms_kx, "ms_queries": ms_kq,
                               "fp64_tflops": fp64_flops / ((ms_kx + ms_kq) / 1e3) / 1e12},
            "sphering_init_s": init_s, "pairs_per_s": P * 1e3 / ms_step,
            "grad_max_rel_err_vs_fp64_oracle": rel}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "refine-200k-d128":
        return run_learn(args)
    if args.workload == "study-recall-vs-d":
        import torch
        from paper_2410_22347_gb300 import build_lib
        build_lib.build()
        from paper_2410_22347_gb300 import study
        rows = study.recall_vs_d(torch.device("cuda", 0), **args.overrides)
        print(json.dumps({"metric": "10-recall@10 of the reduced inner product (no re-rank) vs exact",
                          "workload": "study-recall-vs-d", "data": "synthetic", "rows": rows}), flush=True)
        return 0
    return run_glv(args)


if __name__ == "__main__":
    sys.exit(main())
