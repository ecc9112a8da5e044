#!/usr/bin/env python3
"""Benchmark of the GleanVec eager multi-step search on GB300.

One step = one pass of the whole hot path over one batch of queries with device-resident
inputs:  glv_project_queries -> glv_score_topk (fused scoring + top-kappa) -> glv_rerank.
Headline workload (the line's value): graph-1M-d160 -- 1M x 768 database, d = 160, C = 32
clusters, 10,000 OOD queries, 2,048 random candidate ids per query (graph-search-like
gathers), kappa = 100 re-ranked to k = 10, reduced rows stored in BF16 (FP8 and FP32 stores
timed beside it).  The default run also times, under "configs":

* precision-10M-d128 -- 10M x 512, d = 128, C = 64, 10,000 OOD + 10,000 ID queries per step,
  4,096 candidates each, kappa = 200: FP8 (one scale per row), BF16 and FP32 stores; recall
  of the final top 10 against the FP64 oracle pipeline (R1) and against the exact top 10
  over the candidates (R2); a kappa sweep, and each store's queries/s at the smallest kappa
  whose R2 reaches 0.9 (the equal-recall comparison);
* batching-2M-d192 -- 2M x 768, d = 192, C = 48, 8,192 queries with lognormal list lengths:
  eager launches, the step as one CUDA-graph replay, and every query launched on its own.

Every workload also reports its a0 build (glv_build_reduced) against the HBM roofline and
the projection GEMM against the tensor peaks (BF16 from the driver's peaks file, TF32
measured here with cuBLAS).

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
FALLBACK_BF16_TFLOPS = 1900.0


HEADLINE = "graph-1M-d160"
EXTRA_CONFIGS = ("precision-10M-d128", "batching-2M-d192")
# (headline store, the other stores timed beside it) per workload
STORES = {"graph-1M-d160": ("bf16", "fp8,f32"), "precision-10M-d128": ("fp8", "bf16,f32"),
          "batching-2M-d192": ("bf16", ""), "exhaustive-10k": ("f32", "")}
KAPPA_SWEEP = (10, 20, 50, 100, 200, 400, 800)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="glv", choices=["glv", "reference"])
    p.add_argument("--workload", default=HEADLINE)
    p.add_argument("--store", default=None, choices=["f32", "bf16", "fp8"])
    p.add_argument("--compare-stores", default=None, help="comma list of other stores to time too ('none': none)")
    p.add_argument("--configs", default="auto",
                   help="comma list of further workloads timed under 'configs' ('auto': the precision and "
                        "batching workloads when the headline workload runs without overrides; 'none')")
    p.add_argument("--kappa-sweep", default="auto",
                   help="comma list of re-rank depths to sweep ('auto': the precision workload's sweep)")
    p.add_argument("--cpu-sample", type=int, default=256, help="queries in the CPU-baseline sample")
    p.add_argument("--recall-sample", type=int, default=256)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--ref-queries-per-step", type=int, default=256)
    p.add_argument("--no-autotune", action="store_true", help="keep the library's default scoring configuration")
    p.add_argument("--score-config", default=None,
                   help="G/mode/carveout_kb/schedule: install this scoring configuration instead of autotuning")
    p.add_argument("--graph", action="store_true", help="also time the step as a captured CUDA graph")
    p.add_argument("--queries", default=None, choices=["ood", "id", "ood+id"],
                   help="query distribution (default: the workload's own)")
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
    """Roofline denominators: the measured copy bandwidth and BF16 GEMM throughput on
    the GB300s, else the recipe's fallback figures."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            mp = json.load(f)
        return {"hbm_gbs": float(mp["hbm_gbs"]), "bf16_tflops": float(mp["bf16_tflops"]),
                "bf16_tflops_sustained": float(mp.get("bf16_tflops_sustained", 0.0)) or None, "source": "measured"}
    except Exception:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "bf16_tflops": FALLBACK_BF16_TFLOPS, "bf16_tflops_sustained": None,
                "source": "fallback"}


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
    "kernels.cuh", "score.cu") + tuple(f"score_{t}_fused_{m}.cu" for t in ("f32", "bf16", "fp8") for m in ("m0", "m1", "w")))


# DRAM bytes per candidate of the fused score + top-kappa kernel (dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture, divided by the candidates of that launch), per
# (workload, store), with the hash of the kernel sources the counters were taken with; the
# summaries and the capture commands are in profiles/.  A row whose hash no longer matches
# the sources gives traffic null.
TRAFFIC = {
    ("graph-1M-d160", "bf16"): ("7f7a0753cc7b76cb", (1.241791e+09 + 1.717197e+07) / (2000 * 2048)),
    ("precision-10M-d128", "fp8"): ("7f7a0753cc7b76cb", (1.318681e+09 + 1.312358e+07) / (2000 * 4096)),
    ("batching-2M-d192", "bf16"): ("7f7a0753cc7b76cb", (2.939976e+09 + 1.532518e+07) / (4096 * 1868.338623046875)),
}


def recorded_traffic(workload: str, store: str):
    row = TRAFFIC.get((workload, store))
    if row is None or row[0] != source_sha(*KERNEL_SOURCES):
        return None
    return row[1]


# ---------------------------------------------------------------------------------------
# oracle (CPU baseline / reference arm / recall checks) on a bounded sample
# ---------------------------------------------------------------------------------------

def oracle_subproblem(w, qsel):
    """Restrict the problem to the database rows the selected queries touch (a valid GleanVec
    problem on its own: tags and reduced rows are per row).  The rows are gathered where the
    workload lives (on the GPU for the GPU arm), then copied to the host; the oracle computes
    the cluster tags and reduced rows of the touched rows itself (timed as prep_s)."""
    import numpy as np
    import torch
    import oracle
    off = w.off.cpu().numpy()
    qsel = np.asarray(qsel)
    lists = [w.ids[int(off[j]):int(off[j + 1])] for j in qsel]
    cat = torch.cat(lists) if lists else torch.zeros(0, dtype=torch.int32, device=w.ids.device)
    uniq = torch.unique(cat)
    lids = torch.searchsorted(uniq, cat).to(torch.int32)
    Xs = w.X[uniq.long()].cpu().numpy()
    Qs = w.Q[torch.as_tensor(qsel, device=w.Q.device).long()].cpu().numpy()
    loff = np.zeros(len(qsel) + 1, np.int64)
    loff[1:] = np.cumsum([len(l) for l in lists])
    t0 = time.perf_counter()
    tags = oracle.assign_tags(Xs, w.mu.cpu().numpy())
    Xr = oracle.build_reduced(Xs, tags, w.B.cpu().numpy())
    prep = time.perf_counter() - t0
    return dict(X=Xs, Q=Qs, A=w.A.cpu().numpy(), tags=tags, Xr=Xr, off=loff, ids=lids.cpu().numpy(),
                uniq=uniq.cpu().numpy(), prep_s=prep)


def _global(sp, ids):
    import numpy as np
    return np.where(ids >= 0, sp["uniq"][np.clip(ids, 0, None)], -1)


def oracle_search_timed(sp, kappa, k, repeats=1):
    """The oracle's whole search of the sample (project, score, top-kappa, re-rank), best of
    `repeats` wall times; returns (seconds, final scores, final global ids)."""
    import oracle
    best = None
    out = None
    for _ in range(repeats):
        t0 = time.perf_counter()
        out = oracle.search(sp["X"], sp["Xr"], sp["tags"], sp["A"], sp["Q"], sp["off"], sp["ids"], kappa, k)
        dt = time.perf_counter() - t0
        best = dt if best is None else min(best, dt)
    s, i = out
    return best, s, _global(sp, i)


def oracle_reduced_scores(sp):
    import oracle
    s, _ = oracle.score(oracle.project(sp["Q"], sp["A"]), sp["Xr"], sp["tags"], sp["off"], sp["ids"])
    return s


def oracle_final_ids(sp, red, kappa, k):
    """Final top-k global ids of the oracle pipeline at re-rank depth kappa (0: no re-rank),
    from its FP64 reduced scores `red`."""
    import oracle
    if kappa == 0:
        _, ids = oracle.topk(red, sp["off"], sp["ids"], k)
        return _global(sp, ids)
    _, surv = oracle.topk(red, sp["off"], sp["ids"], kappa)
    _, fid, _ = oracle.rerank(sp["X"], sp["Q"], surv, k)
    return _global(sp, fid)


def oracle_exact_ids(sp, k):
    """Exact top-k of <q, x> over each sampled query's whole candidate list (global ids)."""
    import oracle
    _, ids = oracle.exact_topk(sp["X"], sp["Q"], sp["off"], sp["ids"], k)
    return _global(sp, ids)


# ---------------------------------------------------------------------------------------
# reference arm: the oracle, timed on the host cores
# ---------------------------------------------------------------------------------------

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    from paper_2410_22347_gb300 import synth

    oracle.set_threads(os.cpu_count() or 1)
    w = synth.workload(args.workload, device="cpu", queries=args.queries, **args.overrides)
    nq = w.Q.shape[0]
    per = min(args.ref_queries_per_step, nq)
    nsteps = args.warmup + args.steps
    sels = [np.arange(s * per, s * per + per) % nq for s in range(nsteps)]
    allq = np.unique(np.concatenate(sels))
    sp = oracle_subproblem(w, allq)
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
        "config": {"workload": args.workload, "queries_per_step": per,
                   "candidates_per_query": int(w.off[-1]) // nq, "kappa": w.kappa, "k": w.k},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                         "sample": f"{per} queries per step, reduced rows precomputed for the "
                                   f"{len(sp['uniq'])} rows they touch ({sp['prep_s']:.1f} s, untimed)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------
# GPU arm: building blocks
# ---------------------------------------------------------------------------------------

def _events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def search_step(glv, ix, w, b, kappa, ev=None):
    """One step of the hot path over the whole batch: projection, fused score + top-kappa,
    re-rank (kappa = 0: top k of the reduced scores, no re-rank)."""
    if ev:
        ev[0].record()
    glv.glv_project_queries(w.Q, ix.A, ix.compute, Qp=b["Qp"], workspace=b["pws"], d_status=ix.status)
    if ev:
        ev[1].record()
    kk = kappa if kappa > 0 else w.k
    glv.glv_score_topk(b["Qp"], ix.Xred, ix.row_stride, ix.scales, ix.dt, ix.tags, w.off, w.ids, kk,
                       scores_scratch=b["scores"], workspace=b["tws"], out_s=b["ts"] if kappa > 0 else b["fs"],
                       out_id=b["ti"] if kappa > 0 else b["fi"], d_status=ix.status)
    if ev:
        ev[2].record()
    if kappa > 0:
        glv.glv_rerank(w.X, w.Q, b["ti"], w.k, out_s=b["fs"], out_id=b["fi"], d_status=ix.status)
    if ev:
        ev[3].record()
    return b["fs"], b["fi"]


def time_search(glv, ix, w, kappa, steps, warmup, flush, world, sampler=None, label=None):
    """Times `steps` search steps with CUDA events on the launching stream (L2 evicted before
    each step, outside the events); returns the per-step and per-kernel means."""
    import torch
    import torch.distributed as dist
    nq = w.Q.shape[0]
    total = int(w.off[-1])
    b = ix._buffers(nq, total, max(kappa, w.k), w.k)
    for _ in range(warmup):
        search_step(glv, ix, w, b, kappa)
    torch.cuda.synchronize()
    evs = [_events(4) for _ in range(steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.__enter__()
    t0 = time.perf_counter()
    if label:
        torch.cuda.nvtx.range_push(label)  # lets a profiler select the timed launches
    for s in range(steps):
        flush.zero_()
        search_step(glv, ix, w, b, kappa, evs[s])
    if label:
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = None
    if sampler:
        sampler.__exit__()
        clocks = sampler.summary()
    if world > 1:
        dist.barrier()
    per_step = [evs[s][0].elapsed_time(evs[s][3]) for s in range(steps)]
    kern = [[evs[s][t].elapsed_time(evs[s][t + 1]) for s in range(steps)] for t in range(3)]
    tot_ms = max_over_ranks(sum(per_step))
    assert ix.device_status() == 0, "device reported an error during the bench"
    return dict(ms_per_step=tot_ms / steps, value=job_throughput(nq * steps, world, tot_ms),
                kernels_ms={n: statistics.mean(v) for n, v in zip(("project", "score_topk", "rerank"), kern)},
                wall_s=wall, clocks=clocks)


def timed_ms(fn, flush, reps):
    """Mean CUDA-event time of fn() over reps calls, L2 evicted before each."""
    import torch
    fn()
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = _events(2)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return sum(ms) / len(ms)


def gather_ceiling_ms(glv, ix, w, flush):
    """The same rows for the same candidate ids, read with no arithmetic (glv_gather_rows)."""
    import torch
    gout = torch.empty(int(w.off[-1]), dtype=torch.float32, device=w.ids.device)
    ms = timed_ms(lambda: glv.glv_gather_rows(ix.Xred, ix.row_stride, w.ids, out=gout), flush, 10)
    del gout
    return ms


def roofline_block(glv, ix, st, w, score_ms, gather_ms, peaks, name):
    """HBM roofline of the fused score + top-kappa kernel: algorithmic bytes per launch (per
    candidate: the reduced row's d elements, the FP8 row scale, the 4-byte id) over its
    CUDA-event time, against the measured copy bandwidth."""
    total = int(w.off[-1])
    bpc = ix.d * glv.elem_bytes(ix.dt) + (4 if st == "fp8" else 0) + 4
    alg = total * bpc
    ach = alg / (score_ms / 1e3) / 1e9
    gbytes = total * (ix.row_stride + 8)
    hbm = peaks["hbm_gbs"]
    tr = recorded_traffic(name, st)
    return {"kernel": "glv_score_topk (score_topk_kernel)", "bound": "hbm", "achieved": ach, "peak": hbm,
            "unit": "GB/s", "frac": ach / hbm, "peak_source": f"{peaks['source']} hbm_gbs",
            "traffic": None if tr is None else tr * total, "algorithmic_bytes_per_launch": alg,
            "bytes_per_candidate": bpc, "kernel_ms": score_ms,
            "gather_ceiling": {"kernel": "glv_gather_rows (same rows, same ids, no arithmetic)", "ms": gather_ms,
                               "achieved_GBs": gbytes / (gather_ms / 1e3) / 1e9,
                               "frac_of_copy_peak": gbytes / (gather_ms / 1e3) / 1e9 / hbm,
                               "score_topk_frac_of_ceiling": gather_ms / score_ms}}


def build_block(glv, ix, w, flush, peaks):
    """Time of the a0 build (glv_build_reduced) into the index's own store, and its HBM
    roofline: X read once, tags, B, and the store (and FP8 scales) written."""
    import torch
    N, D = w.X.shape
    C, d, _ = w.B.shape
    ws = torch.empty(max(int(glv.lib().glv_build_reduced_workspace_size(N, C)), 1), dtype=torch.uint8,
                     device=w.X.device)
    ms = timed_ms(lambda: glv.glv_build_reduced(w.X, ix.tags, w.B, ix.dt, Xred=ix.Xred, row_stride=ix.row_stride,
                                                scales=ix.scales, workspace=ws), flush, 3)
    nbytes = N * D * 4 + N * 2 + C * d * D * 4 + N * ix.row_stride + (N * 4 if ix.scales is not None else 0)
    ach = nbytes / (ms / 1e3) / 1e9
    return {"kernel": "glv_build_reduced (grouping + build_gemm_kernel)", "ms": ms, "bound": "hbm",
            "algorithmic_bytes": nbytes, "achieved": ach, "unit": "GB/s", "peak": peaks["hbm_gbs"],
            "frac": ach / peaks["hbm_gbs"], "tflops": 2.0 * N * D * d / (ms / 1e3) / 1e12}


def projection_block(glv, res, w, peaks, store_compute):
    """Tensor roofline of the projection GEMM Qp = Q [A_1; ...; A_C]^T (its launches' event
    time, operand preparation included): BF16 operands against the measured BF16 peak, the
    FP32 mode (three TF32 MMAs per product) against the measured TF32 peak."""
    nq, D = w.Q.shape
    C, d, _ = w.A.shape
    flops = 2.0 * nq * D * C * d
    out = {}
    for st, r in res.items():
        ms = r["kernels_ms"]["project"]
        if store_compute[st] == 1:
            ach = flops / (ms / 1e3) / 1e12
            out[st] = {"operands": "bf16", "ms": ms, "tflops": ach, "peak": peaks["bf16_tflops"],
                       "frac": ach / peaks["bf16_tflops"], "peak_source": f"{peaks['source']} bf16_tflops"}
        elif peaks.get("tf32_tflops"):
            ach = 3 * flops / (ms / 1e3) / 1e12
            out[st] = {"operands": "f32 as 3 TF32 products (hi*hi + hi*lo + lo*hi)", "ms": ms,
                       "tf32_tflops_executed": ach, "peak": peaks["tf32_tflops"],
                       "frac": ach / peaks["tf32_tflops"], "peak_source": "tf32 measured in this run (cuBLAS)"}
    return out


def measure_tf32_peak(dev):
    """Dense TF32 throughput of cuBLAS on this GPU (8192^3, best of 10): the denominator of
    the FP32-mode projection, which the driver's peaks file does not carry."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        n = 8192
        a = torch.randn(n, n, device=dev)
        bm = torch.randn(n, n, device=dev)
        for _ in range(3):
            torch.matmul(a, bm)
        torch.cuda.synchronize()
        best = None
        for _ in range(10):
            e0, e1 = _events(2)
            e0.record()
            torch.matmul(a, bm)
            e1.record()
            e1.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        return 2.0 * n ** 3 / (best / 1e3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def tune_block(glv, ix, w, kappa, args):
    from paper_2410_22347_gb300.autotune import tune_score
    if args.score_config:
        G, mode, carve, sched = (int(x) for x in args.score_config.split("/"))
        glv.glv_set_score_config(ix.dt, G, mode, carve, sched)
        table = "given on the command line"
    elif args.no_autotune:
        G, mode, carve, sched = glv.glv_get_score_config(ix.dt, ix.d)
        table = "library default"
    else:  # untimed set-up: pick the scoring configuration for this store on this workload
        G, mode, carve, sched, table = tune_score(ix, w.Q, w.off, w.ids, max(kappa, w.k), use_cache=False)
    return {"lanes_per_candidate": G, "gather_mode": mode, "smem_carveout_kb": carve, "schedule": sched,
            "ms_by_config(G/mode/carveout_kb/schedule)": table}


def batching_block(glv, ix, w, args, flush, world, dev):
    """The step as one CUDA-graph replay, and every query launched on its own."""
    import torch
    nq, D = w.Q.shape
    C, d, _ = w.A.shape
    total = int(w.off[-1])
    kappa = w.kappa
    b = ix._buffers(nq, total, kappa, w.k)
    out = {}
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        search_step(glv, ix, w, b, kappa)  # warm the buffers on the capture stream
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        search_step(glv, ix, w, b, kappa)
    gms = max_over_ranks(timed_ms(g.replay, flush, max(5, min(args.steps, 50))))
    out["graph"] = {"ms_per_step": gms, "value": job_throughput(nq, world, gms)}
    nsub = min(args.per_query or 1024, nq)
    Qp1 = torch.empty(1, C, d, dtype=torch.float32, device=dev)
    pws1 = torch.empty(max(glv.project_workspace_bytes(1, D, C, d, ix.compute), 1), dtype=torch.uint8, device=dev)
    lib = glv.lib()
    stv = glv._stream(None)

    def one(j):
        # every query on its own: projection, scoring + top-kappa, re-rank (pointer offsets)
        lib.glv_project_queries(w.Q.data_ptr() + j * D * 4, 1, D, ix.A.data_ptr(), C, d, ix.compute,
                                Qp1.data_ptr(), pws1.data_ptr(), None, stv)
        lib.glv_score_topk(Qp1.data_ptr(), 1, C, d, ix.Xred.data_ptr(), ix.row_stride,
                           None if ix.scales is None else ix.scales.data_ptr(), ix.dt, ix.tags.data_ptr(),
                           ix.N, w.off.data_ptr() + j * 8, w.ids.data_ptr(), total, kappa,
                           b["scores"].data_ptr(), b["tws"].data_ptr(), b["ts"].data_ptr() + j * kappa * 4,
                           b["ti"].data_ptr() + j * kappa * 4, None, stv)
        lib.glv_rerank(w.X.data_ptr(), ix.N, D, w.Q.data_ptr() + j * D * 4, 1,
                       b["ti"].data_ptr() + j * kappa * 4, kappa, w.k,
                       b["fs"].data_ptr() + j * w.k * 4, b["fi"].data_ptr() + j * w.k * 4, None, stv)

    def all_one():
        for j in range(nsub):
            one(j)
    pms = max_over_ranks(timed_ms(all_one, flush, 1))
    out["per_query_launches"] = {"queries": nsub, "ms": pms, "value": job_throughput(nsub, world, pms)}
    return out


def e2e_block(glv, ix, w, args, world, flush):
    """End to end through the host-buffer entry point (glv_search_host): every step copies
    its queries and candidate lists from pinned host memory and reads its top k back, inside
    the timed region.  Steps alternate over two streams (HostSearchPipeline), so one batch's
    copies overlap the other's search; the serial figure is one batch alone on one stream."""
    import torch
    from paper_2410_22347_gb300.index import HostSearchPipeline
    nq = w.Q.shape[0]
    Qh = w.Q.cpu().pin_memory()
    offh = w.off.cpu().pin_memory()
    idsh = w.ids.cpu().pin_memory()
    outs = torch.empty(nq, w.k, dtype=torch.float32, pin_memory=True)
    outi = torch.empty(nq, w.k, dtype=torch.int32, pin_memory=True)
    serial_ms = max_over_ranks(timed_ms(lambda: ix.search_host(Qh, offh, idsh, w.kappa, w.k, outs, outi), flush,
                                        max(5, min(args.steps, 20))))
    pipe = HostSearchPipeline(ix, w.kappa, w.k)
    for _ in range(max(3, args.warmup)):
        pipe.submit(Qh, offh, idsh, outs, outi)
    pipe.synchronize()
    steps = max(10, min(args.steps, 50))
    e0, e1 = _events(2)
    e0.record()
    pipe.begin()
    for _ in range(steps):
        pipe.submit(Qh, offh, idsh, outs, outi)
    pipe.end()
    e1.record()
    e1.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / steps)
    assert ix.device_status() == 0
    h2d = Qh.numel() * 4 + offh.numel() * 8 + idsh.numel() * 4
    d2h = outs.numel() * 4 + outi.numel() * 4
    return {"value": job_throughput(nq, world, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
            "path": f"glv_search_host (C ABI, host buffers), {steps} steps over two streams (copies of one "
                    f"batch overlap the search of the other); inputs larger than L2",
            "serial_ms_per_batch": serial_ms}


def query_kinds(w, name):
    """(label, query index array) per query kind of the batch."""
    import numpy as np
    nq = w.Q.shape[0]
    from paper_2410_22347_gb300 import synth
    mix = synth.WORKLOADS.get(name, {}).get("queries", "ood")
    if mix == "ood+id":
        return [("ood", np.arange(nq // 2)), ("id", np.arange(nq // 2, nq))]
    return [(mix, np.arange(nq))]


def sample_queries(w, name, n, seed=12345):
    """n queries drawn evenly from each query kind of the batch (sorted)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    kinds = query_kinds(w, name)
    per = max(1, n // len(kinds))
    sel = [np.sort(rng.choice(ix, size=min(per, len(ix)), replace=False)) for _, ix in kinds]
    return np.concatenate(sel), [(lab, len(s)) for (lab, _), s in zip(kinds, sel)]


def recall_by_kind(found, truth, counts):
    import oracle
    out, o = {}, 0
    for lab, n in counts:
        out[lab] = oracle.recall(found[o:o + n], truth[o:o + n])
        o += n
    out["all"] = oracle.recall(found, truth)
    return out

# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------

def measure_workload(name, args, *, dev, rank, world, local, flush, peaks, stores, headline, overrides):
    """Times one workload: every store's search step (autotuned), its fused kernel's roofline
    and gather ceiling, its a0 build; on rank 0, recall of each store's final top 10 against
    the FP64 oracle pipeline (R1) and against the exact top 10 over the candidates (R2); and,
    where asked, a kappa sweep and the batching comparison."""
    import numpy as np
    import torch
    import oracle
    from paper_2410_22347_gb300 import glv, synth
    from paper_2410_22347_gb300.index import GleanVecIndex

    w = synth.workload(name, device=dev, replica=rank, queries=args.queries if headline else None, **overrides)
    nq, D = w.Q.shape
    C, d, _ = w.A.shape
    total = int(w.off[-1])
    idx = {}
    for st in stores:
        first = next(iter(idx.values()), None)
        idx[st] = GleanVecIndex(w.X, w.A, w.B, mu=w.mu if first is None else None,
                                tags=None if first is None else first.tags, store=st)
    torch.cuda.synchronize()
    res, tuned, roof, builds = {}, {}, {}, {}
    clocks = None
    for si, st in enumerate(stores):
        ix = idx[st]
        tuned[st] = tune_block(glv, ix, w, w.kappa, args)
        sampler = ClockSampler(local) if si == 0 else None
        label = f"timed_{st}" if headline else f"timed_{name}_{st}"
        r = time_search(glv, ix, w, w.kappa, args.steps, args.warmup, flush, world, sampler=sampler, label=label)
        if si == 0:
            clocks = r.pop("clocks")
        else:
            r.pop("clocks")
        res[st] = r
        roof[st] = roofline_block(glv, ix, st, w, r["kernels_ms"]["score_topk"], gather_ceiling_ms(glv, ix, w, flush),
                                  peaks, name)
        builds[st] = build_block(glv, ix, w, flush, peaks)
    out = {"workload": name, "N": int(w.X.shape[0]), "D": D, "d": d, "C": C, "queries": nq,
           "query_mix": synth.WORKLOADS.get(name, {}).get("queries", "ood") if not args.queries or not headline
           else args.queries,
           "candidates_per_query": total / nq, "candidates_per_query_max": int((w.off[1:] - w.off[:-1]).max()),
           "kappa": w.kappa, "k": w.k, "clocks": clocks, "autotune": tuned, "build": builds,
           "projection": projection_block(glv, res, w, peaks, {st: idx[st].compute for st in stores}),
           "stores": {st: {"value": r["value"], "ms_per_step": r["ms_per_step"], "kernels_ms": r["kernels_ms"],
                           "roofline": roof[st]} for st, r in res.items()}}
    out["_results"] = res
    out["_launches_per_step"] = {st: 5 + (tuned[st]["schedule"] & 1) for st in stores}

    if name == "batching-2M-d192" or (headline and (args.graph or args.per_query)):
        out["batching"] = batching_block(glv, idx[stores[0]], w, args, flush, world, dev)
        out["batching"]["eager"] = {"ms_per_step": res[stores[0]]["ms_per_step"], "value": res[stores[0]]["value"]}

    if headline and args.lazy:
        ix = idx[stores[0]]
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
        le, ee = timed_ms(lazy_step, flush, 10), timed_ms(eager_step, flush, 10)
        out["lazy_vs_eager"] = {"lazy_ms": le, "eager_ms": ee, "visited_clusters_mean": float(vis.float().mean()),
                                "visited_clusters_max": int(vis.max()), "clusters": C}

    if headline:
        out["e2e"] = e2e_block(glv, idx[stores[0]], w, args, world, flush)

    # ---- recall against the FP64 oracle (rank 0, bounded sample) ----
    if rank == 0:
        oracle.set_threads(os.cpu_count() or 1)
        qsel, counts = sample_queries(w, name, args.recall_sample)
        sp = oracle_subproblem(w, qsel)
        red = oracle_reduced_scores(sp)
        exact = oracle_exact_ids(sp, w.k)
        ref = oracle_final_ids(sp, red, w.kappa, w.k)
        rec = {}
        for st in stores:
            b = idx[st]._buffers(nq, total, max(w.kappa, w.k), w.k)
            _, fi = search_step(glv, idx[st], w, b, w.kappa)
            got = fi.cpu().numpy()[qsel]
            rec[st] = {"R1_vs_oracle_pipeline": recall_by_kind(got, ref, counts),
                       "R2_vs_exact_top10": recall_by_kind(got, exact, counts)}
        out["recall_10at10"] = rec
        out["recall_sample"] = (f"{len(qsel)} queries ({', '.join(f'{n} {lab}' for lab, n in counts)}); oracle "
                                f"restricted to the {len(sp['uniq'])} rows they touch")
        if args.score_error and headline:
            out["score_error_vs_fp64_oracle"] = score_error_block(glv, idx, w, sp, qsel, stores)
        if args.kappa_sweep != "none" and (name == "precision-10M-d128" or (headline and args.kappa_sweep != "auto")):
            kaps = KAPPA_SWEEP if args.kappa_sweep in ("auto",) else [int(x) for x in args.kappa_sweep.split(",")]
            out["kappa_sweep"], out["equal_recall"] = kappa_sweep_block(glv, idx, w, stores, kaps, sp, red, exact,
                                                                        qsel, counts, args, flush, world)
        if headline and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline_block(w, sp, qsel, args)
    for ix in idx.values():
        ix._buf = {}
    del idx, w
    torch.cuda.empty_cache()
    return out


def score_error_block(glv, idx, w, sp, qsel, stores):
    """Reduced-space scores of the sample, each store against the unquantised FP64 oracle
    (rows whose GPU tag differs from the oracle's near-tie decision are left out)."""
    import numpy as np
    import oracle as orc
    nq = w.Q.shape[0]
    offn = w.off.cpu().numpy()
    red, _ = orc.score(orc.project(sp["Q"], sp["A"]), sp["Xr"], sp["tags"], sp["off"], sp["ids"])
    gtags = next(iter(idx.values())).tags.cpu().numpy()
    rows = sp["uniq"][sp["ids"]]
    same = gtags[rows] == sp["tags"][sp["ids"]]
    qn = np.linalg.norm(orc.project(sp["Q"], sp["A"]), axis=2)
    xn = np.linalg.norm(sp["Xr"], axis=1)
    cj = np.repeat(np.arange(len(qsel)), np.diff(sp["off"]))
    scale = np.maximum(np.abs(red), qn[cj, sp["tags"][sp["ids"]]] * xn[sp["ids"]])
    errs = {}
    for st in stores:
        ix = idx[st]
        b = ix._buffers(nq, int(w.off[-1]), w.kappa, w.k)
        glv.glv_project_queries(w.Q, ix.A, ix.compute, Qp=b["Qp"], workspace=b["pws"])
        sc = glv.glv_score_candidates(b["Qp"], ix.Xred, ix.row_stride, ix.scales, ix.dt, ix.tags, w.off, w.ids)
        allsc = sc.cpu().numpy()
        got = np.concatenate([allsc[offn[j]:offn[j + 1]] for j in qsel])
        rel = np.abs(got - red)[same] / scale[same]
        errs[st] = {"max_rel": float(rel.max()), "mean_rel": float(rel.mean()),
                    "p99_rel": float(np.quantile(rel, 0.99))}
    return errs


def kappa_sweep_block(glv, idx, w, stores, kaps, sp, red, exact, qsel, counts, args, flush, world):
    """Each store at re-rank depths kappa in kaps: queries/s of the whole step and recall of the
    final top 10 against the oracle pipeline at that kappa (R1) and against the exact top 10
    (R2).  Equal recall: each store at the smallest kappa whose R2 reaches 0.9."""
    nq = w.Q.shape[0]
    sweep, best = {}, {}
    for st in stores:
        ix = idx[st]
        rows = []
        for kap in kaps:
            if kap < w.k:
                continue
            r = time_search(glv, ix, w, kap, min(args.steps, 10), min(args.warmup, 2), flush, world)
            b = ix._buffers(nq, int(w.off[-1]), kap, w.k)
            _, fi = search_step(glv, ix, w, b, kap)
            got = fi.cpu().numpy()[qsel]
            rows.append({"kappa": kap, "value": r["value"], "ms_per_step": r["ms_per_step"],
                         "kernels_ms": r["kernels_ms"],
                         "R1": recall_by_kind(got, oracle_final_ids(sp, red, kap, w.k), counts)["all"],
                         "R2": recall_by_kind(got, exact, counts)})
        sweep[st] = rows
        pick = {}
        for key, get in (("R1", lambda row: row["R1"]), ("R2", lambda row: row["R2"]["all"])):
            ok = [row for row in rows if get(row) >= 0.9]
            pick[key] = ({"kappa": ok[0]["kappa"], "value": ok[0]["value"], "recall": get(ok[0])} if ok else
                         {"kappa": None, "note": f"no kappa of the sweep reaches {key} >= 0.9"})
        best[st] = pick
    return sweep, {"target": "the smallest kappa of the sweep whose final 10-recall@10 reaches 0.9: R1 against the "
                             "FP64 oracle pipeline at that kappa (the metric), R2 against the exact top 10 over the "
                             "candidates",
                   "by_store": best}


def cpu_baseline_block(w, sp, qsel, args):
    """The FP64 oracle's whole search of a bounded sample of the queries, timed on the host
    cores: all threads and one thread."""
    import numpy as np
    import oracle
    nq = w.Q.shape[0]
    if args.cpu_sample != len(qsel):
        rng = np.random.default_rng(777)
        csel = np.sort(rng.choice(nq, size=min(args.cpu_sample, nq), replace=False))
        sp = oracle_subproblem(w, csel)
    else:
        csel = qsel
    nthreads = os.cpu_count() or 1
    oracle.set_threads(nthreads)
    t_all, _, _ = oracle_search_timed(sp, w.kappa, w.k, repeats=3)
    cores = oracle.get_threads()
    n1 = max(1, len(csel) // 8)
    sub = dict(sp)
    sub["Q"] = sp["Q"][:n1]
    sub["off"] = sp["off"][:n1 + 1]
    sub["ids"] = sp["ids"][:int(sp["off"][n1])]
    oracle.set_threads(1)
    t_one, _, _ = oracle_search_timed(sub, w.kappa, w.k, repeats=1)
    oracle.set_threads(nthreads)
    return {"value": len(csel) / t_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{len(csel)} of the {nq} queries (all their candidates); reduced rows precomputed untimed "
                      f"for the {len(sp['uniq'])} rows they touch; best of 3",
            "single_thread": {"value": n1 / t_one, "unit": UNIT, "cores": 1,
                              "sample": f"the first {n1} of those queries, one run"}}


def run_glv(args):
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
    from paper_2410_22347_gb300 import glv

    peaks = measured_peaks()
    peaks["tf32_tflops"] = measure_tf32_peak(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2
    head_store, others = STORES.get(args.workload, ("bf16", ""))
    store = args.store or head_store
    compare = others if args.compare_stores is None else args.compare_stores
    stores = [store] + [s for s in compare.split(",") if s and s not in (store, "none")]
    common = dict(dev=dev, rank=rank, world=world, local=local, flush=flush, peaks=peaks)
    head = measure_workload(args.workload, args, stores=stores, headline=True, overrides=args.overrides, **common)
    configs = {}
    if args.configs == "auto":
        extra = EXTRA_CONFIGS if (args.workload == HEADLINE and not args.overrides) else ()
    else:
        extra = tuple(c for c in args.configs.split(",") if c and c != "none")
    for name in extra:
        hs, ot = STORES[name]
        st = [hs] + [s for s in ot.split(",") if s]
        cfg = measure_workload(name, args, stores=st, headline=False, overrides={}, **common)
        cfg.pop("_results")
        cfg.pop("_launches_per_step")
        configs[name] = cfg
    if world > 1:
        dist.barrier()
    if rank != 0:
        return 0

    res = head.pop("_results")
    lps = head.pop("_launches_per_step")
    hs = head["stores"][store]
    rec = head.get("recall_10at10", {}).get(store, {}).get("R1_vs_oracle_pipeline", {}).get("all")
    idx_compute = head["projection"].get(store, {}).get("operands", "")
    line = {
        "metric": METRIC,
        "value": hs["value"],
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": hs["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": store,
        "data": "synthetic",
        "config": {"workload": args.workload, "overrides": args.overrides or None, "N": head["N"], "D": head["D"],
                   "d": head["d"], "C": head["C"], "queries_per_gpu": head["queries"],
                   "candidates_per_query": head["candidates_per_query"], "kappa": head["kappa"], "k": head["k"],
                   "reduced_row_store": store, "accumulate": "f32", "projection_operands": idx_compute,
                   "query_mix": head["query_mix"],
                   "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}"},
        "roofline": hs["roofline"],
        "kernels_ms": hs["kernels_ms"],
        "e2e": head.get("e2e"),
        "gpu_launches": lps[store] * args.steps,
        "clocks": head["clocks"],
        "modes": head["stores"],
        "autotune": head["autotune"],
        "build": head["build"],
        "projection": head["projection"],
        "peaks": {k: v for k, v in peaks.items()},
        "recall_10at10": head.get("recall_10at10"),
        "recall_sample": head.get("recall_sample"),
        "cpu_baseline": head.get("cpu_baseline"),
        "configs": configs or None,
    }
    for k in ("batching", "lazy_vs_eager", "score_error_vs_fp64_oracle", "kappa_sweep", "equal_recall"):
        if k in head:
            line[k] = head[k]
    if rec is not None and rec < 0.9:
        line["warning"] = f"{store} recall {rec:.3f} below 0.9"
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_learn(args):
    """Differentiation workload: 200k database + 20k OOD learning queries, D = 768, d = 128,
    C = 16.  Times the FP64 second moments, the LeanVec-Sphering initialisation (host
    Cholesky and eigendecompositions) and refinement minibatches of 4096 pairs (forward,
    loss, backward and Adam, all in the library's kernels), and checks one minibatch gradient
    against the FP64 oracle."""
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
    adam = [(torch.zeros_like(A), torch.zeros_like(A)), (torch.zeros_like(B), torch.zeros_like(B))]
    nstep = [0]

    def minibatch():
        qi = torch.randint(0, w.Q.shape[0], (P,), generator=g, device=dev, dtype=torch.int32)
        xi = torch.randint(0, n, (P,), generator=g, device=dev, dtype=torch.int32)
        A.grad = None
        B.grad = None
        loss = learn.pair_loss(A, B, w.Q, w.X, tags, qi, xi)
        loss.backward()
        nstep[0] += 1
        with torch.no_grad():
            for prm, (m, v) in zip((A, B), adam):
                learn.glv_adam_step(prm, prm.grad, m, v, nstep[0], 1e-4)
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
    _, gp = learn.glv_pair_loss(s, t, want_loss=False, want_grad=True)
    dA, dB = learn.glv_pair_backward(w.Q, w.X, tags, C, qi, xi, u, v, gp)
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
