"""Autotuner for the gather-score kernels.

The scoring kernels are instantiated for several lanes-per-candidate group sizes and three
row-gather modes (register loads, pipelined register loads, bulk copies into shared memory;
see csrc/score_launch.cuh), and each launch may cap the SM's shared-memory carveout (fewer
CTAs, more L1 for the rows in flight).  Which combination keeps
HBM busiest depends on the row width, the store type, the candidate-list lengths and the
GPU, so ``tune_score`` times every offered configuration of the fused score + top-kappa
call on the caller's own workload (CUDA events on the launching stream, L2 evicted between
repetitions), installs the fastest through ``glv_set_score_config`` and caches it in a JSON
file keyed by GPU name, store type, row width, cluster count and mean list length.
"""
from __future__ import annotations

import json
import os

import torch

from . import glv

CACHE = os.environ.get("GLV_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "glv", "autotune.json"))


def _key(dt: int, d: int, C: int, mean_len: float) -> str:
    name = torch.cuda.get_device_name()
    return f"v7|{name}|dt{dt}|d{d}|C{C}|L{int(round(mean_len, -1))}"


def _load_cache() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _save_cache(c: dict) -> None:
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE)
    except OSError:
        pass


def configurations(dt: int):
    # the fused call gathers into registers (modes 0 and 1; it maps the bulk mode to 0); the
    # wide schedules (bit 1) exist for mode 0 and the two smaller lane counts
    for sched in glv.SCORE_SCHEDULES:
        for G in glv.SCORE_GROUPS[dt]:
            for mode in (0, 1):
                if (sched & 2) and (mode != 0 or G not in glv.SCORE_GROUPS[dt][:2]):
                    continue
                for carve in glv.SCORE_CARVEOUTS:
                    yield G, mode, carve, sched


def tune_score(index, Q, off, ids, kappa: int, reps: int = 5, use_cache: bool = True, verbose: bool = False):
    """Pick the fastest scoring configuration for ``index``'s store on this workload.
    Returns (G, gather_mode, carveout_kb, schedule, table) where table maps
    "G/mode/carveout/schedule" to the mean ms per call."""
    nq = Q.shape[0]
    mean_len = ids.shape[0] / max(nq, 1)
    key = _key(index.dt, index.d, index.C, mean_len) + f"|k{kappa}"
    cache = _load_cache() if use_cache else {}
    if key in cache:
        e = cache[key]
        G, mode, carve, sched = e["G"], e["mode"], e.get("carve", 0), e.get("sched", 1)
        glv.glv_set_score_config(index.dt, G, mode, carve, sched)
        return G, mode, carve, sched, e.get("table", {})
    b = index._buffers(nq, ids.shape[0], kappa, kappa)
    glv.glv_project_queries(Q, index.A, index.compute, Qp=b["Qp"], workspace=b["pws"])
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=Q.device)  # 256 MB > L2
    table = {}
    seen = set()
    for G, mode, carve, sched in configurations(index.dt):
        glv.glv_set_score_config(index.dt, G, mode, carve, sched)
        eff = glv.glv_get_score_config(index.dt, index.d)
        if eff in seen:  # this choice cannot serve the row width; it maps onto one already timed
            continue
        seen.add(eff)

        def run():
            glv.glv_score_topk(b["Qp"], index.Xred, index.row_stride, index.scales, index.dt, index.tags, off,
                               ids, kappa, scores_scratch=b["scores"], workspace=b["tws"], out_s=b["ts"], out_id=b["ti"])
        run()
        torch.cuda.synchronize()
        ms = 0.0
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run()
            e1.record()
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        table["/".join(str(x) for x in eff)] = ms / reps
        if verbose:
            print(f"  score config G={eff[0]:2d} mode={eff[1]} carveout={eff[2]} schedule={eff[3]}: "
                  f"{ms / reps:.3f} ms", flush=True)
    best = min(table, key=table.get)
    G, mode, carve, sched = (int(x) for x in best.split("/"))
    glv.glv_set_score_config(index.dt, G, mode, carve, sched)
    if use_cache:
        cache[key] = {"G": G, "mode": mode, "carve": carve, "sched": sched, "table": table}
        _save_cache(cache)
    return G, mode, carve, sched, table
