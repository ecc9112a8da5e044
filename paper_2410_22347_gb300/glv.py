"""Thin Python binding of libglv (the C ABI in include/glv.h).

Argument marshalling only: every step of the search path runs in the library's CUDA
kernels.  Functions carry the C names and take torch CUDA tensors (for their device
memory) plus the current torch CUDA stream; each checks shapes/dtypes, passes raw
pointers, and raises ``GlvError`` on a non-OK status.  Importing this module loads
``libglv.so`` and fails loudly if it is missing or broken: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build_lib

GLV_OK, GLV_ERR_INVALID_ARG, GLV_ERR_BAD_ID, GLV_ERR_UNSUPPORTED, GLV_ERR_CUDA, GLV_ERR_TIMEOUT = range(6)
GLV_F32, GLV_BF16, GLV_FP8_E4M3 = 0, 1, 2
GLV_MAX_KAPPA = 1024
DTYPES = {"f32": GLV_F32, "bf16": GLV_BF16, "fp8": GLV_FP8_E4M3}

LIB_PATH = build_lib.LIB


class GlvError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        super().__init__(f"{fn} failed: {status_string(status)} (status {status})")


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libglv.so not built ({LIB_PATH}); run __graft_entry__.build() or "
                          "python -m paper_2410_22347_gb300.build_lib")
    lib = ctypes.CDLL(LIB_PATH)
    P, i64, i32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t
    sig = {
        "glv_abi_version": (i32, []),
        "glv_last_device_status": (i32, [P, P]),
        "glv_status_string": (ctypes.c_char_p, [i32]),
        "glv_min_row_stride": (i64, [i32, i32]),
        "glv_assign_tags": (i32, [P, i64, i32, P, i32, P, P, P]),
        "glv_kmeans_workspace_size": (sz, [i64, i32, i32]),
        "glv_kmeans_update": (i32, [P, i64, i32, P, i32, P, P, P, P, P]),
        "glv_build_reduced_workspace_size": (sz, [i64, i32]),
        "glv_build_reduced": (i32, [P, i64, i32, P, P, i32, i32, i32, P, i64, P, P, P, P]),
        "glv_build_reduced_noalloc": (i32, [P, i64, i32, P, P, i32, i32, i32, P, i64, P, P, P]),
        "glv_project_queries_workspace_size": (sz, [i64, i32, i32, i32, i32]),
        "glv_project_queries": (i32, [P, i64, i32, P, i32, i32, i32, P, P, P, P]),
        "glv_score_candidates": (i32, [P, i64, i32, i32, P, i64, P, i32, P, i64, P, P, P, P, P]),
        "glv_score_topk_workspace_size": (sz, [i64, i64]),
        "glv_score_topk": (i32, [P, i64, i32, i32, P, i64, P, i32, P, i64, P, P, i64, i32, P, P, P, P, P, P]),
        "glv_topk": (i32, [P, P, P, i64, i32, P, P, P]),
        "glv_score_lazy": (i32, [P, i64, i32, P, i32, i32, P, i64, P, i32, P, i64, P, P, P, P, P, P]),
        "glv_set_score_config": (i32, [i32, i32, i32, i32, i32]),
        "glv_get_score_config": (i32, [i32, i32, P, P, P, P]),
        "glv_rerank": (i32, [P, i64, i32, P, i64, P, i32, i32, P, P, P, P]),
        "glv_gather_rows": (i32, [P, i64, i64, P, i64, P, P, P]),
        "glv_check_bounded_wait": (i32, [ctypes.c_uint32, P, P]),
        "glv_search_workspace_size": (sz, [i64, i32, i32, i32, i32, i64, i32]),
        "glv_search": (i32, [P, i64, i32, P, i64, P, i32, i32, i32, P, i64, P, i32, P, P, P, i64, i32, i32,
                             P, P, P, P, P]),
        "glv_search_host_workspace_size": (sz, [i64, i32, i32, i32, i32, i64, i32, i32]),
        "glv_search_host": (i32, [P, i64, i32, P, i64, P, i32, i32, i32, P, i64, P, i32, P, P, P, i64, i32, i32,
                                  P, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def lib() -> ctypes.CDLL:
    return _lib


def status_string(s: int) -> str:
    return _lib.glv_status_string(int(s)).decode()


def glv_last_device_status(d_status, stream=None) -> int:
    """Waits for the stream and returns the device status word (0 = no error recorded)."""
    _need(d_status, torch.int32, "d_status", 1)
    return int(_lib.glv_last_device_status(_ptr(d_status), _stream(stream)))


def abi_version() -> int:
    return int(_lib.glv_abi_version())


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _need(t: torch.Tensor, dtype, name: str, ndim: int | None = None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if ndim is not None and t.dim() != ndim:
        raise ValueError(f"{name} must have {ndim} dims")


def _check(fn: str, st: int):
    if st != GLV_OK:
        raise GlvError(fn, st)


def min_row_stride(d: int, dt: int) -> int:
    return int(_lib.glv_min_row_stride(int(d), int(dt)))


def elem_bytes(dt: int) -> int:
    return {GLV_F32: 4, GLV_BF16: 2, GLV_FP8_E4M3: 1}[dt]


# ---------------------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------------------

def glv_assign_tags(X: torch.Tensor, mu: torch.Tensor, tags: torch.Tensor | None = None,
                    best_ip: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    _need(X, torch.float32, "X", 2)
    _need(mu, torch.float32, "mu", 2)
    N, D = X.shape
    if tags is None:
        tags = torch.empty(N, dtype=torch.uint16, device=X.device)
    _need(tags, torch.uint16, "tags", 1)
    if best_ip is not None:
        _need(best_ip, torch.float32, "best_ip", 1)
    _check("glv_assign_tags", _lib.glv_assign_tags(_ptr(X), N, D, _ptr(mu), mu.shape[0], _ptr(tags),
                                                   _ptr(best_ip), _stream(stream)))
    return tags


def glv_kmeans_update(X, tags, mu, counts=None, d_status=None, stream=None):
    """Spherical k-means M-step in place on mu (C x D); returns (mu, counts)."""
    _need(X, torch.float32, "X", 2)
    _need(tags, torch.uint16, "tags", 1)
    _need(mu, torch.float32, "mu", 2)
    N, D = X.shape
    C = mu.shape[0]
    if counts is None:
        counts = torch.empty(C, dtype=torch.int32, device=X.device)
    ws = torch.empty(max(int(_lib.glv_kmeans_workspace_size(N, D, C)), 1), dtype=torch.uint8, device=X.device)
    _check("glv_kmeans_update", _lib.glv_kmeans_update(_ptr(X), N, D, _ptr(tags), C, _ptr(mu), _ptr(counts),
                                                       _ptr(ws), _ptr(d_status), _stream(stream)))
    return mu, counts


def glv_build_reduced(X, tags, B, dt: int, Xred=None, row_stride: int | None = None, scales=None,
                      workspace=None, d_status=None, stream=None):
    """Returns (Xred uint8 [N, row_stride], scales or None)."""
    _need(X, torch.float32, "X", 2)
    _need(tags, torch.uint16, "tags", 1)
    _need(B, torch.float32, "B", 3)
    N, D = X.shape
    C, d, _ = B.shape
    if row_stride is None:
        row_stride = min_row_stride(d, dt)
    if Xred is None:
        Xred = torch.empty(N, row_stride, dtype=torch.uint8, device=X.device)
    if dt == GLV_FP8_E4M3 and scales is None:
        scales = torch.empty(N, dtype=torch.float32, device=X.device)
    if workspace is None:
        ws = int(_lib.glv_build_reduced_workspace_size(N, C))
        workspace = torch.empty(max(ws, 1), dtype=torch.uint8, device=X.device)
    _check("glv_build_reduced",
           _lib.glv_build_reduced(_ptr(X), N, D, _ptr(tags), _ptr(B), C, d, dt, _ptr(Xred),
                                  row_stride, _ptr(scales), _ptr(workspace), _ptr(d_status),
                                  _stream(stream)))
    return Xred, scales


def glv_build_reduced_noalloc(X, tags, B, dt: int, Xred, row_stride: int, scales=None, d_status=None,
                              stream=None):
    """glv_build_reduced without a workspace: the caller passes only inputs and outputs
    (Xred, and scales for FP8); the scratch is the library's own fixed device array."""
    _need(X, torch.float32, "X", 2)
    _need(tags, torch.uint16, "tags", 1)
    _need(B, torch.float32, "B", 3)
    N, D = X.shape
    C, d, _ = B.shape
    _check("glv_build_reduced_noalloc",
           _lib.glv_build_reduced_noalloc(_ptr(X), N, D, _ptr(tags), _ptr(B), C, d, dt, _ptr(Xred),
                                          row_stride, _ptr(scales), _ptr(d_status), _stream(stream)))
    return Xred, scales


def project_workspace_bytes(nq: int, D: int, C: int, d: int, compute: int) -> int:
    return int(_lib.glv_project_queries_workspace_size(nq, D, C, d, compute))


def glv_project_queries(Q, A, compute: int = GLV_F32, Qp=None, workspace=None, d_status=None,
                        stream=None, tensor_cores: bool = True):
    """Qp = Q . [A_1; ...; A_C]^T.  With tensor_cores (default) a workspace is allocated if not
    given; tensor_cores=False with compute=GLV_F32 selects the SIMT FP32 kernel."""
    _need(Q, torch.float32, "Q", 2)
    _need(A, torch.float32, "A", 3)
    nq, D = Q.shape
    C, d, _ = A.shape
    if Qp is None:
        Qp = torch.empty(nq, C, d, dtype=torch.float32, device=Q.device)
    if workspace is None and (tensor_cores or compute != GLV_F32):
        workspace = torch.empty(max(project_workspace_bytes(nq, D, C, d, compute), 1), dtype=torch.uint8,
                                device=Q.device)
    _check("glv_project_queries",
           _lib.glv_project_queries(_ptr(Q), nq, D, _ptr(A), C, d, compute, _ptr(Qp), _ptr(workspace),
                                    _ptr(d_status), _stream(stream)))
    return Qp


def glv_score_candidates(Qp, Xred, row_stride: int, scales, dt: int, tags, off, ids, scores=None,
                         d_status=None, stream=None, d: int | None = None):
    _need(Qp, torch.float32, "Qp", 3)
    _need(tags, torch.uint16, "tags", 1)
    _need(off, torch.int64, "cand_off", 1)
    _need(ids, torch.int32, "cand_ids", 1)
    nq, C, dq = Qp.shape
    d = dq if d is None else d
    N = tags.shape[0]
    if scores is None:
        scores = torch.empty(ids.shape[0], dtype=torch.float32, device=Qp.device)
    _check("glv_score_candidates",
           _lib.glv_score_candidates(_ptr(Qp), nq, C, d, _ptr(Xred), row_stride, _ptr(scales), dt,
                                     _ptr(tags), N, _ptr(off), _ptr(ids), _ptr(scores),
                                     _ptr(d_status), _stream(stream)))
    return scores


def glv_score_lazy(Q, A, Xred, row_stride: int, scales, dt: int, tags, off, ids, scores=None, visited=None,
                   d_status=None, stream=None):
    """Algorithm 3 (lazy): scores with q_c = A_c q formed per visited cluster inside the
    kernel.  Returns (scores, visited-cluster count per query)."""
    _need(Q, torch.float32, "Q", 2)
    _need(A, torch.float32, "A", 3)
    _need(tags, torch.uint16, "tags", 1)
    _need(off, torch.int64, "cand_off", 1)
    _need(ids, torch.int32, "cand_ids", 1)
    nq, D = Q.shape
    C, d, _ = A.shape
    if scores is None:
        scores = torch.empty(max(ids.shape[0], 1), dtype=torch.float32, device=Q.device)
    if visited is None:
        visited = torch.empty(nq, dtype=torch.int32, device=Q.device)
    _check("glv_score_lazy", _lib.glv_score_lazy(_ptr(Q), nq, D, _ptr(A), C, d, _ptr(Xred), row_stride, _ptr(scales),
                                                 dt, _ptr(tags), tags.shape[0], _ptr(off), _ptr(ids), _ptr(scores),
                                                 _ptr(visited), _ptr(d_status), _stream(stream)))
    return scores, visited


def score_topk_workspace_bytes(nq: int, n_candidates: int) -> int:
    return int(_lib.glv_score_topk_workspace_size(int(nq), int(n_candidates)))


def glv_score_topk(Qp, Xred, row_stride: int, scales, dt: int, tags, off, ids, kappa: int, scores_scratch=None,
                   out_s=None, out_id=None, d_status=None, stream=None, d: int | None = None, workspace=None):
    """Fused scoring + top-kappa (same results as glv_score_candidates then glv_topk)."""
    _need(Qp, torch.float32, "Qp", 3)
    _need(tags, torch.uint16, "tags", 1)
    _need(off, torch.int64, "cand_off", 1)
    _need(ids, torch.int32, "cand_ids", 1)
    nq, C, dq = Qp.shape
    d = dq if d is None else d
    N = tags.shape[0]
    n_cand = ids.shape[0]
    if scores_scratch is None:
        scores_scratch = torch.empty(max(n_cand, 1), dtype=torch.float32, device=Qp.device)
    if workspace is None:
        workspace = torch.empty(max(score_topk_workspace_bytes(nq, n_cand), 1), dtype=torch.uint8, device=Qp.device)
    if out_s is None:
        out_s = torch.empty(nq, kappa, dtype=torch.float32, device=Qp.device)
    if out_id is None:
        out_id = torch.empty(nq, kappa, dtype=torch.int32, device=Qp.device)
    _check("glv_score_topk",
           _lib.glv_score_topk(_ptr(Qp), nq, C, d, _ptr(Xred), row_stride, _ptr(scales), dt, _ptr(tags), N,
                               _ptr(off), _ptr(ids), n_cand, kappa, _ptr(scores_scratch), _ptr(workspace),
                               _ptr(out_s), _ptr(out_id), _ptr(d_status), _stream(stream)))
    return out_s, out_id


SCORE_GROUPS = {GLV_F32: (4, 8, 16, 32), GLV_BF16: (4, 8, 16, 32), GLV_FP8_E4M3: (2, 4, 8, 32)}


GATHER_MODES = (0, 1, 2)  # registers, registers pipelined, bulk copies into shared memory

# shared-memory carveout caps the autotuner tries, KB (164 leaves about 92 KB of the SM's
# 256 KB to L1 for the rows in flight).  The driver's choice (0, still accepted by
# glv_set_score_config) is not offered: alone it times within 0.1% of a cap, but when searches
# run on two streams at once (HostSearchPipeline) it made the pipelined step slower than one
# batch run alone (measured 2.96-3.02 ms against 1.79-1.84 ms with a cap, per 10k queries).
SCORE_CARVEOUTS = (132, 164)

# fused-call schedules, bit 0: planned work items (long lists cut into chunks), else one CTA per
# query; bit 1: wide CTAs (512 threads, twice the keys on chip); bit 2: L2 prefetch of the next
# candidate's row
SCORE_SCHEDULES = (1, 0, 3, 2, 5, 4, 7, 6)


def glv_set_score_config(dt: int, lanes_per_candidate: int, gather_mode: int, smem_carveout_kb: int = 0,
                         schedule: int = 1) -> None:
    _check("glv_set_score_config", _lib.glv_set_score_config(dt, int(lanes_per_candidate), int(gather_mode),
                                                              int(smem_carveout_kb), int(schedule)))


def glv_get_score_config(dt: int, d: int) -> tuple[int, int, int, int]:
    """(lanes per candidate, gather mode, carveout cap KB, fused schedule) used for rows of width d."""
    g, p, c, h = (ctypes.c_int32(0) for _ in range(4))
    _check("glv_get_score_config", _lib.glv_get_score_config(dt, int(d), ctypes.byref(g), ctypes.byref(p),
                                                              ctypes.byref(c), ctypes.byref(h)))
    return int(g.value), int(p.value), int(c.value), int(h.value)


def glv_topk(scores, off, ids, kappa: int, out_s=None, out_id=None, stream=None):
    _need(scores, torch.float32, "scores", 1)
    _need(off, torch.int64, "cand_off", 1)
    _need(ids, torch.int32, "cand_ids", 1)
    nq = off.shape[0] - 1
    if out_s is None:
        out_s = torch.empty(nq, kappa, dtype=torch.float32, device=scores.device)
    if out_id is None:
        out_id = torch.empty(nq, kappa, dtype=torch.int32, device=scores.device)
    _check("glv_topk", _lib.glv_topk(_ptr(scores), _ptr(off), _ptr(ids), nq, kappa, _ptr(out_s),
                                     _ptr(out_id), _stream(stream)))
    return out_s, out_id


def glv_rerank(X, Q, surv_id, k: int, out_s=None, out_id=None, d_status=None, stream=None):
    _need(X, torch.float32, "X", 2)
    _need(Q, torch.float32, "Q", 2)
    _need(surv_id, torch.int32, "surv_id", 2)
    N, D = X.shape
    nq, kappa = surv_id.shape
    if out_s is None:
        out_s = torch.empty(nq, k, dtype=torch.float32, device=Q.device)
    if out_id is None:
        out_id = torch.empty(nq, k, dtype=torch.int32, device=Q.device)
    _check("glv_rerank", _lib.glv_rerank(_ptr(X), N, D, _ptr(Q), nq, _ptr(surv_id), kappa, k,
                                         _ptr(out_s), _ptr(out_id), _ptr(d_status), _stream(stream)))
    return out_s, out_id


def glv_gather_rows(rows, row_bytes: int, ids, out=None, d_status=None, stream=None):
    """Gather calibration: every row ids[p] of the row-major store ``rows`` (uint8, n_rows x
    row_bytes) read whole, out[p] = its words summed as floats (no other arithmetic)."""
    _need(rows, torch.uint8, "rows")
    _need(ids, torch.int32, "ids", 1)
    n_rows = rows.numel() // row_bytes
    if out is None:
        out = torch.empty(ids.shape[0], dtype=torch.float32, device=ids.device)
    _check("glv_gather_rows", _lib.glv_gather_rows(_ptr(rows), int(row_bytes), n_rows, _ptr(ids), ids.shape[0],
                                                   _ptr(out), _ptr(d_status), _stream(stream)))
    return out


def glv_search(X, Q, A, compute: int, Xred, row_stride: int, scales, dt: int, tags, off, ids, kappa: int, k: int,
               workspace=None, out_s=None, out_id=None, d_status=None, stream=None):
    """The whole search in one library call (projection -> fused score + top-kappa -> re-rank)."""
    _need(X, torch.float32, "X", 2)
    _need(Q, torch.float32, "Q", 2)
    _need(A, torch.float32, "A", 3)
    _need(tags, torch.uint16, "tags", 1)
    _need(off, torch.int64, "cand_off", 1)
    _need(ids, torch.int32, "cand_ids", 1)
    N, D = X.shape
    nq = Q.shape[0]
    C, d, _ = A.shape
    n_cand = ids.shape[0]
    if workspace is None:
        ws = int(_lib.glv_search_workspace_size(nq, D, C, d, compute, n_cand, kappa))
        workspace = torch.empty(max(ws, 1), dtype=torch.uint8, device=Q.device)
    if out_s is None:
        out_s = torch.empty(nq, k, dtype=torch.float32, device=Q.device)
    if out_id is None:
        out_id = torch.empty(nq, k, dtype=torch.int32, device=Q.device)
    _check("glv_search", _lib.glv_search(_ptr(X), N, D, _ptr(Q), nq, _ptr(A), C, d, compute, _ptr(Xred), row_stride,
                                         _ptr(scales), dt, _ptr(tags), _ptr(off), _ptr(ids), n_cand, kappa, k,
                                         _ptr(workspace), _ptr(out_s), _ptr(out_id), _ptr(d_status),
                                         _stream(stream)))
    return out_s, out_id


def search_host_workspace_bytes(nq: int, D: int, C: int, d: int, compute: int, n_candidates: int, kappa: int,
                                k: int) -> int:
    return int(_lib.glv_search_host_workspace_size(nq, D, C, d, compute, n_candidates, kappa, k))


def _need_host(t: torch.Tensor, dtype, name: str):
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a host (CPU) tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def glv_search_host(X, Q_h, A, compute: int, Xred, row_stride: int, scales, dt: int, tags, off_h, ids_h, kappa: int,
                    k: int, workspace, out_s_h, out_id_h, d_status=None, stream=None):
    """glv_search from host buffers: Q_h, off_h, ids_h in and out_s_h, out_id_h out are host tensors
    (pinned for asynchronous copies); the copies and the search are enqueued on ``stream``."""
    _need(X, torch.float32, "X", 2)
    _need(A, torch.float32, "A", 3)
    _need(tags, torch.uint16, "tags", 1)
    _need_host(Q_h, torch.float32, "Q_h")
    _need_host(off_h, torch.int64, "off_h")
    _need_host(ids_h, torch.int32, "ids_h")
    _need_host(out_s_h, torch.float32, "out_s_h")
    _need_host(out_id_h, torch.int32, "out_id_h")
    N, D = X.shape
    nq = Q_h.shape[0]
    C, d, _ = A.shape
    _check("glv_search_host", _lib.glv_search_host(
        _ptr(X), N, D, ctypes.c_void_p(Q_h.data_ptr()), nq, _ptr(A), C, d, compute, _ptr(Xred), row_stride,
        _ptr(scales), dt, _ptr(tags), ctypes.c_void_p(off_h.data_ptr()), ctypes.c_void_p(ids_h.data_ptr()),
        ids_h.shape[0], kappa, k, _ptr(workspace), ctypes.c_void_p(out_s_h.data_ptr()),
        ctypes.c_void_p(out_id_h.data_ptr()), _ptr(d_status), _stream(stream)))
    return out_s_h, out_id_h


def glv_check_bounded_wait(limit_us: int, d_status, stream=None) -> None:
    """Runs a device wait on a barrier nothing completes, bounded by limit_us; the status word
    receives GLV_ERR_TIMEOUT when the limit passes."""
    _need(d_status, torch.int32, "d_status", 1)
    _check("glv_check_bounded_wait", _lib.glv_check_bounded_wait(int(limit_us), _ptr(d_status), _stream(stream)))
