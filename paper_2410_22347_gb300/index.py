"""User-facing GleanVec index on one GPU, built on the C ABI.

``GleanVecIndex`` owns the device-resident database X, cluster tags, the per-cluster
(A_c, B_c) and the reduced store x_i^low = B_{c_i} x_i, and runs the eager multi-step
search of Algorithm 1 / Algorithm 4 with four library calls:

    glv_project_queries -> glv_score_topk (fused scoring + top-kappa) -> glv_rerank

``search`` takes device tensors; ``search_host`` takes host tensors (pinned when given
pinned memory), copies them in, searches and copies the top-k back on the same stream.
``HostSearchPipeline`` streams a sequence of host-resident batches: the copies of the next
batch run on a copy stream while the current one is searched.  Every step runs in libglv's
kernels; torch only provides device memory and the streams.
"""
from __future__ import annotations

import torch

from . import glv


class GleanVecIndex:
    def __init__(self, X: torch.Tensor, A: torch.Tensor, B: torch.Tensor, *, tags: torch.Tensor | None = None,
                 mu: torch.Tensor | None = None, store: str = "bf16", project: str | None = None, stream=None):
        if tags is None:
            if mu is None:
                raise ValueError("give cluster tags or landmarks mu")
            tags = glv.glv_assign_tags(X, mu, stream=stream)
        self.X, self.A, self.B, self.tags = X, A, B, tags
        self.N, self.D = X.shape
        self.C, self.d, _ = A.shape
        self.dt = glv.DTYPES[store]
        # low-precision stores pair with BF16 projection operands; the FP32 store keeps FP32
        self.compute = glv.DTYPES[project if project is not None else ("f32" if store == "f32" else "bf16")]
        self.row_stride = glv.min_row_stride(self.d, self.dt)
        self.status = torch.zeros(1, dtype=torch.int32, device=X.device)
        self.Xred, self.scales = glv.glv_build_reduced(X, tags, B, self.dt, d_status=self.status,
                                                       stream=stream)
        self._buf = {}
        self._h2d = {}

    def _buffers(self, nq: int, total: int, kappa: int, k: int):
        key = (nq, total, kappa, k)
        b = self._buf.get(key)
        if b is None:
            dev = self.X.device
            b = dict(
                Qp=torch.empty(nq, self.C, self.d, dtype=torch.float32, device=dev),
                pws=torch.empty(max(glv.project_workspace_bytes(nq, self.D, self.C, self.d, self.compute), 1),
                                dtype=torch.uint8, device=dev),
                scores=torch.empty(max(total, 1), dtype=torch.float32, device=dev),
                tws=torch.empty(max(glv.score_topk_workspace_bytes(nq, total), 1), dtype=torch.uint8, device=dev),
                ts=torch.empty(nq, kappa, dtype=torch.float32, device=dev),
                ti=torch.empty(nq, kappa, dtype=torch.int32, device=dev),
                fs=torch.empty(nq, k, dtype=torch.float32, device=dev),
                fi=torch.empty(nq, k, dtype=torch.int32, device=dev),
            )
            self._buf = {key: b}
        return b

    def search(self, Q: torch.Tensor, off: torch.Tensor, ids: torch.Tensor, kappa: int, k: int,
               stream=None):
        """Eager multi-step search of the CSR candidate lists (device tensors).  Returns
        (scores, ids) of shape nq x k.  kappa == 0: no re-rank (top k of reduced scores)."""
        nq = Q.shape[0]
        b = self._buffers(nq, ids.shape[0], max(kappa, k), k)
        glv.glv_project_queries(Q, self.A, self.compute, Qp=b["Qp"], workspace=b["pws"], d_status=self.status,
                                stream=stream)
        if kappa <= 0:
            glv.glv_score_topk(b["Qp"], self.Xred, self.row_stride, self.scales, self.dt, self.tags, off, ids, k,
                               scores_scratch=b["scores"], workspace=b["tws"], out_s=b["fs"], out_id=b["fi"],
                               d_status=self.status,
                               stream=stream)
            return b["fs"], b["fi"]
        glv.glv_score_topk(b["Qp"], self.Xred, self.row_stride, self.scales, self.dt, self.tags, off, ids, kappa,
                           scores_scratch=b["scores"], workspace=b["tws"], out_s=b["ts"], out_id=b["ti"],
                           d_status=self.status,
                           stream=stream)
        glv.glv_rerank(self.X, Q, b["ti"], k, out_s=b["fs"], out_id=b["fi"], d_status=self.status,
                       stream=stream)
        return b["fs"], b["fi"]

    def search_host(self, Q_h: torch.Tensor, off_h: torch.Tensor, ids_h: torch.Tensor, kappa: int, k: int,
                    out_s_h: torch.Tensor | None = None, out_id_h: torch.Tensor | None = None, stream=None):
        """Host-in, host-out search: copies the queries and candidate lists to the device,
        searches, copies the top-k back (asynchronously on the stream when the host
        tensors are pinned; call torch.cuda.synchronize / stream.synchronize to wait)."""
        dev = self.X.device
        st = stream if stream is not None else torch.cuda.current_stream()
        with torch.cuda.stream(st):
            key = (tuple(Q_h.shape), tuple(off_h.shape), tuple(ids_h.shape))
            d = self._h2d.get(key)
            if d is None:
                d = (torch.empty(Q_h.shape, dtype=torch.float32, device=dev),
                     torch.empty(off_h.shape, dtype=torch.int64, device=dev),
                     torch.empty(ids_h.shape, dtype=torch.int32, device=dev))
                self._h2d = {key: d}
            Qd, offd, idsd = d
            Qd.copy_(Q_h, non_blocking=True)
            offd.copy_(off_h, non_blocking=True)
            idsd.copy_(ids_h, non_blocking=True)
            fs, fi = self.search(Qd, offd, idsd, kappa, k, stream=st)
            if out_s_h is None:
                out_s_h = torch.empty(fs.shape, dtype=fs.dtype, pin_memory=True)
                out_id_h = torch.empty(fi.shape, dtype=fi.dtype, pin_memory=True)
            out_s_h.copy_(fs, non_blocking=True)
            out_id_h.copy_(fi, non_blocking=True)
        return out_s_h, out_id_h

    def device_status(self) -> int:
        """First device-side error recorded since the last reset (0 = none); synchronises."""
        return int(self.status.item())

    def reset_status(self):
        self.status.zero_()


class HostSearchPipeline:
    """Streams host-resident query batches through an index.

    ``submit`` enqueues one batch (pinned host tensors: queries, CSR candidate lists, and the
    top-k outputs) and returns at once.  The host-to-device copies of a batch run on a copy
    stream, so they overlap the search of the batch before it on the compute stream; the
    top-k of each batch is copied back on the compute stream right after its search.
    Device input buffers rotate over ``depth`` slots: a slot is refilled only after the
    search that read it has finished.  ``synchronize`` waits for everything submitted.
    """

    def __init__(self, index: GleanVecIndex, kappa: int, k: int, depth: int = 2, stream=None):
        if depth < 2:
            raise ValueError("depth >= 2 (one batch copying while another is searched)")
        self.ix, self.kappa, self.k, self.depth = index, kappa, k, depth
        self.compute = stream if stream is not None else torch.cuda.current_stream()
        self.copy = torch.cuda.Stream(device=index.X.device)
        self._slots = [None] * depth
        self._done = [None] * depth
        self._n = 0

    def _slot(self, s: int, Q_h, off_h, ids_h):
        key = (tuple(Q_h.shape), tuple(off_h.shape), tuple(ids_h.shape))
        cur = self._slots[s]
        if cur is None or cur[0] != key:
            dev = self.ix.X.device
            cur = (key, torch.empty(Q_h.shape, dtype=torch.float32, device=dev),
                   torch.empty(off_h.shape, dtype=torch.int64, device=dev),
                   torch.empty(ids_h.shape, dtype=torch.int32, device=dev))
            self._slots[s] = cur
        return cur[1:]

    def begin(self):
        """Order the copy stream after the work already enqueued on the compute stream (for
        timing: an event recorded on the compute stream before begin() precedes every
        copy submitted after it)."""
        self.copy.wait_stream(self.compute)

    def submit(self, Q_h: torch.Tensor, off_h: torch.Tensor, ids_h: torch.Tensor, out_s_h: torch.Tensor,
               out_id_h: torch.Tensor) -> torch.cuda.Event:
        s = self._n % self.depth
        self._n += 1
        Qd, offd, idsd = self._slot(s, Q_h, off_h, ids_h)
        if self._done[s] is not None:
            self.copy.wait_event(self._done[s])   # the search that last read this slot
        with torch.cuda.stream(self.copy):
            Qd.copy_(Q_h, non_blocking=True)
            offd.copy_(off_h, non_blocking=True)
            idsd.copy_(ids_h, non_blocking=True)
            copied = torch.cuda.Event()
            copied.record(self.copy)
        self.compute.wait_event(copied)
        with torch.cuda.stream(self.compute):
            fs, fi = self.ix.search(Qd, offd, idsd, self.kappa, self.k, stream=self.compute)
            out_s_h.copy_(fs, non_blocking=True)
            out_id_h.copy_(fi, non_blocking=True)
            done = torch.cuda.Event()
            done.record(self.compute)
        self._done[s] = done
        return done

    def synchronize(self):
        self.compute.synchronize()
        self.copy.synchronize()
