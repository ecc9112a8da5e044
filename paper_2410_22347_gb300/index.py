"""User-facing GleanVec index on one GPU, built on the C ABI.

``GleanVecIndex`` owns the device-resident database X, cluster tags, the per-cluster
(A_c, B_c) and the reduced store x_i^low = B_{c_i} x_i, and runs the eager multi-step
search of Algorithm 1 / Algorithm 4 with four library calls:

    glv_project_queries -> glv_score_topk (fused scoring + top-kappa) -> glv_rerank

``search`` takes device tensors; ``search_host`` takes host tensors (pinned when given
pinned memory) and runs the library's host-buffer entry point, which copies them in, searches
and copies the top-k back on one stream.  ``HostSearchPipeline`` streams a sequence of
host-resident batches over alternating streams, so one batch's copies overlap another's
search.  Every step runs in libglv's
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
        """Host-in, host-out search through one library call (glv_search_host): the copies of
        the queries and candidate lists in, the search and the copy of the top-k out are all
        enqueued on the stream (asynchronous with pinned host tensors; synchronise the stream
        before reading the outputs)."""
        nq = Q_h.shape[0]
        if out_s_h is None:
            out_s_h = torch.empty(nq, k, dtype=torch.float32, pin_memory=True)
            out_id_h = torch.empty(nq, k, dtype=torch.int32, pin_memory=True)
        ws = self._host_workspace(nq, ids_h.shape[0], kappa, k, slot=0)
        glv.glv_search_host(self.X, Q_h, self.A, self.compute, self.Xred, self.row_stride, self.scales, self.dt,
                            self.tags, off_h, ids_h, kappa, k, ws, out_s_h, out_id_h, d_status=self.status,
                            stream=stream)
        return out_s_h, out_id_h

    def _host_workspace(self, nq: int, n_cand: int, kappa: int, k: int, slot: int):
        key = (nq, n_cand, kappa, k, slot)
        ws = self._h2d.get(key)
        if ws is None:
            nbytes = glv.search_host_workspace_bytes(nq, self.D, self.C, self.d, self.compute, n_cand, kappa, k)
            ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=self.X.device)
            self._h2d = {kk: v for kk, v in self._h2d.items() if kk[:4] == key[:4]}
            self._h2d[key] = ws
        return ws

    def device_status(self) -> int:
        """First device-side error recorded since the last reset (0 = none); synchronises."""
        return int(self.status.item())

    def reset_status(self):
        self.status.zero_()


class HostSearchPipeline:
    """Streams host-resident query batches through an index with the host-buffer entry point.

    ``submit`` enqueues one batch (pinned host tensors: queries, CSR candidate lists, and the
    top-k outputs) as one glv_search_host call and returns at once.  Batches rotate over
    ``depth`` streams, each with its own device workspace, so the host-to-device copies of one
    batch overlap the search of the batch before it; calls on the same stream (and so on the
    same workspace) run in order.  ``synchronize`` waits for everything submitted.
    """

    def __init__(self, index: GleanVecIndex, kappa: int, k: int, depth: int = 2, stream=None):
        if depth < 2:
            raise ValueError("depth >= 2 (one batch copying while another is searched)")
        self.ix, self.kappa, self.k, self.depth = index, kappa, k, depth
        self.origin = stream if stream is not None else torch.cuda.current_stream()
        self.streams = [torch.cuda.Stream(device=index.X.device) for _ in range(depth)]
        self._n = 0

    def begin(self):
        """Order every pipeline stream after the work already enqueued on the origin stream
        (for timing: an event recorded there before begin() precedes every batch submitted
        after it)."""
        for st in self.streams:
            st.wait_stream(self.origin)

    def submit(self, Q_h: torch.Tensor, off_h: torch.Tensor, ids_h: torch.Tensor, out_s_h: torch.Tensor,
               out_id_h: torch.Tensor) -> torch.cuda.Event:
        s = self._n % self.depth
        self._n += 1
        st = self.streams[s]
        ws = self.ix._host_workspace(Q_h.shape[0], ids_h.shape[0], self.kappa, self.k, slot=s)
        ix = self.ix
        glv.glv_search_host(ix.X, Q_h, ix.A, ix.compute, ix.Xred, ix.row_stride, ix.scales, ix.dt, ix.tags, off_h,
                            ids_h, self.kappa, self.k, ws, out_s_h, out_id_h, d_status=ix.status, stream=st)
        done = torch.cuda.Event()
        done.record(st)
        return done

    def end(self):
        """Order the origin stream after every batch submitted so far."""
        for st in self.streams:
            self.origin.wait_stream(st)

    def synchronize(self):
        for st in self.streams:
            st.synchronize()
