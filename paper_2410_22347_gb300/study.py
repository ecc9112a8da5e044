"""Synthetic analogue of the paper's brute-force accuracy comparison of GleanVec and
LeanVec-Sphering (Section 5.2): 10-recall@10 of the top 10 by the reduced inner product
(no re-rank) against the exact top 10, as a function of the target dimensionality d, for
C = 1 (linear LeanVec-Sphering) and several cluster counts C (GleanVec), on OOD queries.

Everything runs on the GPU through the library: landmarks by spherical k-means (Appendix A),
per-cluster LeanVec-Sphering from FP64 second moments (Algorithm 5), the reduced store, and the
exhaustive fused scoring + top-k; the exact ground truth comes from the same fused kernel on
an identity reduction (d = D, A = B = I, FP32 store), i.e. exact FP32 inner products.
"""
from __future__ import annotations

import torch

from . import glv, kmeans, learn, synth
from .index import GleanVecIndex


def recall_vs_d(device, N=100_000, D=256, n_learn=10_000, nq=1000, K_db=64, d_list=(16, 32, 64, 96, 128),
                C_list=(1, 16, 48), k=10, seed_cfg=7):
    # database and OOD queries from the synthetic mixtures; learning and test queries are
    # disjoint draws of the same query distribution
    w = synth.make_workload(N=N, D=D, d=8, C=1, nq=n_learn + nq, K_db=K_db, cands=1, kappa=0, k=1,
                            cfg=seed_cfg, device=device)
    X = w.X
    Q_learn = w.Q[:n_learn].contiguous()
    Q = w.Q[n_learn:].contiguous()
    off = torch.arange(nq + 1, device=device, dtype=torch.int64) * N
    ids = torch.arange(N, device=device, dtype=torch.int32).repeat(nq)

    # exact ground truth: identity reduction, FP32 store
    eye = torch.eye(D, device=device, dtype=torch.float32).unsqueeze(0).contiguous()
    exact = GleanVecIndex(X, eye, eye, tags=torch.zeros(N, dtype=torch.uint16, device=device), store="f32",
                          project="f32")
    _, gt = exact.search(Q, off, ids, 0, k)
    gt = gt.clone()
    del exact

    def recall(found):
        hit = (found.unsqueeze(2) == gt.unsqueeze(1)).any(dim=2).sum().item()
        return hit / (k * nq)

    rows = []
    for C in C_list:
        if C == 1:
            tags = torch.zeros(N, dtype=torch.uint16, device=device)
        else:
            mu, _ = kmeans.spherical_kmeans(X, C, iters=10, sample=100_000, seed=C)
            tags = glv.glv_assign_tags(X, mu)
        for d in d_list:
            A, B = learn.sphering_init(Q_learn, X, tags, C, d)
            ix = GleanVecIndex(X, A, B, tags=tags, store="f32", project="f32")
            _, found = ix.search(Q, off, ids, 0, k)
            rows.append({"C": C, "d": d, "recall_10at10": recall(found)})
            del ix
    return rows
