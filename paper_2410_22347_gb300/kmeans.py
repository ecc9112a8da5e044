"""Spherical k-means landmarks (Appendix A; step 2 of Algorithm 5) on the GPU.

E-step: glv_assign_tags (c_i = argmax_c <x_i, mu_c>, Eq. cluster_tag).  M-step:
glv_kmeans_update (mu_c = normalised sum of its members, FP64 sums).  Seeding: k-means++ on
the normalised sample, each new landmark drawn with probability proportional to
(1 - max_c <x, mu_c>)^2 (the spherical analogue of the squared distance to the nearest
landmark).  As in the paper, the landmarks are learned from a uniform random sample of the
normalised database (1e5 points by default).
"""
from __future__ import annotations

import torch

from . import glv


def _normalised(X: torch.Tensor) -> torch.Tensor:
    return (X / X.norm(dim=1, keepdim=True).clamp_min(1e-30)).contiguous()


def kmeanspp(S: torch.Tensor, C: int, gen: torch.Generator) -> torch.Tensor:
    """k-means++ seeding of C landmarks among the rows of S (unit rows)."""
    n = S.shape[0]
    first = int(torch.randint(0, n, (1,), generator=gen, device=S.device))
    mu = torch.empty(C, S.shape[1], dtype=torch.float32, device=S.device)
    mu[0] = S[first]
    tags = torch.empty(n, dtype=torch.uint16, device=S.device)
    best = torch.empty(n, dtype=torch.float32, device=S.device)
    for c in range(1, C):
        glv.glv_assign_tags(S, mu[:c].contiguous(), tags=tags, best_ip=best)
        w = (1.0 - best).clamp_min(0.0) ** 2
        if float(w.sum()) <= 0.0:
            w = torch.ones_like(w)
        mu[c] = S[int(torch.multinomial(w, 1, generator=gen))]
    return mu


def spherical_kmeans(X: torch.Tensor, C: int, iters: int = 10, sample: int = 100_000, seed: int = 0):
    """Landmarks (C x D, unit rows) and the objective sum <x, mu_c(x)> per iteration."""
    gen = torch.Generator(device=X.device)
    gen.manual_seed(seed)
    n = X.shape[0]
    if sample and n > sample:
        rows = torch.randperm(n, generator=gen, device=X.device)[:sample]
        S = _normalised(X[rows])
    else:
        S = _normalised(X)
    mu = kmeanspp(S, C, gen)
    tags = torch.empty(S.shape[0], dtype=torch.uint16, device=X.device)
    best = torch.empty(S.shape[0], dtype=torch.float32, device=X.device)
    history = []
    for _ in range(iters):
        glv.glv_assign_tags(S, mu, tags=tags, best_ip=best)
        history.append(float(best.double().sum()))
        glv.glv_kmeans_update(S, tags, mu)
    return mu, history
