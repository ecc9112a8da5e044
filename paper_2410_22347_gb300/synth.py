"""Seeded synthetic inputs for the GleanVec search path.

This module is the one piece of code that both the CUDA path and the oracle consume.
It holds none of the method's arithmetic: it only draws database vectors, queries,
landmarks, projection matrices and candidate lists.  Cluster tags (Eq. cluster_tag),
reduced rows, scores and everything downstream are computed by the code under test.

The paper's datasets (its dataset table and appendix) are not available; these inputs
stand in for them with the same shapes and the same ID / OOD structure:

* database: a mixture of ``K`` Gaussians with uniform weights, means ``mu_k ~ N(0, I_D)``
  and covariance ``R_k diag(j^-alpha) R_k^T`` (``R_k`` Haar-orthogonal per component,
  ``alpha = 1``), every vector L2-normalised afterwards;
* out-of-distribution queries: means ``R_o mu_k`` for one shared Haar rotation ``R_o``,
  fresh Haar bases, ``alpha = 0.5``, L2-normalised;
* in-distribution queries: drawn from the database mixture itself (``queries="ood+id"``: the
  first half of the batch out-of-distribution, the second half in-distribution);
* landmarks: ``C`` distinct database rows drawn uniformly (already unit norm);
* projections: ``A_c = B_c = P_c`` with ``P_c`` a Haar-random row-orthonormal d x D
  matrix (QR of a Gaussian matrix, signs fixed by diag(R));
* candidate lists: CSR ``(off, ids)``; ids uniform over [0, N) without replacement
  within a list; list lengths either fixed or lognormal (arithmetic mean ``mean``,
  ``sigma``) clipped to ``[lo, hi]``.

Seeds follow ``base + 100 * cfg + {0 data, 1 queries, 2 landmarks, 3 projections,
4 candidates}`` with base 2410022347.  Generation runs on whatever torch device is
given, so the large workloads are drawn directly in device memory.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

SEED_BASE = 2410022347


def seed_for(cfg: int, part: str) -> int:
    off = {"data": 0, "queries": 1, "landmarks": 2, "proj": 3, "cands": 4, "pairs": 5}[part]
    return SEED_BASE + 100 * cfg + off


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def haar_orthogonal(n: int, count: int, g: torch.Generator, device) -> torch.Tensor:
    """``count`` Haar-distributed n x n orthogonal matrices (float32)."""
    z = torch.randn(count, n, n, generator=g, device=device, dtype=torch.float32)
    q, r = torch.linalg.qr(z)
    sgn = torch.sign(torch.diagonal(r, dim1=-2, dim2=-1))
    sgn = torch.where(sgn == 0, torch.ones_like(sgn), sgn)
    return q * sgn.unsqueeze(-2)


def row_orthonormal(d: int, D: int, count: int, g: torch.Generator, device) -> torch.Tensor:
    """``count`` Haar-random d x D matrices with orthonormal rows (float32)."""
    z = torch.randn(count, D, d, generator=g, device=device, dtype=torch.float32)
    q, r = torch.linalg.qr(z)
    sgn = torch.sign(torch.diagonal(r, dim1=-2, dim2=-1))
    sgn = torch.where(sgn == 0, torch.ones_like(sgn), sgn)
    return (q * sgn.unsqueeze(-2)).transpose(-1, -2).contiguous()


def _l2n(x: torch.Tensor) -> torch.Tensor:
    return x / x.norm(dim=1, keepdim=True).clamp_min(1e-30)


def mixture(n: int, D: int, means: torch.Tensor, alpha: float, g: torch.Generator, device,
            chunk: int = 1 << 18) -> torch.Tensor:
    """n L2-normalised samples of a uniform-weight Gaussian mixture with the given means
    and per-component covariance ``R_k diag(j^-alpha) R_k^T`` (fresh Haar ``R_k``)."""
    K = means.shape[0]
    R = haar_orthogonal(D, K, g, device)
    sd = torch.arange(1, D + 1, device=device, dtype=torch.float32).pow(-alpha / 2.0)
    comp = torch.randint(0, K, (n,), generator=g, device=device)
    out = torch.empty(n, D, device=device, dtype=torch.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        z = torch.randn(e - s, D, generator=g, device=device, dtype=torch.float32) * sd
        cs = comp[s:e]
        x = torch.empty_like(z)
        for k in range(K):
            sel = (cs == k).nonzero(as_tuple=True)[0]
            if sel.numel():
                x[sel] = means[k] + z[sel] @ R[k].T
        out[s:e] = _l2n(x)
    return out


def candidate_lists(nq: int, N: int, lengths: torch.Tensor, g: torch.Generator, device):
    """CSR candidate lists: ``off`` (nq+1, int64), ``ids`` (off[-1], int32).  Within a
    list the ids are distinct and uniform over [0, N); their order is the draw order."""
    lengths = lengths.to(device=device, dtype=torch.int64)
    if int(lengths.max()) > N:
        raise ValueError("candidate list longer than the database")
    off = torch.zeros(nq + 1, dtype=torch.int64, device=device)
    off[1:] = torch.cumsum(lengths, 0)
    total = int(off[-1])
    seg = torch.repeat_interleave(torch.arange(nq, device=device), lengths)
    ids = torch.randint(0, N, (total,), generator=g, device=device, dtype=torch.int64)
    for _ in range(64):
        key = seg * N + ids
        sk, perm = torch.sort(key)
        dup = torch.zeros(total, dtype=torch.bool, device=device)
        if total > 1:
            dup[1:] = sk[1:] == sk[:-1]
        ndup = int(dup.sum())
        if ndup == 0:
            break
        pos = perm[dup]
        ids[pos] = torch.randint(0, N, (ndup,), generator=g, device=device, dtype=torch.int64)
    else:
        raise RuntimeError("could not draw distinct candidates")
    return off, ids.to(torch.int32)


def lognormal_lengths(nq: int, mean: float, sigma: float, lo: int, hi: int,
                      g: torch.Generator, device) -> torch.Tensor:
    """List lengths ~ lognormal with arithmetic mean ``mean`` (mu = ln mean - sigma^2/2),
    rounded and clipped to [lo, hi]."""
    mu = math.log(mean) - 0.5 * sigma * sigma
    z = torch.randn(nq, generator=g, device=device, dtype=torch.float64)
    return torch.exp(mu + sigma * z).round().clamp(lo, hi).to(torch.int64)


@dataclass
class Workload:
    X: torch.Tensor          # N x D float32, unit rows
    Q: torch.Tensor          # nq x D float32, unit rows
    mu: torch.Tensor         # C x D float32 landmarks (unit)
    A: torch.Tensor          # C x d x D float32
    B: torch.Tensor          # C x d x D float32
    off: torch.Tensor        # nq+1 int64
    ids: torch.Tensor        # total int32
    kappa: int
    k: int
    name: str


def make_workload(*, N: int, D: int, d: int, C: int, nq: int, K_db: int, cands,
                  kappa: int, k: int, cfg: int, device="cpu", queries: str = "ood",
                  name: str = "", replica: int = 0) -> Workload:
    """Draw one workload.  ``cands`` is an int (fixed list length; N means exhaustive
    in id order), or a tuple ("lognormal", mean, sigma, lo, hi).  ``replica`` > 0 draws
    a different query set and candidate lists over the same database (one per GPU when
    the queries are sharded across processes)."""
    g = _gen(seed_for(cfg, "data"), device)
    means = torch.randn(K_db, D, generator=g, device=device, dtype=torch.float32)
    X = mixture(N, D, means, 1.0, g, device)

    gq = _gen(seed_for(cfg, "queries") + 1_000_003 * replica, device)
    if queries == "ood":
        Ro = haar_orthogonal(D, 1, gq, device)[0]
        Q = mixture(nq, D, means @ Ro.T, 0.5, gq, device)
    elif queries == "id":
        Q = mixture(nq, D, means, 1.0, gq, device)
    elif queries == "ood+id":  # first half out-of-distribution, second half in-distribution
        Ro = haar_orthogonal(D, 1, gq, device)[0]
        Qo = mixture(nq // 2, D, means @ Ro.T, 0.5, gq, device)
        gi = _gen(seed_for(cfg, "queries") + 7 + 1_000_003 * replica, device)
        Q = torch.cat([Qo, mixture(nq - nq // 2, D, means, 1.0, gi, device)])
    else:
        raise ValueError(queries)

    gl = _gen(seed_for(cfg, "landmarks"), device)
    pick = torch.randperm(N, generator=gl, device=device)[:C]
    mu = X[pick].clone()

    gp = _gen(seed_for(cfg, "proj"), device)
    P = row_orthonormal(d, D, C, gp, device)
    A = P.clone()
    B = P.clone()

    gc = _gen(seed_for(cfg, "cands") + 1_000_003 * replica, device)
    if isinstance(cands, int) and cands == N:
        off = torch.arange(nq + 1, device=device, dtype=torch.int64) * N
        ids = torch.arange(N, device=device, dtype=torch.int32).repeat(nq)
    elif isinstance(cands, int):
        off, ids = candidate_lists(nq, N, torch.full((nq,), cands, dtype=torch.int64), gc, device)
    else:
        _, mean, sigma, lo, hi = cands
        lens = lognormal_lengths(nq, mean, sigma, lo, hi, gc, device)
        off, ids = candidate_lists(nq, N, lens, gc, device)
    return Workload(X, Q, mu, A, B, off, ids, kappa, k, name)


# The workloads the paper's setting is exercised on (shapes of the dataset table: D in
# {512, 768}, d in 128..192; graph-search-like random candidate gathers).
WORKLOADS = {
    "exhaustive-10k": dict(N=10_000, D=512, d=128, C=8, nq=100, K_db=16, cands=10_000,
                           kappa=0, k=10, cfg=0),
    "graph-1M-d160": dict(N=1_000_000, D=768, d=160, C=32, nq=10_000, K_db=64, cands=2048,
                          kappa=100, k=10, cfg=1),
    "precision-10M-d128": dict(N=10_000_000, D=512, d=128, C=64, nq=20_000, K_db=64,
                               cands=4096, kappa=200, k=10, cfg=2, queries="ood+id"),
    "batching-2M-d192": dict(N=2_000_000, D=768, d=192, C=48, nq=8192, K_db=64,
                             cands=("lognormal", 2000.0, 1.2, 64, 32768), kappa=100, k=10,
                             cfg=3),
}


def workload(name: str, device="cpu", **override) -> Workload:
    """One of the named workloads, drawn on ``device``; keyword overrides change its fields
    (``queries=None`` keeps the workload's own query mix)."""
    kw = dict(WORKLOADS[name])
    kw.update({k: v for k, v in override.items() if v is not None})
    return make_workload(device=device, name=name, **kw)
