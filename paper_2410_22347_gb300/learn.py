"""Learning side of GleanVec on the GPU: LeanVec-Sphering per cluster (Algorithm 2 inside
Algorithm 5, in the eigendecomposition form of Section 3.2) and its gradient refinement.

* ``second_moments`` -- K = sum v v^T per cluster, FP64 on the GPU (glv_second_moments).
* ``sphering_init``  -- K_Q and K_{X_c} on the GPU; on the host, eigendecompositions:
  K_Q = U S^2 U^T gives W = U S U^T and W^+ (pseudo-inverse below 1e-12 S_max); the d leading
  eigenvectors of W K_{X_c} W give P_c; A_c = P_c W^+, B_c = P_c W.  W is shared by all
  clusters (every cluster uses the same learning queries).
* ``PairScore``      -- torch.autograd.Function whose forward is glv_pair_forward
  (s_p = <A_c q_p, B_c x_p>, t_p = <q_p, x_p>) and whose backward is glv_pair_backward
  (dA_c = sum g_p (B_c x_p) q_p^T, dB_c = sum g_p (A_c q_p) x_p^T).
* ``refine``         -- minimises sum_p (t_p - s_p)^2 (the inner-product approximation loss of
  Section 2.1 over GleanVec pairs) over random minibatches of (query, database) pairs.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import glv

_lib = glv.lib()
_P, _i64, _i32, _sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t
for _name, _res, _args in (
        ("glv_second_moments_workspace_size", _sz, [_i64, _i32]),
        ("glv_second_moments", _i32, [_P, _i64, _i32, _P, _i32, _P, _P, _P, _P]),
        ("glv_pair_workspace_size", _sz, [_i64, _i32]),
        ("glv_pair_forward", _i32, [_P, _i64, _P, _i64, _i32, _P, _P, _P, _i32, _i32, _P, _P, _i64, _P, _P, _P, _P,
                                    _P, _P, _P]),
        ("glv_pair_backward", _i32, [_P, _i64, _P, _i64, _i32, _P, _i32, _i32, _P, _P, _i64, _P, _P, _P, _P, _P, _P,
                                     _P, _P])):
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

_ptr = glv._ptr
_stream = glv._stream
_need = glv._need
_check = glv._check


def glv_second_moments(V: torch.Tensor, tags: torch.Tensor | None = None, C: int = 1, d_status=None, stream=None):
    """C x D x D float64 second moments (one D x D matrix when tags is None)."""
    _need(V, torch.float32, "V", 2)
    n, D = V.shape
    if tags is not None:
        _need(tags, torch.uint16, "tags", 1)
    K = torch.empty(C, D, D, dtype=torch.float64, device=V.device)
    ws = None
    if tags is not None:
        ws = torch.empty(max(int(_lib.glv_second_moments_workspace_size(n, C)), 1), dtype=torch.uint8,
                         device=V.device)
    _check("glv_second_moments", _lib.glv_second_moments(_ptr(V), n, D, _ptr(tags), C, _ptr(K), _ptr(ws),
                                                         _ptr(d_status), _stream(stream)))
    return K


def _pair_ws(P: int, C: int, device):
    return torch.empty(max(int(_lib.glv_pair_workspace_size(P, C)), 1), dtype=torch.uint8, device=device)


def glv_pair_forward(Q, X, tags, A, B, qi, xi, d_status=None, stream=None):
    """Returns (s, t, u, v) for the pairs (qi[p], xi[p])."""
    for t_, n_, nd in ((Q, "Q", 2), (X, "X", 2), (A, "A", 3), (B, "B", 3)):
        _need(t_, torch.float32, n_, nd)
    _need(tags, torch.uint16, "tags", 1)
    _need(qi, torch.int32, "qi", 1)
    _need(xi, torch.int32, "xi", 1)
    C, d, D = A.shape
    P = qi.shape[0]
    dev = Q.device
    s = torch.empty(P, dtype=torch.float32, device=dev)
    t = torch.empty(P, dtype=torch.float32, device=dev)
    u = torch.empty(P, d, dtype=torch.float32, device=dev)
    v = torch.empty(P, d, dtype=torch.float32, device=dev)
    _check("glv_pair_forward", _lib.glv_pair_forward(
        _ptr(Q), Q.shape[0], _ptr(X), X.shape[0], D, _ptr(tags), _ptr(A), _ptr(B), C, d, _ptr(qi), _ptr(xi), P,
        _ptr(s), _ptr(t), _ptr(u), _ptr(v), _ptr(_pair_ws(P, C, dev)), _ptr(d_status), _stream(stream)))
    return s, t, u, v


def glv_pair_backward(Q, X, tags, C: int, qi, xi, u, v, g, d_status=None, stream=None):
    """Returns (dA, dB), C x d x D, for upstream gradient g = dL/ds."""
    P, d = u.shape
    D = Q.shape[1]
    dev = Q.device
    dA = torch.empty(C, d, D, dtype=torch.float32, device=dev)
    dB = torch.empty(C, d, D, dtype=torch.float32, device=dev)
    g = g.contiguous().to(torch.float32)
    _check("glv_pair_backward", _lib.glv_pair_backward(
        _ptr(Q), Q.shape[0], _ptr(X), X.shape[0], D, _ptr(tags), C, d, _ptr(qi), _ptr(xi), P, _ptr(u), _ptr(v),
        _ptr(g), _ptr(dA), _ptr(dB), _ptr(_pair_ws(P, C, dev)), _ptr(d_status), _stream(stream)))
    return dA, dB


class PairScore(torch.autograd.Function):
    """s_p = <A_c q_p, B_c x_p> (differentiable in A and B) and t_p = <q_p, x_p> (constant)."""

    @staticmethod
    def forward(ctx, A, B, Q, X, tags, qi, xi):
        s, t, u, v = glv_pair_forward(Q, X, tags, A.detach().contiguous(), B.detach().contiguous(), qi, xi)
        ctx.save_for_backward(Q, X, tags, qi, xi, u, v)
        ctx.C = A.shape[0]
        ctx.mark_non_differentiable(t)
        return s, t

    @staticmethod
    def backward(ctx, gs, gt):
        Q, X, tags, qi, xi, u, v = ctx.saved_tensors
        dA, dB = glv_pair_backward(Q, X, tags, ctx.C, qi, xi, u, v, gs)
        return dA, dB, None, None, None, None, None


def pair_loss(A, B, Q, X, tags, qi, xi):
    """sum_p (t_p - s_p)^2 with autograd through the library's kernels."""
    s, t = PairScore.apply(A, B, Q, X, tags, qi, xi)
    return ((t - s) ** 2).sum()


# ---------------------------------------------------------------------------------------
# LeanVec-Sphering initialisation (host eigendecompositions of GPU FP64 statistics)
# ---------------------------------------------------------------------------------------

def _sphering(KQ: np.ndarray, KX: np.ndarray, d: int, rel_tol: float = 1e-12):
    lam, U = np.linalg.eigh(0.5 * (KQ + KQ.T))
    S = np.sqrt(np.clip(lam, 0.0, None))
    keep = S > rel_tol * S.max()
    Sinv = np.zeros_like(S)
    Sinv[keep] = 1.0 / S[keep]
    W = (U * S) @ U.T
    Winv = (U * Sinv) @ U.T
    M = W @ KX @ W
    mu, V = np.linalg.eigh(0.5 * (M + M.T))
    order = np.argsort(mu)[::-1]
    P = V[:, order[:d]].T
    return P @ Winv, P @ W


def sphering_init(Q_learn: torch.Tensor, X_learn: torch.Tensor, tags: torch.Tensor, C: int, d: int):
    """Per-cluster LeanVec-Sphering: returns A, B (C x d x D float32 on the device)."""
    KQ = glv_second_moments(Q_learn)[0].cpu().numpy()
    KX = glv_second_moments(X_learn, tags, C).cpu().numpy()
    D = KQ.shape[0]
    A = np.zeros((C, d, D))
    B = np.zeros((C, d, D))
    for c in range(C):
        A[c], B[c] = _sphering(KQ, KX[c], d)
    dev = Q_learn.device
    return (torch.from_numpy(A).to(device=dev, dtype=torch.float32).contiguous(),
            torch.from_numpy(B).to(device=dev, dtype=torch.float32).contiguous())


def refine(A: torch.Tensor, B: torch.Tensor, Q: torch.Tensor, X: torch.Tensor, tags: torch.Tensor, steps: int,
           batch: int = 4096, lr: float = 1e-3, seed: int = 0):
    """Adam on sum_p (t_p - s_p)^2 over uniform random (query, database) minibatches.
    Returns the refined (A, B) and the per-step minibatch losses."""
    A = A.detach().clone().requires_grad_(True)
    B = B.detach().clone().requires_grad_(True)
    opt = torch.optim.Adam([A, B], lr=lr)
    g = torch.Generator(device=Q.device)
    g.manual_seed(seed)
    losses = []
    for _ in range(steps):
        qi = torch.randint(0, Q.shape[0], (batch,), generator=g, device=Q.device, dtype=torch.int32)
        xi = torch.randint(0, X.shape[0], (batch,), generator=g, device=Q.device, dtype=torch.int32)
        opt.zero_grad(set_to_none=True)
        loss = pair_loss(A, B, Q, X, tags, qi, xi)
        loss.backward()
        opt.step()
        losses.append(float(loss.detach()))
    return A.detach(), B.detach(), losses
