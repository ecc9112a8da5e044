"""Learning side of GleanVec on the GPU: LeanVec-Sphering per cluster (Algorithm 2 inside
Algorithm 5, in the eigendecomposition form of Section 3.2) and its gradient refinement.

* ``second_moments`` -- K = sum v v^T per cluster, FP64 on the GPU (glv_second_moments).
* ``sphering_init``  -- K_Q and K_{X_c} on the GPU; on the host, a Cholesky whitening
  K_Q = L L^T and the d leading eigenvectors U_d of L^T K_{X_c} L give A_c = U_d^T L^{-1},
  B_c = U_d^T L^T -- the solution of Algorithm 2 reached through another factor of K_Q than
  its W = U S U^T (see ``sphering_factors``).  L is shared by all clusters (every cluster
  uses the same learning queries).
* ``PairLoss``       -- torch.autograd.Function for L = sum_p (t_p - s_p)^2 (the inner-product
  approximation loss of Section 2.1 over GleanVec pairs): forward glv_pair_forward
  (s_p = <A_c q_p, B_c x_p>, t_p = <q_p, x_p>) and glv_pair_loss (FP64 sum); backward
  glv_pair_loss (g_p = -2 (t_p - s_p)) and glv_pair_backward (dA_c = sum g_p (B_c x_p) q_p^T,
  dB_c = sum g_p (A_c q_p) x_p^T).
* ``refine``         -- minimises L over random minibatches of (query, database) pairs with
  Adam steps in the library (glv_adam_step); torch holds the tensors and runs the autograd
  bookkeeping only.
"""
from __future__ import annotations

import ctypes

import numpy as np
import scipy.linalg
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
                                     _P, _P]),
        ("glv_pair_loss", _i32, [_P, _P, _i64, _P, _P, _P, _P]),
        ("glv_adam_step", _i32, [_P, _P, _P, _P, _i64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_float, _i32, _P])):
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


def glv_pair_loss(s, t, weight=None, want_loss: bool = True, want_grad: bool = False, stream=None):
    """loss = sum_p (t_p - s_p)^2 (FP64 scalar tensor) and/or g = -2 w (t - s) (FP32), with w
    the device scalar ``weight`` (float64) or 1."""
    _need(s, torch.float32, "s", 1)
    _need(t, torch.float32, "t", 1)
    P = s.shape[0]
    loss = torch.empty((), dtype=torch.float64, device=s.device) if want_loss else None
    g = torch.empty(P, dtype=torch.float32, device=s.device) if want_grad else None
    if weight is not None:
        _need(weight, torch.float64, "weight", 0)
    _check("glv_pair_loss", _lib.glv_pair_loss(_ptr(s), _ptr(t), P, _ptr(weight), _ptr(loss), _ptr(g),
                                               _stream(stream)))
    return loss, g


def glv_adam_step(param: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor, step: int,
                  lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream=None):
    """One in-place Adam step on contiguous FP32 tensors (param, m, v updated)."""
    for t_, n_ in ((param, "param"), (grad, "grad"), (m, "m"), (v, "v")):
        _need(t_, torch.float32, n_, param.dim())
    _check("glv_adam_step", _lib.glv_adam_step(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(), lr, beta1,
                                               beta2, eps, step, _stream(stream)))


class PairLoss(torch.autograd.Function):
    """L = sum_p (t_p - s_p)^2 with s_p = <A_c q_p, B_c x_p> and t_p = <q_p, x_p>: forward by
    glv_pair_forward and glv_pair_loss, backward by glv_pair_loss (g = dL/ds, scaled by the
    upstream gradient on the device) and the hand-written glv_pair_backward."""

    @staticmethod
    def forward(ctx, A, B, Q, X, tags, qi, xi):
        s, t, u, v = glv_pair_forward(Q, X, tags, A.detach().contiguous(), B.detach().contiguous(), qi, xi)
        loss, _ = glv_pair_loss(s, t)
        ctx.save_for_backward(Q, X, tags, qi, xi, s, t, u, v)
        ctx.C = A.shape[0]
        return loss

    @staticmethod
    def backward(ctx, gout):
        Q, X, tags, qi, xi, s, t, u, v = ctx.saved_tensors
        _, g = glv_pair_loss(s, t, weight=gout.detach().to(torch.float64).contiguous(), want_loss=False,
                             want_grad=True)
        dA, dB = glv_pair_backward(Q, X, tags, ctx.C, qi, xi, u, v, g)
        return dA, dB, None, None, None, None, None


def pair_loss(A, B, Q, X, tags, qi, xi):
    """sum_p (t_p - s_p)^2 (FP64 scalar) with autograd through the library's kernels."""
    return PairLoss.apply(A, B, Q, X, tags, qi, xi)


# ---------------------------------------------------------------------------------------
# LeanVec-Sphering initialisation (host eigendecompositions of GPU FP64 statistics)
# ---------------------------------------------------------------------------------------

def sphering_factors(KQ: np.ndarray, KX: np.ndarray, d: int):
    """LeanVec-Sphering of one cluster (Algorithm 2) through a Cholesky whitening.

    Algorithm 2 takes W = U S U^T from the SVD of the stacked queries; what the derivation of
    Section 3.2 uses of W is only W^T W = Q Q^T = K_Q.  Any factor W' = O W with O orthogonal
    has that property, and the solution does not depend on the choice: the d leading
    eigenvectors of W' K_X W'^T are O times those of W K_X W, so with U_d holding them as
    columns,  A = U_d^T W'^{-T}  and  B = U_d^T W'  are the paper's P W^{-1} and P W (up to
    the sign of each row pair, and a rotation inside a repeated eigenvalue).  Here W' = L^T
    with K_Q = L L^T the Cholesky factorisation, so

        A = U_d^T L^{-1}  (a triangular solve),   B = U_d^T L^T = (L U_d)^T,

    with U_d the leading eigenvectors of L^T K_X L.  K_Q must be positive definite (the
    learning queries span R^D); a singular K_Q raises ValueError (the pseudo-inverse that
    Section 3.2 allows for that case is not offered here).
    Returns (A, B, W' = L^T, eigenvalues of L^T K_X L in descending order)."""
    KQ = np.asarray(KQ, np.float64)
    KX = np.asarray(KX, np.float64)
    try:
        L = np.linalg.cholesky(0.5 * (KQ + KQ.T))
    except np.linalg.LinAlgError as e:
        raise ValueError("the query second-moment matrix K_Q is not positive definite") from e
    piv = np.diag(L)
    if not piv.min() > 1e-6 * piv.max():  # pivots^2 spread beyond 1e-12: numerically singular
        raise ValueError("the query second-moment matrix K_Q is numerically singular")
    M = L.T @ KX @ L
    lam, V = np.linalg.eigh(0.5 * (M + M.T))
    lam, V = lam[::-1], V[:, ::-1]
    Ud = V[:, :d]
    A = scipy.linalg.solve_triangular(L, Ud, lower=True, trans="T").T  # U_d^T L^{-1}
    B = (L @ Ud).T
    return A, B, L.T, lam


def sphering_init(Q_learn: torch.Tensor, X_learn: torch.Tensor, tags: torch.Tensor, C: int, d: int):
    """Per-cluster LeanVec-Sphering: returns A, B (C x d x D float32 on the device)."""
    KQ = glv_second_moments(Q_learn)[0].cpu().numpy()
    KX = glv_second_moments(X_learn, tags, C).cpu().numpy()
    D = KQ.shape[0]
    A = np.zeros((C, d, D))
    B = np.zeros((C, d, D))
    for c in range(C):
        A[c], B[c], _, _ = sphering_factors(KQ, KX[c], d)
    dev = Q_learn.device
    return (torch.from_numpy(A).to(device=dev, dtype=torch.float32).contiguous(),
            torch.from_numpy(B).to(device=dev, dtype=torch.float32).contiguous())


def refine(A: torch.Tensor, B: torch.Tensor, Q: torch.Tensor, X: torch.Tensor, tags: torch.Tensor, steps: int,
           batch: int = 4096, lr: float = 1e-3, seed: int = 0):
    """Adam (glv_adam_step) on sum_p (t_p - s_p)^2 over uniform random (query, database)
    minibatches.  Returns the refined (A, B) and the per-step minibatch losses."""
    A = A.detach().clone().contiguous().requires_grad_(True)
    B = B.detach().clone().contiguous().requires_grad_(True)
    state = [(torch.zeros_like(A), torch.zeros_like(A)), (torch.zeros_like(B), torch.zeros_like(B))]
    g = torch.Generator(device=Q.device)
    g.manual_seed(seed)
    losses = []
    for step in range(1, steps + 1):
        qi = torch.randint(0, Q.shape[0], (batch,), generator=g, device=Q.device, dtype=torch.int32)
        xi = torch.randint(0, X.shape[0], (batch,), generator=g, device=Q.device, dtype=torch.int32)
        A.grad = None
        B.grad = None
        loss = pair_loss(A, B, Q, X, tags, qi, xi)
        loss.backward()
        with torch.no_grad():
            for (p, (m, v)) in zip((A, B), state):
                glv_adam_step(p, p.grad, m, v, step, lr)
        losses.append(loss.detach())
    return A.detach(), B.detach(), [float(x) for x in losses]
