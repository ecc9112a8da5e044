"""FP64 CPU oracle for the GleanVec eager search path (arXiv 2410.22347).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The CUDA
library never imports, links or calls it, and this package never imports the CUDA
library: the two share no code.  The only module both sides use is the seeded input
generator ``paper_2410_22347_gb300.synth``, which holds none of the method's
arithmetic.

The search-path routines live in ``glv_oracle.c`` (plain FP64 loops, compiled with gcc
into ``liboracle.so`` next to this file); this module marshals numpy arrays into them.
The learning-side routines (LeanVec-Sphering, Algorithm 2 in its eigendecomposition
form of Section 3.2) are written here in numpy FP64, with ``numpy.linalg.eigh`` as the
eigendecomposition primitive.

Parity pins of every routine are in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "glv_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``glv_oracle.c`` with gcc (FP64, OpenMP over queries) if stale."""
    with _lock:
        stale = force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-fPIC",
                   "-shared", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    sig = {
        "glvo_set_threads": (None, [i32]),
        "glvo_get_threads": (i32, []),
        "glvo_assign_tags": (None, [P, i64, i32, P, i32, P, P]),
        "glvo_build_reduced": (None, [P, i64, i32, P, P, i32, i32, P]),
        "glvo_project": (None, [P, i64, i32, P, i32, i32, P]),
        "glvo_score": (i32, [P, i64, i32, i32, P, P, i64, P, P, P]),
        "glvo_topk": (None, [P, P, P, i64, i32, P, P]),
        "glvo_rerank": (i32, [P, i64, i32, P, i64, P, i32, i32, P, P]),
        "glvo_exact_topk": (i32, [P, i64, i32, P, i64, P, P, i32, P, P]),
        "glvo_search": (i32, [P, i64, i32, P, P, P, i32, i32, P, i64, P, P, i32, i32, P, P]),
        "glvo_bf16_encode": (None, [P, i64, P]),
        "glvo_bf16_decode": (None, [P, i64, P]),
        "glvo_e4m3_decode": (None, [P, i64, P]),
        "glvo_e4m3_encode": (None, [P, i64, P]),
        "glvo_quantize_fp8_rows": (None, [P, i64, i32, P, P]),
        "glvo_pair_loss_grad": (f64, [P, P, i32, P, P, P, i32, i32, P, P, i64, P, P]),
        "glvo_second_moment": (None, [P, i64, i32, P, i32, P]),
        "glvo_kmeans_update": (None, [P, i64, i32, P, i32, P, P, P]),
        "glvo_spherical_objective": (f64, [P, i64, i32, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _c(a: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> None:
    _load().glvo_set_threads(int(n))


def get_threads() -> int:
    return int(_load().glvo_get_threads())


# ------------------------------------------------------------------------------------
# search path (C, FP64)
# ------------------------------------------------------------------------------------

def assign_tags(X, mu, return_margin: bool = False):
    """Eq. (cluster_tag), Section 4: c_i = argmax_c <x_i, mu_c>, ties to the lowest c."""
    X = _c(X, np.float32)
    mu = _c(mu, np.float32)
    N, D = X.shape
    C = mu.shape[0]
    tags = np.empty(N, np.uint16)
    margin = np.empty(N, np.float64)
    _load().glvo_assign_tags(_p(X), N, D, _p(mu), C, _p(tags), _p(margin))
    return (tags, margin) if return_margin else tags


def build_reduced(X, tags, B):
    """Eq. (X_low), Section 4 (read with g): x_i^low = B_{c_i} x_i, FP64, N x d."""
    X = _c(X, np.float32)
    tags = _c(tags, np.uint16)
    B = _c(B, np.float32)
    N, D = X.shape
    C, d, D2 = B.shape
    assert D2 == D
    Xr = np.empty((N, d), np.float64)
    _load().glvo_build_reduced(_p(X), N, D, _p(tags), _p(B), C, d, _p(Xr))
    return Xr


def project(Q, A):
    """Algorithm 4 preprocess: Qp[j, c] = A_c q_j, FP64, nq x C x d."""
    Q = _c(Q, np.float32)
    A = _c(A, np.float32)
    nq, D = Q.shape
    C, d, _ = A.shape
    Qp = np.empty((nq, C, d), np.float64)
    _load().glvo_project(_p(Q), nq, D, _p(A), C, d, _p(Qp))
    return Qp


def score(Qp, Xr, tags, off, ids):
    """Algorithm 4 inner-product: s[p] = <Qp[j, c_i], Xr[i]> for candidate p = (j, i).

    Returns (scores FP64 of length off[-1], bad_id_flag)."""
    Qp = _c(Qp, np.float64)
    Xr = _c(Xr, np.float64)
    tags = _c(tags, np.uint16)
    off = _c(off, np.int64)
    ids = _c(ids, np.int32)
    nq, C, d = Qp.shape
    N = Xr.shape[0]
    s = np.empty(int(off[-1]), np.float64)
    bad = _load().glvo_score(_p(Qp), nq, C, d, _p(Xr), _p(tags), N, _p(off), _p(ids), _p(s))
    return s, bool(bad)


def topk(s, off, ids, kappa: int):
    """Per-query top-kappa, score descending, ties to the smaller id, NaN last; padding
    slots get (-inf, -1)."""
    s = _c(s, np.float64)
    off = _c(off, np.int64)
    ids = _c(ids, np.int32)
    nq = off.shape[0] - 1
    out_s = np.empty((nq, kappa), np.float64)
    out_id = np.empty((nq, kappa), np.int32)
    _load().glvo_topk(_p(s), _p(off), _p(ids), nq, kappa, _p(out_s), _p(out_id))
    return out_s, out_id


def rerank(X, Q, surv, k: int):
    """Algorithm 1 post-processing: exact <q, x> over full D for the survivors (id -1 =
    empty slot), top k.  Returns (scores, ids, bad_id_flag)."""
    X = _c(X, np.float32)
    Q = _c(Q, np.float32)
    surv = _c(surv, np.int32)
    N, D = X.shape
    nq, kappa = surv.shape
    out_s = np.empty((nq, k), np.float64)
    out_id = np.empty((nq, k), np.int32)
    bad = _load().glvo_rerank(_p(X), N, D, _p(Q), nq, _p(surv), kappa, k, _p(out_s), _p(out_id))
    return out_s, out_id, bool(bad)


def exact_topk(X, Q, off, ids, k: int):
    """Exact maximum-inner-product top k (Section 2) over each query's candidate list."""
    X = _c(X, np.float32)
    Q = _c(Q, np.float32)
    off = _c(off, np.int64)
    ids = _c(ids, np.int32)
    N, D = X.shape
    nq = off.shape[0] - 1
    out_s = np.empty((nq, k), np.float64)
    out_id = np.empty((nq, k), np.int32)
    _load().glvo_exact_topk(_p(X), N, D, _p(Q), nq, _p(off), _p(ids), k, _p(out_s), _p(out_id))
    return out_s, out_id


def search(X, Xr, tags, A, Q, off, ids, kappa: int, k: int):
    """Whole eager multi-step search (Algorithm 1 with Algorithm 4), query by query."""
    X = _c(X, np.float32)
    Xr = _c(Xr, np.float64)
    tags = _c(tags, np.uint16)
    A = _c(A, np.float32)
    Q = _c(Q, np.float32)
    off = _c(off, np.int64)
    ids = _c(ids, np.int32)
    N, D = X.shape
    C, d, _ = A.shape
    nq = Q.shape[0]
    out_s = np.empty((nq, k), np.float64)
    out_id = np.empty((nq, k), np.int32)
    _load().glvo_search(_p(X), N, D, _p(Xr), _p(tags), _p(A), C, d, _p(Q), nq, _p(off),
                        _p(ids), kappa, k, _p(out_s), _p(out_id))
    return out_s, out_id


def recall(found_ids, truth_ids) -> float:
    """K-recall@k of Section 5: |S cap G| / K, averaged over queries (K = truth width)."""
    found_ids = np.asarray(found_ids)
    truth_ids = np.asarray(truth_ids)
    K = truth_ids.shape[1]
    hits = 0
    for f, g in zip(found_ids, truth_ids):
        hits += len(set(int(v) for v in f if v >= 0) & set(int(v) for v in g if v >= 0))
    return hits / (K * truth_ids.shape[0])


# ------------------------------------------------------------------------------------
# scalar quantisation (reading: RNE BF16; FP8-e4m3 with one FP32 scale per vector)
# ------------------------------------------------------------------------------------

def bf16_encode(x):
    x = _c(x, np.float32)
    out = np.empty(x.shape, np.uint16)
    _load().glvo_bf16_encode(_p(x), x.size, _p(out))
    return out


def bf16_decode(codes):
    codes = _c(codes, np.uint16)
    out = np.empty(codes.shape, np.float64)
    _load().glvo_bf16_decode(_p(codes), codes.size, _p(out))
    return out


def e4m3_decode(codes):
    codes = _c(codes, np.uint8)
    out = np.empty(codes.shape, np.float64)
    _load().glvo_e4m3_decode(_p(codes), codes.size, _p(out))
    return out


def e4m3_encode(x):
    x = _c(x, np.float64)
    out = np.empty(x.shape, np.uint8)
    _load().glvo_e4m3_encode(_p(x), x.size, _p(out))
    return out


def quantize_fp8_rows(x32):
    """Per-vector FP8-e4m3 quantisation of FP32 rows: returns (codes uint8, scales fp32)."""
    x32 = _c(x32, np.float32)
    rows, d = x32.shape
    codes = np.empty((rows, d), np.uint8)
    scales = np.empty(rows, np.float32)
    _load().glvo_quantize_fp8_rows(_p(x32), rows, d, _p(codes), _p(scales))
    return codes, scales


def dequantize_fp8_rows(codes, scales):
    """Reduced rows as the quantised store represents them: scale_i * decode(code_ij)."""
    return e4m3_decode(codes) * np.asarray(scales, np.float64)[:, None]


# ------------------------------------------------------------------------------------
# learning side (config with refinement): loss, gradients, second moments, Sphering
# ------------------------------------------------------------------------------------

def pair_loss_grad(Q, X, tags, A, B, qi, xi, want_grad: bool = True):
    """Loss sum_p (<q_p, x_p> - <A_c q_p, B_c x_p>)^2 over index pairs (Section 2.1 loss
    restricted to GleanVec pairs) and its gradients w.r.t. every A_c and B_c (FP64)."""
    Q = _c(Q, np.float32)
    X = _c(X, np.float32)
    tags = _c(tags, np.uint16)
    A = _c(A, np.float32)
    B = _c(B, np.float32)
    qi = _c(qi, np.int32)
    xi = _c(xi, np.int32)
    C, d, D = A.shape
    gA = np.empty((C, d, D), np.float64) if want_grad else None
    gB = np.empty((C, d, D), np.float64) if want_grad else None
    loss = _load().glvo_pair_loss_grad(_p(Q), _p(X), D, _p(tags), _p(A), _p(B), C, d, _p(qi),
                                       _p(xi), qi.shape[0], _p(gA), _p(gB))
    return (loss, gA, gB) if want_grad else loss


def second_moment(V, tags=None, cluster: int = -1):
    """K = sum_v v v^T (Section 3.2 summary statistic) in FP64."""
    V = _c(V, np.float32)
    n, D = V.shape
    t = _c(tags, np.uint16) if tags is not None else None
    K = np.empty((D, D), np.float64)
    _load().glvo_second_moment(_p(V), n, D, _p(t), int(cluster), _p(K))
    return K


def sphering_from_moments(KQ, KX, d: int, rel_tol: float = 1e-12):
    """Algorithm 2 (LeanVec-Sphering) in the eigendecomposition form of Section 3.2.

    K_Q = U S^2 U^T  ->  W = U S U^T,  W^+ = U S^+ U^T (pseudo-inverse: singular values
    below rel_tol * S_max are treated as zero);  P = the d leading eigenvectors of
    W K_X W (as rows, eigenvalues descending);  A = P W^+,  B = P W.
    Returns (A, B, W, eigenvalues of W K_X W in descending order)."""
    KQ = np.asarray(KQ, np.float64)
    KX = np.asarray(KX, np.float64)
    lam, U = np.linalg.eigh(0.5 * (KQ + KQ.T))
    S = np.sqrt(np.clip(lam, 0.0, None))
    Sinv = np.where(S > rel_tol * S.max(), 1.0 / np.where(S > 0, S, 1.0), 0.0)
    W = (U * S) @ U.T
    Winv = (U * Sinv) @ U.T
    M = W @ KX @ W
    mu, V = np.linalg.eigh(0.5 * (M + M.T))
    order = np.argsort(mu)[::-1]
    mu = mu[order]
    P = V[:, order[:d]].T
    return P @ Winv, P @ W, W, mu


def gleanvec_sphering(Q_learn, X_learn, tags, C: int, d: int):
    """Algorithm 5 with given landmarks/tags: one LeanVec-Sphering pair per cluster, all
    clusters sharing the same query statistics.  Returns A, B of shape C x d x D (FP64)."""
    KQ = second_moment(Q_learn)
    D = KQ.shape[0]
    A = np.zeros((C, d, D))
    B = np.zeros((C, d, D))
    for c in range(C):
        KX = second_moment(X_learn, tags, c)
        A[c], B[c], _, _ = sphering_from_moments(KQ, KX, d)
    return A, B


# ------------------------------------------------------------------------------------
# spherical k-means (Appendix A)
# ------------------------------------------------------------------------------------

def kmeans_update(X, tags, mu_in):
    """M-step of spherical k-means: mu_c = normalised sum of the rows tagged c (FP64); a
    cluster without members keeps its landmark.  Returns (mu FP64 C x D, counts)."""
    X = _c(X, np.float32)
    tags = _c(tags, np.uint16)
    mu_in = _c(mu_in, np.float32)
    N, D = X.shape
    C = mu_in.shape[0]
    mu = np.empty((C, D), np.float64)
    counts = np.empty(C, np.int64)
    _load().glvo_kmeans_update(_p(X), N, D, _p(tags), C, _p(mu_in), _p(mu), _p(counts))
    return mu, counts


def spherical_objective(X, mu, tags):
    """Appendix A objective sum_i <x_i, mu_{c_i}>."""
    X = _c(X, np.float32)
    mu = _c(mu, np.float32)
    tags = _c(tags, np.uint16)
    N, D = X.shape
    return float(_load().glvo_spherical_objective(_p(X), N, D, _p(mu), _p(tags)))
