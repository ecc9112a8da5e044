"""Flexible target dimensionality (Section 3.1): store x' = P' W x with all D LeanVec-Sphering
directions (P' = every eigenvector of W K_X W, sorted), choose d at search time by reading
the first d elements of each stored row with the first d rows of A' = P' W^+, and re-rank
from the same store, since <A' q, x'> = <q, x> when all D directions are kept."""
import numpy as np
import pytest
import torch

import oracle
from oracle.compare import scores_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def libs():
    from paper_2410_22347_gb300 import build_lib
    build_lib.build()
    from paper_2410_22347_gb300 import glv, learn
    return glv, learn


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def test_prefix_d_search_and_exact_rerank_from_one_store(libs):
    glv, learn = libs
    rng = np.random.default_rng(3)
    N, D, nq = 3000, 64, 20
    sq = np.arange(1, D + 1) ** -0.25
    Q = ((rng.standard_normal((400, D)) * sq) @ np.linalg.qr(rng.standard_normal((D, D)))[0].T).astype(np.float32)
    X = ((rng.standard_normal((N, D)) * np.arange(1, D + 1) ** -0.5) @
         np.linalg.qr(rng.standard_normal((D, D)))[0].T).astype(np.float32)
    tags = np.zeros(N, np.uint16)
    Qt, Xt, tt = _t(Q), _t(X), _t(tags)
    A, B = learn.sphering_init(Qt, Xt, tt, 1, D)          # all D directions, descending order
    store, _ = glv.glv_build_reduced(Xt, tt, B, glv.GLV_F32)   # x' = P' W x, D floats per row
    rs = glv.min_row_stride(D, glv.GLV_F32)
    lists = [rng.permutation(N)[:300] for _ in range(nq)]
    off = np.zeros(nq + 1, np.int64)
    off[1:] = np.cumsum([len(l) for l in lists])
    ids = np.concatenate(lists).astype(np.int32)
    An, Bn = A.cpu().numpy(), B.cpu().numpy()
    Qs = Q[:nq]
    for d in (8, 24, D):
        Ad = A[:, :d, :].contiguous()
        Qp = glv.glv_project_queries(_t(Qs), Ad, glv.GLV_F32)
        got = glv.glv_score_candidates(Qp, store, rs, None, glv.GLV_F32, tt, _t(off), _t(ids), d=d).cpu().numpy()
        ref, _ = oracle.score(oracle.project(Qs, An[:, :d]), oracle.build_reduced(X, tags, Bn[:, :d]), tags, off, ids)
        scale = (np.linalg.norm(oracle.project(Qs, An[:, :d])[:, 0], axis=1)[np.repeat(np.arange(nq), 300)] *
                 np.linalg.norm(oracle.build_reduced(X, tags, Bn[:, :d]), axis=1)[ids])
        ok, worst, _ = scores_close(got, ref, scale, 1e-5)
        assert ok, (d, worst)
    # d = D: the store reproduces the exact inner products (re-rank from the same store)
    ip = np.concatenate([Qs[j].astype(np.float64) @ X[lists[j]].T.astype(np.float64) for j in range(nq)])
    scale = np.linalg.norm(Qs, axis=1)[np.repeat(np.arange(nq), 300)] * np.linalg.norm(X[ids], axis=1)
    assert np.all(np.abs(got - ip) <= 1e-4 * scale)
