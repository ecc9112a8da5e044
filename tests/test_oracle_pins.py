"""Pins of the FP64 oracle against facts the paper and mathematics fix.

No test here re-types an oracle formula: each one reaches the expected value by a
different route (a hand-worked example, a special case that reduces to a textbook or
library routine, an algebraic identity, an invariance, or brute force on tiny inputs),
chosen so that a dropped term, a wrong sign or index, a transposed operand or a wrong
tie rule in the oracle fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed=0):
    return np.random.default_rng(seed)


def _unit(rng, n, D):
    x = rng.standard_normal((n, D))
    return (x / np.linalg.norm(x, axis=1, keepdims=True)).astype(np.float32)


def _csr(lists):
    off = np.zeros(len(lists) + 1, np.int64)
    off[1:] = np.cumsum([len(l) for l in lists])
    ids = np.concatenate([np.asarray(l, np.int32) for l in lists]) if lists else np.zeros(0, np.int32)
    return off, ids


def _py_rank(pairs):
    """Textbook ordering by Python's sort: NaN last, score descending, id ascending."""
    return sorted(pairs, key=lambda t: (math.isnan(t[0]), -t[0] if not math.isnan(t[0]) else 0.0, t[1]))


# ---------------------------------------------------------------------------------------
# hand-worked example (values derived by hand from the definitions; see the fixture)
# ---------------------------------------------------------------------------------------

def test_worked_example_by_hand():
    g = json.load(open(os.path.join(GOLDEN, "worked_example.json")))
    X = np.array(g["X"], np.float32)
    mu = np.array(g["mu"], np.float32)
    A = np.array(g["A"], np.float32)
    B = np.array(g["B"], np.float32)
    Q = np.array(g["Q"], np.float32)
    off = np.array(g["cand_off"], np.int64)
    ids = np.array(g["cand_ids"], np.int32)

    tags = oracle.assign_tags(X, mu)
    assert tags.tolist() == g["tags"]
    Xr = oracle.build_reduced(X, tags, B)
    np.testing.assert_array_equal(Xr, np.array(g["Xr"], float))
    Qp = oracle.project(Q, A)
    np.testing.assert_array_equal(Qp, np.array(g["Qp"], float))
    s, bad = oracle.score(Qp, Xr, tags, off, ids)
    assert not bad
    np.testing.assert_array_equal(s, np.array(g["scores"], float))
    for kappa, k in ((2, 1), (3, 2)):
        ts, ti = oracle.topk(s, off, ids, kappa)
        ref = g[f"topk_kappa{kappa}"]
        assert ti.tolist() == ref["ids"]
        np.testing.assert_array_equal(ts, np.array(ref["scores"], float))
        rs, ri, bad = oracle.rerank(X, Q, ti, k)
        ref = g[f"rerank_kappa{kappa}_k{k}"]
        assert ri.tolist() == ref["ids"] and not bad
        np.testing.assert_array_equal(rs, np.array(ref["scores"], float))
        fs, fi = oracle.search(X, Xr, tags, A, Q, off, ids, kappa, k)
        assert fi.tolist() == ref["ids"]
    es, ei = oracle.exact_topk(X, Q, off, ids, 3)
    assert ei.tolist() == g["exact_top3"]["ids"]
    np.testing.assert_array_equal(es, np.array(g["exact_top3"]["scores"], float))


# ---------------------------------------------------------------------------------------
# invariant (i): d = D and A_c = B_c = I reduce the GleanVec score to the exact inner
# product <q, x> (Eq. GleanVec approximation with identity maps), computed here by BLAS.
# ---------------------------------------------------------------------------------------

def test_identity_maps_give_exact_inner_product():
    rng = _rng(1)
    N, D, C, nq = 300, 24, 5, 7
    X = _unit(rng, N, D)
    Q = _unit(rng, nq, D)
    mu = _unit(rng, C, D)
    I = np.broadcast_to(np.eye(D, dtype=np.float32), (C, D, D)).copy()
    tags = oracle.assign_tags(X, mu)
    Xr = oracle.build_reduced(X, tags, I)
    Qp = oracle.project(Q, I)
    off, ids = _csr([rng.permutation(N)[:50 + 10 * j] for j in range(nq)])
    s, _ = oracle.score(Qp, Xr, tags, off, ids)
    ip = Q.astype(np.float64) @ X.astype(np.float64).T
    ref = np.concatenate([ip[j, ids[off[j]:off[j + 1]]] for j in range(nq)])
    np.testing.assert_allclose(s, ref, rtol=0, atol=1e-13)


# ---------------------------------------------------------------------------------------
# invariant (ii): C = 1 is linear LeanVec, <A q, B x> (Section 2.1), by BLAS matmuls;
# and C > 1 with every cluster holding the same (A, B) is the same LeanVec score.
# ---------------------------------------------------------------------------------------

def test_single_cluster_is_linear_leanvec():
    rng = _rng(2)
    N, D, d, nq = 200, 32, 7, 5
    X = _unit(rng, N, D)
    Q = _unit(rng, nq, D)
    A1 = rng.standard_normal((1, d, D)).astype(np.float32)
    B1 = rng.standard_normal((1, d, D)).astype(np.float32)
    off, ids = _csr([rng.permutation(N)[:40] for _ in range(nq)])
    lean = (Q.astype(np.float64) @ A1[0].T.astype(np.float64)) @ (
        X.astype(np.float64) @ B1[0].T.astype(np.float64)).T
    ref = np.concatenate([lean[j, ids[off[j]:off[j + 1]]] for j in range(nq)])

    tags1 = np.zeros(N, np.uint16)
    s1, _ = oracle.score(oracle.project(Q, A1), oracle.build_reduced(X, tags1, B1), tags1, off, ids)
    np.testing.assert_allclose(s1, ref, rtol=1e-12, atol=1e-12)

    C = 6
    tagsC = rng.integers(0, C, N).astype(np.uint16)
    AC = np.repeat(A1, C, axis=0)
    BC = np.repeat(B1, C, axis=0)
    sC, _ = oracle.score(oracle.project(Q, AC), oracle.build_reduced(X, tagsC, BC), tagsC, off, ids)
    np.testing.assert_allclose(sC, ref, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------------------------------
# bilinear identity: <A_c q, B_c x> = q^T (A_c^T B_c) x.  The D x D matrix M_c is formed
# by numpy and applied per candidate; distinct non-symmetric A_c != B_c per cluster make
# a transposed operand, a swapped A/B or a wrong tag lookup fail.
# ---------------------------------------------------------------------------------------

def test_scores_match_bilinear_form():
    rng = _rng(3)
    N, D, d, C, nq = 150, 20, 6, 4, 6
    X = _unit(rng, N, D)
    Q = _unit(rng, nq, D)
    A = rng.standard_normal((C, d, D)).astype(np.float32)
    B = rng.standard_normal((C, d, D)).astype(np.float32)
    tags = rng.integers(0, C, N).astype(np.uint16)
    off, ids = _csr([rng.permutation(N)[:30 + j] for j in range(nq)])
    s, _ = oracle.score(oracle.project(Q, A), oracle.build_reduced(X, tags, B), tags, off, ids)
    M = np.einsum("cri,crk->cik", A.astype(np.float64), B.astype(np.float64))
    ref = []
    for j in range(nq):
        for i in ids[off[j]:off[j + 1]]:
            ref.append(Q[j].astype(np.float64) @ M[tags[i]] @ X[i].astype(np.float64))
    np.testing.assert_allclose(s, np.array(ref), rtol=1e-11, atol=1e-11)


def test_bad_ids_flagged_and_skipped():
    rng = _rng(4)
    N, D, d, C = 20, 8, 3, 2
    X = _unit(rng, N, D)
    A = rng.standard_normal((C, d, D)).astype(np.float32)
    tags = rng.integers(0, C, N).astype(np.uint16)
    Q = _unit(rng, 1, D)
    off, ids = _csr([[0, N, -5, 3]])
    s, bad = oracle.score(oracle.project(Q, A), oracle.build_reduced(X, tags, A), tags, off, ids)
    assert bad and np.isneginf(s[1]) and np.isneginf(s[2]) and np.isfinite(s[0]) and np.isfinite(s[3])
    _, _, bad = oracle.rerank(X, Q, np.array([[0, N]], np.int32), 1)
    assert bad


# ---------------------------------------------------------------------------------------
# invariant (iii): permuting the database (rows, tags, and the ids in the lists with
# them) permutes nothing in the results but the ids.
# ---------------------------------------------------------------------------------------

def test_permutation_invariance():
    rng = _rng(5)
    N, D, d, C, nq = 400, 16, 5, 3, 8
    X = _unit(rng, N, D)
    Q = _unit(rng, nq, D)
    mu = _unit(rng, C, D)
    A = rng.standard_normal((C, d, D)).astype(np.float32)
    B = rng.standard_normal((C, d, D)).astype(np.float32)
    tags = oracle.assign_tags(X, mu)
    Xr = oracle.build_reduced(X, tags, B)
    off, ids = _csr([rng.permutation(N)[:60] for _ in range(nq)])
    fs, fi = oracle.search(X, Xr, tags, A, Q, off, ids, 20, 5)
    s, _ = oracle.score(oracle.project(Q, A), Xr, tags, off, ids)

    perm = rng.permutation(N)           # new row r holds old row perm[r]
    inv = np.empty(N, np.int64)
    inv[perm] = np.arange(N)
    Xp = X[perm]
    tagsp = oracle.assign_tags(Xp, mu)
    np.testing.assert_array_equal(tagsp, tags[perm])
    Xrp = oracle.build_reduced(Xp, tagsp, B)
    idsp = inv[ids].astype(np.int32)
    sp, _ = oracle.score(oracle.project(Q, A), Xrp, tagsp, off, idsp)
    np.testing.assert_array_equal(sp, s)
    # ids change under the permutation, so ties may resolve differently; compare the
    # score sequence and the id sets mapped back
    fsp, fip = oracle.search(Xp, Xrp, tagsp, A, Q, off, idsp, 20, 5)
    np.testing.assert_array_equal(fsp, fs)
    for j in range(nq):
        assert sorted(perm[fip[j]].tolist()) == sorted(fi[j].tolist())


# ---------------------------------------------------------------------------------------
# invariant (iv): top-k against brute force (Python's sort) on tiny inputs with planted
# ties, NaNs, -inf and lists shorter than kappa.
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_topk_brute_force(seed):
    rng = _rng(10 + seed)
    nq = 9
    lists, scores = [], []
    for j in range(nq):
        L = int(rng.integers(0, 40))
        ids = rng.permutation(64)[:L]
        s = np.round(rng.standard_normal(L), 1)       # rounding plants many ties
        if L > 3:
            s[rng.integers(0, L)] = np.nan
            s[rng.integers(0, L)] = -np.inf
        lists.append(ids)
        scores.append(s)
    off, ids = _csr(lists)
    s = np.concatenate(scores) if scores else np.zeros(0)
    for kappa in (1, 5, 17, 45):
        ts, ti = oracle.topk(s, off, ids, kappa)
        for j in range(nq):
            ref = _py_rank(list(zip(scores[j].tolist(), lists[j].tolist())))[:kappa]
            ref_ids = [t[1] for t in ref] + [-1] * (kappa - len(ref))
            assert ti[j].tolist() == ref_ids
            for t, (rs, _) in enumerate(ref):
                assert (math.isnan(rs) and math.isnan(ts[j, t])) or ts[j, t] == rs
            assert np.all(np.isneginf(ts[j, len(ref):]))


def test_rerank_and_exact_topk_brute_force():
    rng = _rng(20)
    N, D, nq = 64, 8, 10
    X = np.round(rng.standard_normal((N, D)), 1).astype(np.float32)
    X[7] = X[3]                                       # duplicate rows: exact ties
    Q = np.round(rng.standard_normal((nq, D)), 1).astype(np.float32)
    surv = np.array([rng.permutation(N)[:12] for _ in range(nq)], np.int32)
    surv[:, 3] = 3
    surv[:, 4] = 7
    surv[0, 5:] = -1                                  # empty slots
    ip = Q.astype(np.float64) @ X.astype(np.float64).T
    for k in (1, 4, 12):
        rs, ri, bad = oracle.rerank(X, Q, surv, k)
        assert not bad
        for j in range(nq):
            cand = [int(i) for i in surv[j] if i >= 0]
            ref = _py_rank([(ip[j, i], i) for i in cand])[:k]
            assert ri[j].tolist() == [t[1] for t in ref] + [-1] * (k - len(ref))
    off, ids = _csr([surv[j][surv[j] >= 0] for j in range(nq)])
    es, ei = oracle.exact_topk(X, Q, off, ids, 4)
    rs, ri, _ = oracle.rerank(X, Q, surv, 4)
    np.testing.assert_array_equal(ei, ri)


def test_assign_tags_brute_force():
    rng = _rng(21)
    N, D, C = 500, 12, 7
    X = _unit(rng, N, D)
    mu = _unit(rng, C, D)
    mu[5] = mu[2]                                     # identical landmarks: every tie -> 2
    tags, margin = oracle.assign_tags(X, mu, return_margin=True)
    ref = np.argmax(X.astype(np.float64) @ mu.astype(np.float64).T, axis=1)  # first max
    np.testing.assert_array_equal(tags, ref)
    assert not np.any(tags == 5)
    srt = np.sort(X.astype(np.float64) @ mu.astype(np.float64).T, axis=1)
    np.testing.assert_allclose(margin, srt[:, -1] - srt[:, -2], atol=1e-14)


# ---------------------------------------------------------------------------------------
# whole search against an independent numpy pipeline
# ---------------------------------------------------------------------------------------

def test_search_matches_numpy_pipeline():
    rng = _rng(22)
    N, D, d, C, nq, kappa, k = 500, 24, 6, 4, 12, 25, 5
    X = _unit(rng, N, D)
    Q = _unit(rng, nq, D)
    A = rng.standard_normal((C, d, D)).astype(np.float32)
    B = rng.standard_normal((C, d, D)).astype(np.float32)
    tags = rng.integers(0, C, N).astype(np.uint16)
    off, ids = _csr([rng.permutation(N)[:int(rng.integers(1, 90))] for _ in range(nq)])
    Xr = oracle.build_reduced(X, tags, B)
    fs, fi = oracle.search(X, Xr, tags, A, Q, off, ids, kappa, k)
    M = np.einsum("cri,crk->cik", A.astype(np.float64), B.astype(np.float64))
    ip = Q.astype(np.float64) @ X.astype(np.float64).T
    for j in range(nq):
        cand = ids[off[j]:off[j + 1]]
        sc = np.array([Q[j].astype(np.float64) @ M[tags[i]] @ X[i].astype(np.float64) for i in cand])
        order = np.lexsort((cand, -sc))[:kappa]
        surv = cand[order]
        order2 = np.lexsort((surv, -ip[j, surv]))[:k]
        ref = surv[order2].tolist()
        assert fi[j].tolist() == ref + [-1] * (k - len(ref))


# ---------------------------------------------------------------------------------------
# scalar quantisation: BF16 and FP8-e4m3 against torch's own conversions (library
# routines), the full 256-code table, ties-to-even, and the quantisation error bound.
# ---------------------------------------------------------------------------------------

def test_bf16_encode_decode_against_torch():
    rng = _rng(30)
    x = np.concatenate([rng.standard_normal(20000).astype(np.float32) * 10.0 ** rng.integers(-30, 30, 20000),
                        np.array([0.0, -0.0, 1.0, -1.0, 3.0e38, -3.0e38, 1e-40, -1e-40,
                                  np.inf, -np.inf], np.float32)]).astype(np.float32)
    # exact ties: 1 + 2^-8 lies halfway between two bf16 values
    x = np.concatenate([x, np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8)], np.float32)])
    codes = oracle.bf16_encode(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(codes, ref)
    dec = oracle.bf16_decode(codes)
    ref_dec = torch.from_numpy(ref.view(np.int16)).view(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(dec, ref_dec)


def test_e4m3_full_code_table_against_torch():
    codes = np.arange(256, dtype=np.uint8)
    dec = oracle.e4m3_decode(codes)
    ref = torch.from_numpy(codes).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    nan = np.isnan(ref)
    assert nan.sum() == 2 and np.isnan(dec[nan]).all()
    np.testing.assert_array_equal(dec[~nan], ref[~nan])
    assert np.nanmax(dec) == 448.0 and np.nanmin(np.abs(dec[dec != 0])) == 2.0 ** -9


def test_e4m3_encode_against_torch_and_ties_to_even():
    rng = _rng(31)
    x = rng.uniform(-448, 448, 50000) * 10.0 ** rng.uniform(-4, 0, 50000)
    x = np.concatenate([x, [0.0, 448.0, -448.0, 2.0 ** -9, 2.0 ** -10, 3 * 2.0 ** -11]])
    x32 = x.astype(np.float32)
    codes = oracle.e4m3_encode(x32.astype(np.float64))
    ref = torch.from_numpy(x32).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    np.testing.assert_array_equal(codes, ref)
    # midpoints between consecutive finite magnitudes go to the even code
    vals = oracle.e4m3_decode(np.arange(127, dtype=np.uint8))
    mids = 0.5 * (vals[:-1] + vals[1:])
    mc = oracle.e4m3_encode(mids)
    assert np.all(mc % 2 == 0)
    # saturation (no infinities in e4m3)
    assert oracle.e4m3_encode(np.array([1e6, -1e6, 449.0]))[:].tolist() == [0x7E, 0xFE, 0x7E]


def test_fp8_row_quantisation_error_bound():
    rng = _rng(32)
    x = rng.standard_normal((300, 77)).astype(np.float32) * 10.0 ** rng.uniform(-3, 1, (300, 1)).astype(np.float32)
    x[5] = 0.0
    codes, scales = oracle.quantize_fp8_rows(x)
    assert scales[5] == 0 and np.all(codes[5] == 0)
    mx = np.abs(x).max(axis=1)
    np.testing.assert_array_equal(scales, (mx / np.float32(448.0)).astype(np.float32))
    deq = oracle.dequantize_fp8_rows(codes, scales)
    # e4m3 keeps 3 mantissa bits: half-ulp error <= 2^-4 relative in the normal range and
    # <= 2^-10 (half the 2^-9 spacing) in units of the scale in the subnormal range
    y = x.astype(np.float64) / scales[:, None].astype(np.float64).clip(1e-300)
    bound = np.maximum(np.abs(y) * 2.0 ** -4, 2.0 ** -10) * scales[:, None] * (1 + 1e-6)
    err = np.abs(deq - x.astype(np.float64))
    assert np.all(err <= bound)
    assert np.all(np.abs(codes[np.arange(300) != 5].astype(np.int64) & 0x7F).max(axis=1) == 0x7E)


# ---------------------------------------------------------------------------------------
# LeanVec-Sphering (Section 3, Algorithm 2 in the eigen form of Section 3.2)
# ---------------------------------------------------------------------------------------

def _ood_sets(rng, D, nq, nx):
    sq = np.arange(1, D + 1) ** -0.25
    sx = np.arange(1, D + 1) ** -0.5
    Rq = np.linalg.qr(rng.standard_normal((D, D)))[0]
    Rx = np.linalg.qr(rng.standard_normal((D, D)))[0]
    Q = (rng.standard_normal((nq, D)) * sq) @ Rq.T
    X = (rng.standard_normal((nx, D)) * sx) @ Rx.T
    return Q.astype(np.float32), X.astype(np.float32)


def test_second_moment_against_blas():
    rng = _rng(40)
    V = rng.standard_normal((200, 9)).astype(np.float32)
    tags = rng.integers(0, 3, 200).astype(np.uint16)
    np.testing.assert_allclose(oracle.second_moment(V), V.T.astype(np.float64) @ V.astype(np.float64), rtol=1e-13)
    sel = V[tags == 1].astype(np.float64)
    np.testing.assert_allclose(oracle.second_moment(V, tags, 1), sel.T @ sel, rtol=1e-13)


def test_sphering_identities():
    rng = _rng(41)
    D, d = 10, 4
    Q, X = _ood_sets(rng, D, 60, 80)
    KQ = oracle.second_moment(Q)
    KX = oracle.second_moment(X)
    A, B, W, lam = oracle.sphering_from_moments(KQ, KX, d)
    # Eq. (QQt identities): W^T W = Q Q^T
    np.testing.assert_allclose(W.T @ W, KQ, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(W, W.T, atol=1e-12)
    # P row-orthonormal: A B^T = P W^-1 W P^T = I_d
    np.testing.assert_allclose(A @ B.T, np.eye(d), atol=1e-9)
    # d = D: A^T B = I, so <A q, B x> = <q, x> exactly (Section 3.1)
    AD, BD, _, _ = oracle.sphering_from_moments(KQ, KX, D)
    np.testing.assert_allclose(AD.T @ BD, np.eye(D), atol=1e-9)


def test_sphering_loss_is_tail_eigenvalue_sum():
    """Brute-force LeanVec loss over all (q, x) pairs (Section 2.1 problem) at the
    Sphering solution equals sum_{i>d} lambda_i(W K_X W): Eq. (LeanVec-Sphering) turns
    the loss into sum_x ||(P^T P - I) W x||^2, which a d-row orthonormal P minimises at
    the tail of the spectrum."""
    rng = _rng(42)
    D, d = 9, 3
    Q, X = _ood_sets(rng, D, 25, 30)
    KQ = oracle.second_moment(Q)
    KX = oracle.second_moment(X)
    A, B, W, lam = oracle.sphering_from_moments(KQ, KX, d)
    qi, xi = np.meshgrid(np.arange(25), np.arange(30), indexing="ij")
    tags = np.zeros(30, np.uint16)
    loss = oracle.pair_loss_grad(Q, X, tags, A[None].astype(np.float32), B[None].astype(np.float32),
                                 qi.ravel(), xi.ravel(), want_grad=False)
    np.testing.assert_allclose(loss, lam[d:].sum(), rtol=2e-5)
    # a random row-orthonormal pair does worse on this OOD data (Section 5.1 claim)
    P = np.linalg.qr(rng.standard_normal((D, d)))[0].T.astype(np.float32)
    worse = oracle.pair_loss_grad(Q, X, tags, P[None], P[None], qi.ravel(), xi.ravel(), want_grad=False)
    assert worse > loss


# ---------------------------------------------------------------------------------------
# gradients of the pair loss: closed form on full cross products, and central finite
# differences (the loss is quadratic in each single entry, so FD is exact up to rounding)
# ---------------------------------------------------------------------------------------

def test_pair_gradients_closed_form_and_fd():
    rng = _rng(43)
    D, d, C = 6, 3, 2
    Q = rng.standard_normal((5, D)).astype(np.float32)
    X = rng.standard_normal((8, D)).astype(np.float32)
    tags = np.array([0, 1, 0, 1, 1, 0, 0, 1], np.uint16)
    A = rng.standard_normal((C, d, D)).astype(np.float32)
    B = rng.standard_normal((C, d, D)).astype(np.float32)
    qi, xi = np.meshgrid(np.arange(5), np.arange(8), indexing="ij")
    loss, gA, gB = oracle.pair_loss_grad(Q, X, tags, A, B, qi.ravel(), xi.ravel())
    KQ = Q.T.astype(np.float64) @ Q.astype(np.float64)
    total = 0.0
    for c in range(C):
        Xc = X[tags == c].astype(np.float64)
        KX = Xc.T @ Xc
        Ac, Bc = A[c].astype(np.float64), B[c].astype(np.float64)
        M = np.eye(D) - Ac.T @ Bc
        total += np.trace(M.T @ KQ @ M @ KX)
        np.testing.assert_allclose(gA[c], -2 * Bc @ KX @ M.T @ KQ, rtol=1e-10, atol=1e-9)
        np.testing.assert_allclose(gB[c], -2 * Ac @ KQ @ M @ KX, rtol=1e-10, atol=1e-9)
    np.testing.assert_allclose(loss, total, rtol=1e-11)
    # central differences with a step of about 1e-3 (2^-10, so that a +- h stays exactly
    # representable in the float32 matrices)
    h = 2.0 ** -10
    for (c, r, k) in [(0, 0, 0), (1, 2, 5), (0, 1, 3)]:
        for which, G in (("A", gA), ("B", gB)):
            Ap, Am, Bp, Bm = A.copy(), A.copy(), B.copy(), B.copy()
            if which == "A":
                Ap[c, r, k] += h
                Am[c, r, k] -= h
            else:
                Bp[c, r, k] += h
                Bm[c, r, k] -= h
            lp = oracle.pair_loss_grad(Q, X, tags, Ap, Bp, qi.ravel(), xi.ravel(), want_grad=False)
            lm = oracle.pair_loss_grad(Q, X, tags, Am, Bm, qi.ravel(), xi.ravel(), want_grad=False)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - G[c, r, k]) <= 1e-8 * max(1.0, abs(G[c, r, k]))


# ---------------------------------------------------------------------------------------
# spherical k-means (Appendix A)
# ---------------------------------------------------------------------------------------

def test_kmeans_update_against_segment_sums():
    rng = _rng(50)
    N, D, C = 700, 12, 6
    X = _unit(rng, N, D)
    tags = rng.integers(0, C - 1, N).astype(np.uint16)        # cluster C-1 stays empty
    mu_in = _unit(rng, C, D)
    mu, counts = oracle.kmeans_update(X, tags, mu_in)
    sums = np.zeros((C, D))
    np.add.at(sums, tags, X.astype(np.float64))
    for c in range(C - 1):
        np.testing.assert_allclose(mu[c], sums[c] / np.linalg.norm(sums[c]), rtol=1e-12, atol=1e-14)
    np.testing.assert_array_equal(mu[C - 1], mu_in[C - 1].astype(np.float64))
    np.testing.assert_array_equal(counts, np.bincount(tags, minlength=C))


def test_kmeans_update_is_the_optimal_unit_landmark():
    """For fixed assignments the normalised sum maximises sum_i <x_i, mu> over unit mu
    (Cauchy-Schwarz), so no random unit vector does better."""
    rng = _rng(51)
    X = _unit(rng, 300, 8)
    tags = np.zeros(300, np.uint16)
    mu, _ = oracle.kmeans_update(X, tags, _unit(rng, 1, 8))
    best = X.astype(np.float64).sum(0) @ mu[0]
    trials = _unit(rng, 2000, 8).astype(np.float64) @ X.astype(np.float64).sum(0)
    assert best >= trials.max() - 1e-12


def test_spherical_kmeans_em_is_monotone():
    rng = _rng(52)
    X = _unit(rng, 2000, 16)
    mu = X[rng.choice(2000, 7, replace=False)].copy()
    prev = -np.inf
    for _ in range(6):
        tags = oracle.assign_tags(X, mu)
        obj_e = oracle.spherical_objective(X, mu, tags)
        assert obj_e >= prev - 1e-9
        mu64, _ = oracle.kmeans_update(X, tags, mu)
        mu = mu64.astype(np.float32)
        prev = oracle.spherical_objective(X, mu, tags)
        assert prev >= obj_e - 1e-4      # the M-step does not lower the objective


# ---------------------------------------------------------------------------------------
# recall (Section 5: k-recall@k = |S cap G| / k, averaged over queries)
# ---------------------------------------------------------------------------------------

def test_recall_hand_counted():
    """Counted by hand: query 0 finds {2, 3} of its truth {3, 2, 9, 10} (its -1 slot is empty);
    query 1 finds all four of {8, 7, 6, 5} in another order; (2 + 4) / (4 * 2) = 0.75."""
    found = [[1, 2, 3, -1], [5, 6, 7, 8]]
    truth = [[3, 2, 9, 10], [8, 7, 6, 5]]
    assert oracle.recall(found, truth) == 0.75


def test_recall_uses_the_truth_width_and_ignores_empty_slots():
    # K is the truth's width (here 2), even when more ids were returned
    assert oracle.recall([[4, 5, 6]], [[6, 9]]) == 0.5
    # -1 marks an empty slot on either side and never counts as a hit
    assert oracle.recall([[-1, -1]], [[-1, -1]]) == 0.0
    assert oracle.recall([[7, -1]], [[7, -1]]) == 0.5
    # duplicates are not counted twice
    assert oracle.recall([[7, 7]], [[7, 8]]) == 0.5
