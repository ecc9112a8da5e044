"""GPU parity: every C-ABI entry point against the FP64 oracle on the same seeded inputs.

Sizes here finish in seconds on the oracle yet span many tiles, several CTAs per query and
ragged tails (odd d, lists of length 0, 1, < kappa, > the top-k key cache).  Tolerances:
FP32 results within 1e-5 of the oracle relative to max(|s|, ||q_c|| ||x||); integer work
(top-k ids, quantised codes) bit-exact, except where floating point decides between two
valid answers, which is then checked for validity (see oracle/compare.py).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle.compare import scores_close, search_equivalent, topk_equivalent

pytestmark = pytest.mark.gpu

TOL = 1e-5
TIE = 1e-6


@pytest.fixture(scope="module")
def glv():
    from paper_2410_22347_gb300 import build_lib
    build_lib.build()
    from paper_2410_22347_gb300 import glv as g
    return g


def dev():
    return torch.device("cuda:0")


def _rng(s):
    return np.random.default_rng(s)


def _unit(rng, n, D):
    x = rng.standard_normal((n, D))
    return (x / np.linalg.norm(x, axis=1, keepdims=True)).astype(np.float32)


def _csr(lists):
    off = np.zeros(len(lists) + 1, np.int64)
    off[1:] = np.cumsum([len(l) for l in lists])
    ids = np.concatenate([np.asarray(l, np.int32) for l in lists]) if len(lists) else np.zeros(0, np.int32)
    return off, ids.astype(np.int32)


def _t(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to(dev()) if dtype is None else t.to(dev(), dtype)


def _status():
    return torch.zeros(1, dtype=torch.int32, device=dev())


def _ragged_lists(rng, nq, N, lens):
    return [rng.permutation(N)[:L] for L in lens]


def _problem(seed, N=3000, D=96, d=27, C=5, nq=23, orth=True):
    rng = _rng(seed)
    X = _unit(rng, N, D)
    Q = _unit(rng, nq, D)
    mu = _unit(rng, C, D)
    if orth:
        A = np.stack([np.linalg.qr(rng.standard_normal((D, d)))[0].T for _ in range(C)]).astype(np.float32)
        B = A.copy()
    else:
        A = (rng.standard_normal((C, d, D)) / np.sqrt(D)).astype(np.float32)
        B = (rng.standard_normal((C, d, D)) / np.sqrt(D)).astype(np.float32)
    tags = oracle.assign_tags(X, mu)
    return rng, X, Q, mu, A, B, tags


# ---------------------------------------------------------------------------------------
# Eq. (cluster_tag)
# ---------------------------------------------------------------------------------------

# (300, 1024, 40), (2000, 768, 130) and (3000, 128, 1000) stage the landmarks in several
# shared-memory tiles (ragged last tile); the tie 40 = 2 straddles a tile boundary
@pytest.mark.parametrize("N,D,C", [(5000, 96, 7), (1000, 768, 32), (777, 33, 1), (300, 1024, 40),
                                   (2000, 768, 130), (3000, 128, 1000)])
def test_assign_tags(glv, N, D, C):
    rng = _rng(N + D + C)
    X = _unit(rng, N, D)
    mu = _unit(rng, C, D)
    if C > 3:
        mu[3] = mu[1]  # exact ties: the lower index must win
    if C > 40:
        mu[40] = mu[2]
    ref, margin = oracle.assign_tags(X, mu, return_margin=True)
    got = glv.glv_assign_tags(_t(X), _t(mu)).cpu().numpy()
    sure = margin > 1e-5
    np.testing.assert_array_equal(got[sure], ref[sure])
    # near-ties: the GPU's choice must be (within tolerance) a maximiser
    ip = X.astype(np.float64) @ mu.astype(np.float64).T
    best = ip.max(axis=1)
    assert np.all(best - ip[np.arange(N), got] <= 1e-5)
    if C > 3:
        assert not np.any(got == 3)
    if C > 40:
        assert not np.any(got == 40)


# ---------------------------------------------------------------------------------------
# Eq. (X_low): reduced store in FP32 / BF16 / FP8
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("D,d,C,orth", [(96, 27, 5, True), (768, 160, 32, True), (64, 64, 3, False),
                                       (100, 1, 2, False), (512, 130, 9, True)])
def test_build_reduced_f32(glv, D, d, C, orth):
    rng, X, Q, mu, A, B, tags = _problem(D * 7 + d, N=2500, D=D, d=d, C=C, orth=orth)
    tags[::97] = C - 1  # make sure the last cluster is populated
    Xr = oracle.build_reduced(X, tags, B)
    st = _status()
    Xred, _ = glv.glv_build_reduced(_t(X), _t(tags), _t(B), glv.GLV_F32, d_status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    rs = glv.min_row_stride(d, glv.GLV_F32)
    raw = Xred.cpu().numpy()
    got = raw.view(np.float32).reshape(len(X), rs // 4)
    np.testing.assert_array_equal(got[:, d:], 0)  # padding zeroed
    scale = np.linalg.norm(B, axis=2)[tags] * np.linalg.norm(X, axis=1)[:, None]
    ok, worst, bad = scores_close(got[:, :d], Xr, scale, TOL)
    assert ok, f"worst {worst}, bad at {bad[:5]}"


def _f32_down(x):
    y = np.asarray(x, np.float64).astype(np.float32)
    return np.where(y.astype(np.float64) > x, np.nextafter(y, np.float32(-np.inf)), y)


def _f32_up(x):
    y = np.asarray(x, np.float64).astype(np.float32)
    return np.where(y.astype(np.float64) < x, np.nextafter(y, np.float32(np.inf)), y)


@pytest.mark.parametrize("D,d,C", [(96, 27, 5), (768, 160, 32), (512, 128, 64)])
def test_build_reduced_bf16(glv, D, d, C):
    rng, X, Q, mu, A, B, tags = _problem(D + d + 1, N=3000, D=D, d=d, C=C)
    Xr = oracle.build_reduced(X, tags, B)
    ref_codes = oracle.bf16_encode(Xr.astype(np.float32))
    Xred, _ = glv.glv_build_reduced(_t(X), _t(tags), _t(B), glv.GLV_BF16)
    rs = glv.min_row_stride(d, glv.GLV_BF16)
    got_codes = Xred.cpu().numpy().view(np.uint16).reshape(len(X), rs // 2)
    np.testing.assert_array_equal(got_codes[:, d:], 0)
    got_codes = got_codes[:, :d]
    scale = np.linalg.norm(B, axis=2)[tags] * np.linalg.norm(X, axis=1)[:, None]
    gd = oracle.bf16_decode(got_codes)
    tol = TOL * scale
    lo = oracle.bf16_decode(oracle.bf16_encode(_f32_down(Xr - tol)))
    hi = oracle.bf16_decode(oracle.bf16_encode(_f32_up(Xr + tol)))
    bad = ~((gd >= lo) & (gd <= hi))
    ndiff = int((got_codes != ref_codes).sum())
    # every code is the rounding of a value within the tolerance (bad); the codes that differ
    # from the rounding of the exact value are the few whose value lies within the FP32-level
    # error of a rounding boundary: with TF32 hi/lo products (error ~2^-21 of the Cauchy-Schwarz
    # scale) about 0.3% of BF16 codes at D = 512..768, so at most 1% may differ
    assert not bad.any() and ndiff <= max(3, Xr.size // 100), (int(bad.sum()), ndiff)


@pytest.mark.parametrize("D,d,C", [(96, 27, 5), (512, 128, 64), (768, 160, 32), (64, 16, 2)])
def test_build_reduced_fp8(glv, D, d, C):
    rng, X, Q, mu, A, B, tags = _problem(D + d + 2, N=3000, D=D, d=d, C=C)
    X[11] = 0.0  # an all-zero row: scale 0, codes 0
    Xr = oracle.build_reduced(X, tags, B)
    ref_codes, ref_scales = oracle.quantize_fp8_rows(Xr.astype(np.float32))
    Xred, scales = glv.glv_build_reduced(_t(X), _t(tags), _t(B), glv.GLV_FP8_E4M3)
    rs = glv.min_row_stride(d, glv.GLV_FP8_E4M3)
    got_codes = Xred.cpu().numpy().reshape(len(X), rs)
    np.testing.assert_array_equal(got_codes[:, d:], 0)
    got_codes = got_codes[:, :d]
    got_scales = scales.cpu().numpy()
    assert got_scales[11] == 0 and np.all(got_codes[11] == 0)
    rowscale = np.linalg.norm(B, axis=2).max(axis=1)[tags] * np.linalg.norm(X, axis=1)
    assert np.all(np.abs(got_scales - ref_scales) <= TOL * rowscale / 448 + 1e-30)
    gd = oracle.e4m3_decode(got_codes)
    # the GPU rounds x_gpu / s_gpu with |x_gpu - x| <= tol_x: bracket in units of s_gpu
    sg = np.where(got_scales > 0, got_scales, 1).astype(np.float64)[:, None]
    tol_x = TOL * rowscale[:, None]
    slack = np.abs(Xr) / sg * 1e-6  # FP32 division rounding
    lo = oracle.e4m3_decode(oracle.e4m3_encode((Xr - tol_x) / sg - slack))
    hi = oracle.e4m3_decode(oracle.e4m3_encode((Xr + tol_x) / sg + slack))
    bad = ~((gd >= lo) & (gd <= hi))
    bad[11] = False
    ndiff = int((got_codes != ref_codes).sum())
    assert not bad.any() and ndiff <= max(3, Xr.size // 1000), (int(bad.sum()), ndiff)


# ---------------------------------------------------------------------------------------
# Algorithm 4 preprocess: projection GEMM
# ---------------------------------------------------------------------------------------

PROJ_CASES = [(23, 96, 27, 5, True), (300, 768, 160, 32, True), (129, 130, 33, 3, False), (1, 7, 3, 2, False),
              (257, 512, 128, 8, True), (2000, 768, 160, 32, True), (700, 200, 96, 4, False)]


@pytest.mark.parametrize("tensor_cores", [False, True], ids=["simt", "tcgen05-3xtf32"])
@pytest.mark.parametrize("nq,D,d,C,orth", PROJ_CASES)
def test_project_queries_f32(glv, nq, D, d, C, orth, tensor_cores):
    rng, X, Q, mu, A, B, tags = _problem(nq + D, N=10, D=D, d=d, C=C, nq=nq, orth=orth)
    ref = oracle.project(Q, A)
    st = _status()
    got = glv.glv_project_queries(_t(Q), _t(A), glv.GLV_F32, d_status=st, tensor_cores=tensor_cores).cpu().numpy()
    assert st.item() == 0
    scale = np.linalg.norm(A, axis=2)[None] * np.linalg.norm(Q, axis=1)[:, None, None]
    ok, worst, bad = scores_close(got, ref, scale, TOL)
    assert ok, f"worst {worst}"


@pytest.mark.parametrize("nq,D,d,C,orth", PROJ_CASES)
def test_project_queries_bf16(glv, nq, D, d, C, orth):
    """BF16 operands: the product of two BF16 values is exact in FP32, so the tensor-core
    result must match the oracle run on the BF16-rounded operands to FP32 accumulation
    accuracy."""
    rng, X, Q, mu, A, B, tags = _problem(nq + D + 7, N=10, D=D, d=d, C=C, nq=nq, orth=orth)
    Qb = oracle.bf16_decode(oracle.bf16_encode(Q)).astype(np.float32)
    Ab = oracle.bf16_decode(oracle.bf16_encode(A)).astype(np.float32)
    ref = oracle.project(Qb, Ab)
    st = _status()
    got = glv.glv_project_queries(_t(Q), _t(A), glv.GLV_BF16, d_status=st).cpu().numpy()
    assert st.item() == 0
    scale = np.linalg.norm(Ab, axis=2)[None] * np.linalg.norm(Qb, axis=1)[:, None, None]
    ok, worst, bad = scores_close(got, ref, scale, TOL)
    assert ok, f"worst {worst}"


# ---------------------------------------------------------------------------------------
# Algorithm 4 inner-product: gather-score, each store type, fed the oracle's own store
# ---------------------------------------------------------------------------------------

def _score_case(glv, dt, seed, d, C, lens, N=2000, D=64, bad_ids=False):
    rng, X, Q, mu, A, B, tags = _problem(seed, N=N, D=D, d=d, C=C, nq=len(lens))
    Xr = oracle.build_reduced(X, tags, B)
    Qp64 = oracle.project(Q, A)
    Qp32 = Qp64.astype(np.float32)
    lists = _ragged_lists(rng, len(lens), N, lens)
    if bad_ids:
        lists[0] = np.concatenate([lists[0], [N, -3, 2 ** 31 - 1]])
    off, ids = _csr(lists)
    rs = glv.min_row_stride(d, dt) + (16 if seed % 2 else 0)  # also a wider-than-needed stride
    store = np.full((N, rs), 0xAB, np.uint8)  # garbage padding: the kernel must mask it
    scales = None
    if dt == glv.GLV_F32:
        x32 = Xr.astype(np.float32)
        store[:, :4 * d] = x32.view(np.uint8).reshape(N, 4 * d)
        xr_used = x32.astype(np.float64)
    elif dt == glv.GLV_BF16:
        c = oracle.bf16_encode(Xr.astype(np.float32))
        store[:, :2 * d] = c.view(np.uint8).reshape(N, 2 * d)
        xr_used = oracle.bf16_decode(c)
    else:
        c, scales = oracle.quantize_fp8_rows(Xr.astype(np.float32))
        store[:, :d] = c
        xr_used = oracle.dequantize_fp8_rows(c, scales)
    ref, bad = oracle.score(Qp32.astype(np.float64), xr_used, tags, off, ids)
    st = _status()
    got = glv.glv_score_candidates(_t(Qp32), _t(store), rs, None if scales is None else _t(scales), dt,
                                   _t(tags), _t(off), _t(ids), d_status=st).cpu().numpy()
    torch.cuda.synchronize()
    assert (st.item() == glv.GLV_ERR_BAD_ID) == bad_ids == bad
    qn = np.linalg.norm(Qp32.astype(np.float64), axis=2)
    xn = np.linalg.norm(xr_used, axis=1)
    cand_j = np.repeat(np.arange(len(lens)), np.diff(off))
    valid = (ids >= 0) & (ids < N)
    scale = np.zeros(len(ids))
    scale[valid] = qn[cand_j[valid], tags[ids[valid]]] * xn[ids[valid]]
    ok, worst, badpos = scores_close(got, ref, scale, TOL)
    assert ok, f"worst {worst} at {badpos[:5]}"
    assert np.all(np.isneginf(got[~valid]))


@pytest.mark.parametrize("dt_name", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("d", [1, 27, 128, 160, 192])
def test_score_candidates(glv, dt_name, d):
    dt = glv.DTYPES[dt_name]
    lens = [0, 1, 5, 64, 333, 1000, 2000, 7, 0, 1999]
    _score_case(glv, dt, 100 + d, d, 6, lens, D=max(d, 64))


@pytest.mark.parametrize("dt_name", ["f32", "bf16", "fp8"])
def test_score_candidates_wide_rows_and_many_clusters(glv, dt_name):
    # d large enough for the 32-lane path; C large for the shared-memory stage
    dt = glv.DTYPES[dt_name]
    _score_case(glv, dt, 7, 400, 3, [300, 50, 1], N=500, D=512)
    _score_case(glv, dt, 8, 24, 300, [1500, 20], N=1600, D=48)


def test_last_device_status_reports_the_word(glv):
    st = _status()
    assert glv.glv_last_device_status(st) == 0
    st.fill_(glv.GLV_ERR_BAD_ID)
    assert glv.glv_last_device_status(st) == glv.GLV_ERR_BAD_ID


def test_score_candidates_bad_ids_flagged(glv):
    _score_case(glv, glv.GLV_F32, 5, 32, 4, [20, 3], bad_ids=True)


def test_score_candidates_exhaustive_few_queries(glv):
    # few queries with long lists: exercises the split of one query over many CTAs
    _score_case(glv, glv.GLV_BF16, 9, 128, 8, [2000, 2000, 1500], N=2000, D=128)


# ---------------------------------------------------------------------------------------
# top-kappa: bit-exact against the oracle on the same FP32 scores
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("kappa", [1, 10, 100, 257, 1024])
def test_topk_exact(glv, kappa):
    rng = _rng(kappa)
    lens = [0, 1, kappa - 1 if kappa > 1 else 0, kappa, kappa + 1, 3000, 9000, 20000, 50]
    lists = [rng.permutation(100000)[:L] for L in lens]
    off, ids = _csr(lists)
    s = rng.standard_normal(len(ids)).astype(np.float32)
    # planted ties (quantised scores), repeated values, NaN and -inf
    s[::3] = np.round(s[::3], 1)
    s[5::101] = np.nan
    s[7::211] = -np.inf
    s[off[6]:off[6] + 5000] = 3.0  # a huge tie group straddling the kappa boundary
    ref_s, ref_id = oracle.topk(s.astype(np.float64), off, ids, kappa)
    gs, gi = glv.glv_topk(_t(s), _t(off), _t(ids), kappa)
    gs, gi = gs.cpu().numpy(), gi.cpu().numpy()
    np.testing.assert_array_equal(gi, ref_id)
    np.testing.assert_array_equal(gs.astype(np.float64), ref_s)


@pytest.mark.parametrize("kappa", [100, 8, 256])
def test_topk_all_equal_scores(glv, kappa):
    # all-equal lists: beyond the key cache, cached with more tied keys than the packed
    # survivors' room (2048, 2000, 1100), with a few hundred (300, 600), and a list whose
    # 1500 largest scores are equal
    rng = _rng(3)
    lens = [12000, 2048, 2000, 1100, 600, 300, 2000]
    off, ids = _csr([rng.permutation(50000)[:L] for L in lens])
    s = np.ones(len(ids), np.float32)
    s[off[6]:off[6] + 500] = rng.standard_normal(500).astype(np.float32) - 5.0
    ref_s, ref_id = oracle.topk(s.astype(np.float64), off, ids, kappa)
    gs, gi = glv.glv_topk(_t(s), _t(off), _t(ids), kappa)
    np.testing.assert_array_equal(gi.cpu().numpy(), ref_id)
    np.testing.assert_array_equal(gs.cpu().numpy().astype(np.float64), ref_s)


@pytest.mark.parametrize("dt_name", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("kappa", [100, 10, 256])
def test_score_topk_fused_wide_ties(glv, dt_name, kappa):
    """Rows repeat three patterns and the tags alternate, so a query's scores take a handful
    of values and the kappa boundary falls inside tie groups of hundreds to thousands of candidates:
    the fused top-kappa must take the smallest ids of the boundary group, as the oracle does."""
    dt = glv.DTYPES[dt_name]
    rng, X, Q, mu, A, B, _ = _problem(500 + kappa, N=9000, D=64, d=32, C=2, nq=9)
    X = X[np.arange(len(X)) % 3]
    tags = (np.arange(len(X)) % 2).astype(np.uint16)
    lens = [2048, 2000, 1100, 700, 300, 130, 2049, 5000, 0]
    off, ids = _csr(_ragged_lists(rng, 9, len(X), lens))
    Xt, tt = _t(X), _t(tags)
    Xred, scales = glv.glv_build_reduced(Xt, tt, _t(B), dt)
    Qp = glv.glv_project_queries(_t(Q), _t(A), glv.GLV_F32)
    rs = glv.min_row_stride(32, dt)
    offt, idst = _t(off), _t(ids)
    st = _status()
    sc = glv.glv_score_candidates(Qp, Xred, rs, scales, dt, tt, offt, idst, d_status=st)
    fs, fi = glv.glv_score_topk(Qp, Xred, rs, scales, dt, tt, offt, idst, kappa, d_status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    scn = sc.cpu().numpy()
    # six (pattern, tag) values, each possibly in two roundings (the summation order of the
    # low-precision gather depends on the candidate's slot)
    assert len(np.unique(scn[off[0]:off[1]])) <= 12
    ref_s, ref_id = oracle.topk(scn.astype(np.float64), off, ids, kappa)
    np.testing.assert_array_equal(fi.cpu().numpy(), ref_id)
    np.testing.assert_array_equal(fs.cpu().numpy().astype(np.float64), ref_s)


# ---------------------------------------------------------------------------------------
# Algorithm 1 post-processing: exact re-rank
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("D,kappa,k", [(768, 100, 10), (512, 200, 10), (97, 33, 7), (1500, 5, 5),
                                       (64, 1024, 10), (8, 1, 1)])
def test_rerank(glv, D, kappa, k):
    rng = _rng(D + kappa)
    N, nq = 4000, 19
    X = _unit(rng, N, D)
    Q = _unit(rng, nq, D)
    surv = np.array([rng.permutation(N)[:kappa] for _ in range(nq)], np.int32)
    surv[0, kappa // 2:] = -1            # partially empty
    surv[1, :] = -1                      # fully empty
    ref_s, ref_id, _ = oracle.rerank(X, Q, surv, k)
    st = _status()
    gs, gi = glv.glv_rerank(_t(X), _t(Q), _t(surv), k, d_status=st)
    gs, gi = gs.cpu().numpy(), gi.cpu().numpy()
    assert st.item() == 0
    ip = Q.astype(np.float64) @ X.astype(np.float64).T
    for j in range(nq):
        ok, why = topk_equivalent(gi[j], ref_id[j], ref_s[j], lambda i: ip[j, i], TIE)
        assert ok, f"query {j}: {why}"
        v = gi[j] >= 0
        assert np.all(np.abs(gs[j][v] - ip[j, gi[j][v]]) <= TOL)
    assert np.all(gi[1] == -1) and np.all(np.isneginf(gs[1]))


def test_rerank_bad_ids_flagged(glv):
    rng = _rng(11)
    X = _unit(rng, 50, 16)
    Q = _unit(rng, 2, 16)
    surv = np.array([[1, 2, 50, 3], [4, -7, 5, 6]], np.int32)
    st = _status()
    gs, gi = glv.glv_rerank(_t(X), _t(Q), _t(surv), 3, d_status=st)
    torch.cuda.synchronize()
    assert st.item() == glv.GLV_ERR_BAD_ID
    gi = gi.cpu().numpy()
    assert 50 not in gi[0] and -7 not in gi[1]


# ---------------------------------------------------------------------------------------
# whole multi-step search (FP32 store): GPU pipeline vs oracle pipeline
# ---------------------------------------------------------------------------------------

def _pipeline(glv, X, Q, A, B, tags, off, ids, kappa, k, dt):
    st = _status()
    Xt, Qt, tt = _t(X), _t(Q), _t(tags)
    Xred, scales = glv.glv_build_reduced(Xt, tt, _t(B), dt, d_status=st)
    Qp = glv.glv_project_queries(Qt, _t(A), glv.GLV_F32 if dt == glv.GLV_F32 else glv.GLV_BF16, d_status=st)
    rs = glv.min_row_stride(A.shape[1], dt)
    sc = glv.glv_score_candidates(Qp, Xred, rs, scales, dt, tt, _t(off), _t(ids), d_status=st)
    ts, ti = glv.glv_topk(sc, _t(off), _t(ids), kappa)
    fs, fi = glv.glv_rerank(Xt, Qt, ti, k, d_status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    return fs.cpu().numpy(), fi.cpu().numpy()


@pytest.mark.parametrize("seed", [0, 1])
def test_search_pipeline_f32(glv, seed):
    from paper_2410_22347_gb300 import synth
    w = synth.make_workload(N=20000, D=256, d=64, C=12, nq=64, K_db=16, cands=1500, kappa=100, k=10,
                            cfg=80 + seed)
    X, Q, mu, A, B = (t.numpy() for t in (w.X, w.Q, w.mu, w.A, w.B))
    off, ids = w.off.numpy(), w.ids.numpy()
    tags = oracle.assign_tags(X, mu)
    Xr = oracle.build_reduced(X, tags, B)
    ref_s, ref_id = oracle.search(X, Xr, tags, A, Q, off, ids, w.kappa, w.k)
    red, _ = oracle.score(oracle.project(Q, A), Xr, tags, off, ids)
    kap, _ = oracle.topk(red, off, ids, w.kappa)
    fs, fi = _pipeline(glv, X, Q, A, B, tags, off, ids, w.kappa, w.k, glv.GLV_F32)
    for j in range(len(Q)):
        lst = ids[off[j]:off[j + 1]]
        rd = dict(zip(lst.tolist(), red[off[j]:off[j + 1]].tolist()))
        ok, why = search_equivalent(fi[j], ref_id[j], ref_s[j],
                                    lambda i: float(Q[j].astype(np.float64) @ X[i].astype(np.float64)),
                                    lambda i: rd[i], kap[j, -1], TIE, TIE)
        assert ok, f"query {j}: {why}"
    assert oracle.recall(fi, ref_id) >= 0.99


@pytest.mark.parametrize("dt_name", ["bf16", "fp8"])
def test_search_pipeline_low_precision_recall(glv, dt_name):
    """Low-precision stores: the final top-10 (after the exact FP32 re-rank) agrees with the
    FP64 oracle pipeline at 10-recall@10 >= 0.9."""
    from paper_2410_22347_gb300 import synth
    w = synth.make_workload(N=20000, D=256, d=64, C=12, nq=64, K_db=16, cands=1500, kappa=100, k=10,
                            cfg=85)
    X, Q, mu, A, B = (t.numpy() for t in (w.X, w.Q, w.mu, w.A, w.B))
    off, ids = w.off.numpy(), w.ids.numpy()
    tags = oracle.assign_tags(X, mu)
    Xr = oracle.build_reduced(X, tags, B)
    ref_s, ref_id = oracle.search(X, Xr, tags, A, Q, off, ids, w.kappa, w.k)
    fs, fi = _pipeline(glv, X, Q, A, B, tags, off, ids, w.kappa, w.k, glv.DTYPES[dt_name])
    assert oracle.recall(fi, ref_id) >= 0.9


# ---------------------------------------------------------------------------------------
# fused scoring + top-kappa: bit-identical to the two-kernel path
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("dt_name", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("nq,kappa", [(700, 100), (700, 1), (650, 1024), (40, 100)])
def test_score_topk_fused_matches_separate(glv, dt_name, nq, kappa):
    dt = glv.DTYPES[dt_name]
    rng, X, Q, mu, A, B, tags = _problem(nq + kappa, N=17000, D=96, d=40, C=7, nq=nq)
    lens = rng.integers(0, 3000, nq)
    # empty, single, exactly kappa, the on-chip key-cache edge, long lists whose scores spill
    # to the scratch (the selection filters them through the sample threshold), and lists cut
    # into 2 and 4 work items (8192 and 16500 candidates) whose chunk lists are merged
    lens[:7] = [0, 1, kappa, 2048, 2049, 5000, 16500]
    lens[10] = 8192
    lens[11:13] = [4096, 4097]  # the key-cache edge of the wide (512-thread) schedule
    lists = _ragged_lists(rng, nq, len(X), lens)
    lists[7] = np.concatenate([lists[7][:10], [len(X) + 5]])  # a bad id
    # bad ids score -inf and tie there: ties go to the smaller (signed) id, so negative ids
    # come first; list 8's -inf group straddles kappa, list 9 is shorter than kappa
    bad = np.concatenate([-np.arange(1, 121), len(X) + np.arange(130)])
    lists[8] = np.concatenate([lists[8][:max(kappa // 2, 1)], rng.permutation(bad)])
    lists[9] = np.array([-5, 7, len(X) + 5])
    off, ids = _csr(lists)
    st = _status()
    Xt, tt = _t(X), _t(tags)
    Xred, scales = glv.glv_build_reduced(Xt, tt, _t(B), dt)
    Qp = glv.glv_project_queries(_t(Q), _t(A), glv.GLV_F32)
    rs = glv.min_row_stride(40, dt)
    offt, idst = _t(off), _t(ids)
    sc = glv.glv_score_candidates(Qp, Xred, rs, scales, dt, tt, offt, idst, d_status=st)
    ts, ti = glv.glv_topk(sc, offt, idst, kappa)
    st2 = _status()
    fs, fi = glv.glv_score_topk(Qp, Xred, rs, scales, dt, tt, offt, idst, kappa, d_status=st2)
    torch.cuda.synchronize()
    assert st.item() == glv.GLV_ERR_BAD_ID and st2.item() == glv.GLV_ERR_BAD_ID
    np.testing.assert_array_equal(fi.cpu().numpy(), ti.cpu().numpy())
    np.testing.assert_array_equal(fs.cpu().numpy().view(np.uint32), ts.cpu().numpy().view(np.uint32))
    # and the separate path against the oracle's top-kappa of the same FP32 scores
    ref_s, ref_id = oracle.topk(sc.cpu().numpy().astype(np.float64), off, ids, kappa)
    np.testing.assert_array_equal(ti.cpu().numpy(), ref_id)


def test_index_search_matches_oracle(glv):
    """The public index API (projection -> fused score/top-kappa -> re-rank) on a workload with
    enough queries for the fused kernel."""
    from paper_2410_22347_gb300 import synth
    from paper_2410_22347_gb300.index import GleanVecIndex
    w = synth.make_workload(N=30000, D=128, d=32, C=9, nq=800, K_db=12, cands=1000, kappa=50, k=10, cfg=86)
    X, Q, mu, A, B = (t.numpy() for t in (w.X, w.Q, w.mu, w.A, w.B))
    off, ids = w.off.numpy(), w.ids.numpy()
    tags = oracle.assign_tags(X, mu)
    Xr = oracle.build_reduced(X, tags, B)
    ref_s, ref_id = oracle.search(X, Xr, tags, A, Q, off, ids, w.kappa, w.k)
    red, _ = oracle.score(oracle.project(Q, A), Xr, tags, off, ids)
    kap, _ = oracle.topk(red, off, ids, w.kappa)
    ix = GleanVecIndex(_t(X), _t(A), _t(B), tags=_t(tags), store="f32")
    fs, fi = ix.search(_t(Q), _t(off), _t(ids), w.kappa, w.k)
    torch.cuda.synchronize()
    assert ix.device_status() == 0
    fi = fi.cpu().numpy()
    for j in range(len(Q)):
        lst = ids[off[j]:off[j + 1]]
        rd = dict(zip(lst.tolist(), red[off[j]:off[j + 1]].tolist()))
        ok, why = search_equivalent(fi[j], ref_id[j], ref_s[j],
                                    lambda i: float(Q[j].astype(np.float64) @ X[i].astype(np.float64)),
                                    lambda i: rd[i], kap[j, -1], TIE, TIE)
        assert ok, f"query {j}: {why}"
    # host-in / host-out path gives the same answer
    hs, hi = ix.search_host(w.Q.pin_memory(), w.off.pin_memory(), w.ids.pin_memory(), w.kappa, w.k)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(hi.numpy(), fi)


@pytest.mark.parametrize("store,kappa,nq", [("bf16", 0, 700), ("bf16", 40, 700), ("f32", 40, 700),
                                            ("fp8", 40, 700), ("bf16", 40, 50)])
def test_one_call_search_matches_index_search(glv, store, kappa, nq):
    """glv_search (one C call, one workspace) gives exactly the results of the three calls
    (FP32 store with the 3xTF32 projection; 50 queries take the split scoring path)."""
    from paper_2410_22347_gb300 import synth
    from paper_2410_22347_gb300.index import GleanVecIndex
    w = synth.make_workload(N=30000, D=128, d=32, C=9, nq=nq, K_db=12, cands=900, kappa=40, k=10, cfg=88)
    X, Q, A, B, mu = (_t(t.numpy()) for t in (w.X, w.Q, w.A, w.B, w.mu))
    off, ids = _t(w.off.numpy()), _t(w.ids.numpy())
    ix = GleanVecIndex(X, A, B, mu=mu, store=store)
    ws, wi = ix.search(Q, off, ids, kappa, w.k)
    ws, wi = ws.cpu().numpy().copy(), wi.cpu().numpy().copy()
    st = _status()
    gs, gi = glv.glv_search(X, Q, ix.A, ix.compute, ix.Xred, ix.row_stride, ix.scales, ix.dt, ix.tags, off, ids,
                            kappa, w.k, d_status=st)
    assert glv.glv_last_device_status(st) == 0
    np.testing.assert_array_equal(gi.cpu().numpy(), wi)
    np.testing.assert_array_equal(gs.cpu().numpy().view(np.uint32), ws.view(np.uint32))


def test_host_pipeline_matches_search(glv):
    """Batches streamed through HostSearchPipeline (copies of one batch overlapping the search
    of the previous one, slots reused) give exactly the results of search() on each batch."""
    from paper_2410_22347_gb300 import synth
    from paper_2410_22347_gb300.index import GleanVecIndex, HostSearchPipeline
    ws = [synth.make_workload(N=30000, D=128, d=32, C=9, nq=700, K_db=12, cands=900, kappa=40, k=10, cfg=87,
                              replica=r) for r in range(5)]
    X, A, B, mu = (_t(t.numpy()) for t in (ws[0].X, ws[0].A, ws[0].B, ws[0].mu))
    ix = GleanVecIndex(X, A, B, mu=mu, store="bf16")
    want = []
    for w in ws:
        fs, fi = ix.search(_t(w.Q.numpy()), _t(w.off.numpy()), _t(w.ids.numpy()), w.kappa, w.k)
        want.append((fs.cpu().numpy().copy(), fi.cpu().numpy().copy()))
    pipe = HostSearchPipeline(ix, ws[0].kappa, ws[0].k)
    outs = []
    for w in ws + ws[:2]:
        o = (torch.empty(700, 10, dtype=torch.float32, pin_memory=True),
             torch.empty(700, 10, dtype=torch.int32, pin_memory=True))
        pipe.submit(w.Q.pin_memory(), w.off.pin_memory(), w.ids.pin_memory(), *o)
        outs.append(o)
    pipe.synchronize()
    assert ix.device_status() == 0
    for b, (s_h, i_h) in enumerate(outs):
        ws_, wi = want[b % len(ws)]
        np.testing.assert_array_equal(i_h.numpy(), wi)
        np.testing.assert_array_equal(s_h.numpy().view(np.uint32), ws_.view(np.uint32))


# ---------------------------------------------------------------------------------------
# every scoring configuration the autotuner may pick stays exact
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("dt_name", ["f32", "bf16", "fp8"])
def test_every_score_configuration_matches_oracle(glv, dt_name):
    dt = glv.DTYPES[dt_name]
    try:
        for G in glv.SCORE_GROUPS[dt]:
            for mode in glv.GATHER_MODES:
                glv.glv_set_score_config(dt, G, mode)
                for d in (27, 160):
                    _score_case(glv, dt, 300 + G + d, d, 5, [0, 1, 700, 33, 2100, 1500], N=2500, D=max(d, 64))
                    _score_case(glv, dt, 301 + G + d, d, 5, [0, 1, 700, 33, 2100, 1500], N=2500, D=max(d, 64),
                                bad_ids=True)
    finally:
        glv.glv_set_score_config(dt, 0, 0)


@pytest.mark.parametrize("dt_name", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("gi", [0, 1, 2])
def test_fused_matches_separate_in_every_gather_mode(glv, dt_name, mode, gi):
    """Gather modes change only how rows travel; the scores (and so the selections) of the
    fused and the stand-alone (split) paths stay bit-identical for every group size."""
    dt = glv.DTYPES[dt_name]
    G = glv.SCORE_GROUPS[dt][gi]
    try:
        glv.glv_set_score_config(dt, G, mode)
        test_score_topk_fused_matches_separate(glv, dt_name, 700, 100)
        test_score_topk_fused_matches_separate(glv, dt_name, 700, 200)
    finally:
        glv.glv_set_score_config(dt, 0, 0)


def test_score_config_roundtrip(glv):
    try:
        glv.glv_set_score_config(glv.GLV_BF16, 8, 1)
        assert glv.glv_get_score_config(glv.GLV_BF16, 160) == (8, 1, 0, 1)
        # 8 lanes x 5 pipelined loads cannot cover a 160-chunk row: falls back to a default
        g, m, _, _ = glv.glv_get_score_config(glv.GLV_BF16, 1280)
        assert m == 0
        glv.glv_set_score_config(glv.GLV_BF16, 4, 2, 164, 0)
        assert glv.glv_get_score_config(glv.GLV_BF16, 160) == (4, 2, 164, 0)
        with pytest.raises(glv.GlvError):
            glv.glv_set_score_config(glv.GLV_BF16, 4, 0, 0, 8)
        glv.glv_set_score_config(glv.GLV_BF16, 8, 0, 132, 2)
        assert glv.glv_get_score_config(glv.GLV_BF16, 160) == (8, 0, 132, 2)
        glv.glv_set_score_config(glv.GLV_BF16, 8, 1, 0, 3)  # no wide kernel with pipelined loads
        assert glv.glv_get_score_config(glv.GLV_BF16, 160) == (8, 1, 0, 1)
        with pytest.raises(glv.GlvError):
            glv.glv_set_score_config(glv.GLV_BF16, 3, 0)
        with pytest.raises(glv.GlvError):
            glv.glv_set_score_config(glv.GLV_BF16, 4, 3)
        with pytest.raises(glv.GlvError):
            glv.glv_set_score_config(glv.GLV_BF16, 4, 0, 8)
    finally:
        glv.glv_set_score_config(glv.GLV_BF16, 0, 0)


@pytest.mark.parametrize("dt_name", ["bf16", "fp8"])
@pytest.mark.parametrize("kappa", [100, 1024])
def test_carveout_and_schedule_change_no_result(glv, dt_name, kappa):
    """The carveout cap changes only the shared-memory / L1 split, the schedule only how work
    is spread over CTAs: scores and selections stay bit-identical (long lists included)."""
    dt = glv.DTYPES[dt_name]
    try:
        for carve in (0, 164):
            for sched in (1, 0, 3, 2, 5, 6):
                glv.glv_set_score_config(dt, 0, 0, carve, sched)
                test_score_topk_fused_matches_separate(glv, dt_name, 700, kappa)
    finally:
        glv.glv_set_score_config(dt, 0, 0)


@pytest.mark.parametrize("dt_name", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("gi", [0, 1])
@pytest.mark.parametrize("sched", [3, 2])
def test_wide_schedule_matches_separate(glv, dt_name, gi, sched):
    """The 512-thread fused kernel (twice the warps per staged query, lists of up to 4096
    candidates selected on chip) returns exactly what the stand-alone scoring and top-kappa
    return, for both lane counts it is built for, with and without the work plan."""
    dt = glv.DTYPES[dt_name]
    G = glv.SCORE_GROUPS[dt][gi]
    try:
        glv.glv_set_score_config(dt, G, 0, 0, sched)
        assert glv.glv_get_score_config(dt, 40)[3] == sched
        for kappa in (100, 200):
            test_score_topk_fused_matches_separate(glv, dt_name, 700, kappa)
    finally:
        glv.glv_set_score_config(dt, 0, 0)


# ---------------------------------------------------------------------------------------
# lazy inner product (Algorithm 3) against the eager path and the oracle
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("dt_name", ["f32", "bf16", "fp8"])
def test_score_lazy_matches_oracle_and_counts_visited_clusters(glv, dt_name):
    dt = glv.DTYPES[dt_name]
    rng, X, Q, mu, A, B, tags = _problem(77, N=4000, D=96, d=40, C=9, nq=30)
    lens = [0, 1, 5, 64, 700, 2000] + [50] * 24
    lists = _ragged_lists(rng, 30, len(X), lens)
    off, ids = _csr(lists)
    Xred, scales = glv.glv_build_reduced(_t(X), _t(tags), _t(B), dt)
    rs = glv.min_row_stride(40, dt)
    st = _status()
    got, visited = glv.glv_score_lazy(_t(Q), _t(A), Xred, rs, scales, dt, _t(tags), _t(off), _t(ids), d_status=st)
    torch.cuda.synchronize()
    assert st.item() == 0
    # visited-cluster counts are exact
    want_vis = [len(set(tags[l].tolist())) for l in lists]
    np.testing.assert_array_equal(visited.cpu().numpy(), want_vis)
    # scores: the oracle on the store's own decoded rows with the exact projection
    Xr = oracle.build_reduced(X, tags, B)
    if dt == glv.GLV_F32:
        xr_used = Xred.cpu().numpy().view(np.float32)[:, :40].astype(np.float64)
    elif dt == glv.GLV_BF16:
        xr_used = oracle.bf16_decode(Xred.cpu().numpy().view(np.uint16)[:, :40])
    else:
        xr_used = oracle.dequantize_fp8_rows(Xred.cpu().numpy()[:, :40], scales.cpu().numpy())
    Qp = oracle.project(Q, A)
    ref, _ = oracle.score(Qp, xr_used, tags, off, ids)
    cand_j = np.repeat(np.arange(30), np.diff(off))
    scale = np.linalg.norm(Qp, axis=2)[cand_j, tags[ids]] * np.linalg.norm(xr_used, axis=1)[ids]
    ok, worst, bad = scores_close(got.cpu().numpy()[:len(ids)], ref, scale, TOL)
    assert ok, worst


# ---------------------------------------------------------------------------------------
# gather calibration kernel
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("row_bytes", [16, 48, 320, 1024])
def test_gather_rows_sums_whole_rows(glv, row_bytes):
    rng = _rng(row_bytes)
    n_rows = 5000
    vals = rng.integers(-8, 8, size=(n_rows, row_bytes // 4)).astype(np.float32)  # exact sums
    rows = torch.from_numpy(vals.view(np.uint8).reshape(n_rows, row_bytes)).to("cuda:0")
    ids = rng.integers(0, n_rows, size=20011).astype(np.int32)
    ids[17] = n_rows + 3
    ids[18] = -1
    st = _status()
    out = glv.glv_gather_rows(rows, row_bytes, _t(ids), d_status=st)
    torch.cuda.synchronize()
    assert st.item() == glv.GLV_ERR_BAD_ID
    ref = np.where((ids >= 0) & (ids < n_rows), vals[np.clip(ids, 0, n_rows - 1)].sum(axis=1), 0.0)
    np.testing.assert_array_equal(out.cpu().numpy(), ref.astype(np.float32))
