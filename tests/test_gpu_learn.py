"""GPU parity of the learning side: FP64 second moments, the per-cluster LeanVec-Sphering
initialisation, the pair forward and the hand-written backward (against the FP64 oracle
gradient and central finite differences), and that refinement lowers the loss."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def learn():
    from paper_2410_22347_gb300 import build_lib
    build_lib.build()
    from paper_2410_22347_gb300 import learn as L
    return L


def dev():
    return torch.device("cuda:0")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def _sets(seed, D, nq, nx, C):
    rng = np.random.default_rng(seed)
    sq = np.arange(1, D + 1) ** -0.25
    sx = np.arange(1, D + 1) ** -0.5
    Rq = np.linalg.qr(rng.standard_normal((D, D)))[0]
    Rx = np.linalg.qr(rng.standard_normal((D, D)))[0]
    Q = ((rng.standard_normal((nq, D)) * sq) @ Rq.T).astype(np.float32)
    X = ((rng.standard_normal((nx, D)) * sx) @ Rx.T).astype(np.float32)
    mu = X[rng.choice(nx, C, replace=False)]
    return rng, Q, X, mu


@pytest.mark.parametrize("n,D,C", [(1000, 64, 1), (3000, 100, 5), (777, 33, 3), (5000, 256, 16)])
def test_second_moments(learn, n, D, C):
    rng, Q, X, mu = _sets(n + D, D, 10, n, max(C, 1))
    tags = oracle.assign_tags(X, mu) if C > 1 else None
    K = learn.glv_second_moments(_t(X), None if tags is None else _t(tags), C).cpu().numpy()
    for c in range(C):
        ref = oracle.second_moment(X, tags, c if tags is not None else -1)
        np.testing.assert_allclose(K[c], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_sphering_init_identities_and_oracle(learn):
    """The product's per-cluster A_c, B_c (GPU FP64 moments, Cholesky-whitened Sphering) satisfy
    Section 3.2's identities on the oracle's own moments -- W^T W = K_Q, A_c B_c^T = I_d, and
    the loss over all learning pairs of cluster c equals the sum of the D - d smallest
    eigenvalues of K_Q K_{X_c} -- and agree with the oracle's symmetric-square-root route in
    A_c^T B_c and in the loss they reach."""
    D, d, C = 48, 12, 4
    rng, Q, X, mu = _sets(5, D, 400, 3000, C)
    tags = oracle.assign_tags(X, mu)
    A, B = learn.sphering_init(_t(Q), _t(X), _t(tags), C, d)
    A, B = A.cpu().numpy().astype(np.float64), B.cpu().numpy().astype(np.float64)
    KQ = oracle.second_moment(Q)
    KQ_gpu = learn.glv_second_moments(_t(Q))[0].cpu().numpy()
    _, _, W, _ = learn.sphering_factors(KQ_gpu, KQ_gpu, d)
    np.testing.assert_allclose(W.T @ W, KQ, rtol=0, atol=1e-10 * np.abs(KQ).max())
    Ar, Br = oracle.gleanvec_sphering(Q, X, tags, C, d)
    for c in range(C):
        KX = oracle.second_moment(X, tags, c)
        # A_c, B_c are FP32 on the device: identities hold to FP32 accuracy of the factors
        np.testing.assert_allclose(A[c] @ B[c].T, np.eye(d), rtol=0, atol=2e-5)
        R = np.eye(D) - A[c].T @ B[c]
        loss = float(np.trace(R.T @ KQ @ R @ KX))
        ev = np.sort(np.linalg.eigvals(KQ @ KX).real)
        tail = float(ev[: D - d].sum())
        assert abs(loss - tail) <= 1e-4 * tail + 1e-6 * float(ev.sum()), (c, loss, tail)
        # eigenvector signs are arbitrary; A_c^T B_c (the reduction's bilinear form) is not
        np.testing.assert_allclose(A[c].T @ B[c], Ar[c].T @ Br[c], atol=2e-5)
    # and the loss each side reaches on sampled pairs is the same
    qi, xi = np.meshgrid(np.arange(400), np.arange(3000), indexing="ij")
    sel = np.random.default_rng(1).choice(qi.size, 20000, replace=False)
    l_gpu = oracle.pair_loss_grad(Q, X, tags, A.astype(np.float32), B.astype(np.float32), qi.ravel()[sel],
                                  xi.ravel()[sel], want_grad=False)
    l_ref = oracle.pair_loss_grad(Q, X, tags, Ar.astype(np.float32), Br.astype(np.float32), qi.ravel()[sel],
                                  xi.ravel()[sel], want_grad=False)
    assert abs(l_gpu - l_ref) <= 1e-4 * l_ref


def test_sphering_init_is_exact_at_full_dimension(learn):
    """d = D: A_c^T B_c = I, so every reduced inner product equals the exact one."""
    D, C = 24, 3
    rng, Q, X, mu = _sets(6, D, 200, 1500, C)
    tags = oracle.assign_tags(X, mu)
    A, B = learn.sphering_init(_t(Q), _t(X), _t(tags), C, D)
    A, B = A.cpu().numpy().astype(np.float64), B.cpu().numpy().astype(np.float64)
    for c in range(C):
        np.testing.assert_allclose(A[c].T @ B[c], np.eye(D), rtol=0, atol=5e-5)


@pytest.mark.parametrize("D,d,C,P", [(64, 16, 3, 500), (128, 32, 16, 4096), (100, 27, 5, 1000)])
def test_pair_forward_and_backward_vs_oracle(learn, D, d, C, P):
    rng, Q, X, mu = _sets(D + P, D, 300, 2000, C)
    tags = oracle.assign_tags(X, mu)
    A = (rng.standard_normal((C, d, D)) / np.sqrt(D)).astype(np.float32)
    B = (rng.standard_normal((C, d, D)) / np.sqrt(D)).astype(np.float32)
    qi = rng.integers(0, 300, P).astype(np.int32)
    xi = rng.integers(0, 2000, P).astype(np.int32)
    st = torch.zeros(1, dtype=torch.int32, device=dev())
    s, t, u, v = learn.glv_pair_forward(_t(Q), _t(X), _t(tags), _t(A), _t(B), _t(qi), _t(xi), d_status=st)
    assert st.item() == 0
    # forward against the oracle's reduced rows and projections
    Xr = oracle.build_reduced(X, tags, B)
    Qp = oracle.project(Q, A)
    s_ref = np.einsum("pr,pr->p", Xr[xi], Qp[qi, tags[xi]])
    t_ref = np.einsum("pk,pk->p", Q[qi].astype(np.float64), X[xi].astype(np.float64))
    scale = np.linalg.norm(Xr[xi], axis=1) * np.linalg.norm(Qp[qi, tags[xi]], axis=1)
    assert np.all(np.abs(s.cpu().numpy() - s_ref) <= 1e-5 * np.maximum(np.abs(s_ref), scale))
    assert np.all(np.abs(t.cpu().numpy() - t_ref) <= 1e-5 * np.linalg.norm(Q[qi], axis=1) * np.linalg.norm(X[xi], axis=1))
    # backward of L = sum (t - s)^2: g = -2 (t - s)
    g = -2.0 * (t - s)
    dA, dB = learn.glv_pair_backward(_t(Q), _t(X), _t(tags), C, _t(qi), _t(xi), u, v, g)
    loss, gA, gB = oracle.pair_loss_grad(Q, X, tags, A, B, qi, xi)
    for got, ref in ((dA.cpu().numpy(), gA), (dB.cpu().numpy(), gB)):
        err = np.abs(got - ref).max()
        assert err <= 1e-4 * np.abs(ref).max(), (err, np.abs(ref).max())


def test_backward_matches_exact_central_differences_of_the_fp64_loss(learn):
    """dL/dA_c and dL/dB_c from the backward kernel (through the autograd function, g from
    glv_pair_loss) against central differences of the FP64 oracle loss.  L is quadratic in
    each entry, so (L(a + h) - L(a - h)) / 2h is its exact derivative; h = 2^-10 keeps a +- h
    exact in FP32 for the |a| < 1 entries used.  Checked entries: where the oracle's gradient
    is at least a tenth of its largest entry; bound 1e-4 relative per entry."""
    D, d, C, P = 64, 16, 3, 2048
    rng, Q, X, mu = _sets(9, D, 200, 1500, C)
    tags_np = oracle.assign_tags(X, mu)
    A_np = (rng.standard_normal((C, d, D)) / np.sqrt(D)).astype(np.float32)
    B_np = (rng.standard_normal((C, d, D)) / np.sqrt(D)).astype(np.float32)
    qi_np = rng.integers(0, 200, P).astype(np.int32)
    xi_np = rng.integers(0, 1500, P).astype(np.int32)
    A = _t(A_np).requires_grad_(True)
    B = _t(B_np).requires_grad_(True)
    loss = learn.pair_loss(A, B, _t(Q), _t(X), _t(tags_np), _t(qi_np), _t(xi_np))
    loss.backward()
    l_ref, gA_ref, gB_ref = oracle.pair_loss_grad(Q, X, tags_np, A_np, B_np, qi_np, xi_np)
    assert abs(loss.item() - l_ref) <= 1e-5 * l_ref
    h = 2.0 ** -10
    pick = np.random.default_rng(4)
    for which, M_np, G, ref in (("A", A_np, A.grad.cpu().numpy(), gA_ref), ("B", B_np, B.grad.cpu().numpy(), gB_ref)):
        big = np.argwhere(np.abs(ref) >= 0.1 * np.abs(ref).max())
        for c, r, k in big[pick.choice(len(big), 6, replace=False)]:
            Mp, Mm = M_np.copy(), M_np.copy()
            Mp[c, r, k] += np.float32(h)
            Mm[c, r, k] -= np.float32(h)
            assert float(Mp[c, r, k]) - float(M_np[c, r, k]) == h and float(M_np[c, r, k]) - float(Mm[c, r, k]) == h
            if which == "A":
                lp = oracle.pair_loss_grad(Q, X, tags_np, Mp, B_np, qi_np, xi_np, want_grad=False)
                lm = oracle.pair_loss_grad(Q, X, tags_np, Mm, B_np, qi_np, xi_np, want_grad=False)
            else:
                lp = oracle.pair_loss_grad(Q, X, tags_np, A_np, Mp, qi_np, xi_np, want_grad=False)
                lm = oracle.pair_loss_grad(Q, X, tags_np, A_np, Mm, qi_np, xi_np, want_grad=False)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - G[c, r, k]) <= 1e-4 * abs(fd), (which, c, r, k, fd, G[c, r, k])


def test_pair_loss_weight_scales_the_gradient(learn):
    """The upstream weight multiplies g on the device: the backward of 4 L is 4 times the
    backward of L (a power of two scales every rounded term exactly; the pairs of a cluster are
    summed in the order the device grouping left them, which may differ between the calls, so
    the sums agree to FP32 summation error)."""
    D, d, C, P = 32, 8, 2, 700
    rng, Q, X, mu = _sets(19, D, 100, 900, C)
    tags = _t(oracle.assign_tags(X, mu))
    A = _t((rng.standard_normal((C, d, D)) / np.sqrt(D)).astype(np.float32))
    B = _t((rng.standard_normal((C, d, D)) / np.sqrt(D)).astype(np.float32))
    qi = _t(rng.integers(0, 100, P).astype(np.int32))
    xi = _t(rng.integers(0, 900, P).astype(np.int32))
    grads = []
    for wgt in (1.0, 4.0):
        A1, B1 = A.clone().requires_grad_(True), B.clone().requires_grad_(True)
        (wgt * learn.pair_loss(A1, B1, _t(Q), _t(X), tags, qi, xi)).backward()
        grads.append((A1.grad.clone(), B1.grad.clone()))
    for g1, g4 in zip(grads[0], grads[1]):
        torch.testing.assert_close(g4, 4.0 * g1, rtol=0, atol=1e-5 * float((4.0 * g1).abs().max()))


def test_adam_step_matches_the_textbook_update(learn):
    """glv_adam_step against torch.optim.Adam (the same published update) over 5 steps."""
    rng = np.random.default_rng(2)
    p0 = rng.standard_normal(10_000).astype(np.float32)
    grads = [rng.standard_normal(10_000).astype(np.float32) for _ in range(5)]
    p = _t(p0.copy())
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    ref = _t(p0.copy()).requires_grad_(True)
    opt = torch.optim.Adam([ref], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for step, g in enumerate(grads, start=1):
        learn.glv_adam_step(p, _t(g), m, v, step, 1e-2)
        ref.grad = _t(g)
        opt.step()
    torch.testing.assert_close(p, ref.detach(), rtol=1e-5, atol=1e-6)


def _all_pairs(nq, nx):
    qi, xi = np.meshgrid(np.arange(nq, dtype=np.int32), np.arange(nx, dtype=np.int32), indexing="ij")
    return torch.from_numpy(qi.ravel()).to(dev()), torch.from_numpy(xi.ravel()).to(dev())


def test_sphering_is_stationary_for_the_full_data_loss(learn):
    """With K_Q and K_X taken from the very pairs of the loss, Sphering minimises it (rank-d
    Eckart-Young truncation of W K_X^(1/2)): the full-data gradient through the backward
    kernel vanishes there, unlike at a perturbed point."""
    D, d, C = 48, 10, 3
    rng, Q, X, mu = _sets(21, D, 150, 2000, C)
    tags = _t(oracle.assign_tags(X, mu))
    Qt, Xt = _t(Q), _t(X)
    A0, B0 = learn.sphering_init(Qt, Xt, tags, C, d)
    qi, xi = _all_pairs(150, 2000)

    def grad_norm(A, B):
        A = A.clone().requires_grad_(True)
        B = B.clone().requires_grad_(True)
        learn.pair_loss(A, B, Qt, Xt, tags, qi, xi).backward()
        return float(torch.cat([A.grad.ravel(), B.grad.ravel()]).norm())

    g_opt = grad_norm(A0, B0)
    g_off = grad_norm(A0 + 0.05 * torch.randn_like(A0), B0 + 0.05 * torch.randn_like(B0))
    assert g_opt < 1e-2 * g_off, (g_opt, g_off)


def test_refine_moves_towards_the_sphering_optimum(learn):
    """From random row-orthonormal A_c = B_c, refinement over random pairs lowers the loss
    substantially, and does not go below the closed-form Sphering optimum (up to noise)."""
    D, d, C = 64, 8, 4
    rng, Q, X, mu = _sets(13, D, 2000, 8000, C)
    tags = _t(oracle.assign_tags(X, mu))
    Qt, Xt = _t(Q), _t(X)
    P = np.stack([np.linalg.qr(rng.standard_normal((D, d)))[0].T for _ in range(C)]).astype(np.float32)
    A0 = B0 = _t(P)
    As, Bs = learn.sphering_init(Qt, Xt, tags, C, d)
    qi, xi = (torch.from_numpy(rng.integers(0, n, 50000).astype(np.int32)).to(dev()) for n in (2000, 8000))
    with torch.no_grad():
        l0 = learn.pair_loss(A0, B0, Qt, Xt, tags, qi, xi).item()
        l_opt = learn.pair_loss(As, Bs, Qt, Xt, tags, qi, xi).item()
    A1, B1, hist = learn.refine(A0, B0, Qt, Xt, tags, steps=400, batch=4096, lr=3e-3, seed=3)
    with torch.no_grad():
        l1 = learn.pair_loss(A1, B1, Qt, Xt, tags, qi, xi).item()
    assert np.isfinite(hist).all()
    assert l1 < 0.8 * l0, (l0, l1, l_opt)
    assert l1 > 0.97 * l_opt, (l0, l1, l_opt)


# ---------------------------------------------------------------------------------------
# spherical k-means (Appendix A)
# ---------------------------------------------------------------------------------------

def test_kmeans_update_vs_oracle(learn):
    from paper_2410_22347_gb300 import glv
    rng, Q, X, mu = _sets(31, 96, 10, 20000, 9)
    X = X / np.linalg.norm(X, axis=1, keepdims=True)
    tags = oracle.assign_tags(X, mu)
    tags[tags == 4] = 3                      # cluster 4 empty: keeps its landmark
    ref, counts = oracle.kmeans_update(X, tags, mu)
    mu_t = _t(mu.astype(np.float32))
    got, gc = glv.glv_kmeans_update(_t(X.astype(np.float32)), _t(tags), mu_t)
    np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=0, atol=2e-7)
    np.testing.assert_array_equal(gc.cpu().numpy(), counts)
    np.testing.assert_array_equal(got.cpu().numpy()[4], mu[4])


def test_best_inner_product_output(learn):
    from paper_2410_22347_gb300 import glv
    rng, Q, X, mu = _sets(32, 64, 10, 5000, 12)
    best = torch.empty(5000, dtype=torch.float32, device=dev())
    tags = glv.glv_assign_tags(_t(X), _t(mu), best_ip=best).cpu().numpy()
    ip = X.astype(np.float64) @ mu.astype(np.float64).T
    np.testing.assert_allclose(best.cpu().numpy(), ip[np.arange(5000), tags], rtol=0,
                               atol=1e-5 * np.abs(ip).max())
    assert np.all(ip.max(axis=1) - ip[np.arange(5000), tags] <= 1e-5 * np.abs(ip).max())


def test_spherical_kmeans_gpu_em_matches_oracle_em(learn):
    """Same seeds: three GPU EM iterations reproduce the oracle's EM (tags agree away from
    near-ties, landmarks to FP32 accuracy) and the objective does not decrease."""
    from paper_2410_22347_gb300 import glv, kmeans
    from paper_2410_22347_gb300 import synth
    w = synth.make_workload(N=30000, D=64, d=8, C=6, nq=1, K_db=12, cands=1, kappa=0, k=1, cfg=87)
    X = w.X.numpy()
    mu0 = X[np.random.default_rng(0).choice(len(X), 6, replace=False)].copy()
    mu_ref = mu0.copy()
    mu_gpu = _t(mu0)
    Xt = _t(X)
    for _ in range(3):
        tags_ref, margin = oracle.assign_tags(X, mu_ref, return_margin=True)
        tags_gpu = glv.glv_assign_tags(Xt, mu_gpu).cpu().numpy()
        sure = margin > 1e-5
        np.testing.assert_array_equal(tags_gpu[sure], tags_ref[sure])
        m64, _ = oracle.kmeans_update(X, tags_ref, mu_ref)
        mu_ref = m64.astype(np.float32)
        glv.glv_kmeans_update(Xt, _t(tags_ref), mu_gpu)   # same assignment on both sides
        np.testing.assert_allclose(mu_gpu.cpu().numpy(), m64, atol=2e-7)
    mu, hist = kmeans.spherical_kmeans(Xt, 6, iters=8, sample=0, seed=1)
    assert all(b >= a - 1e-3 * abs(a) for a, b in zip(hist, hist[1:]))
    np.testing.assert_allclose(np.linalg.norm(mu.cpu().numpy(), axis=1), 1.0, atol=1e-5)
