"""CPU checks of the product's LeanVec-Sphering factors (Algorithm 2 through a Cholesky
whitening, ``learn.sphering_factors``) against what Section 3.2 fixes, on FP64 moments:
W^T W = K_Q, A B^T = I_d, A^T B = I at d = D, and the loss of the learning pairs equals the
sum of the D - d smallest eigenvalues of K_Q K_X (the spectrum of W K_X W^T, taken here from
the non-symmetric product by another routine) -- plus agreement with the oracle's
symmetric-square-root route up to row signs."""
import numpy as np
import pytest

import oracle
from paper_2410_22347_gb300 import build_lib


@pytest.fixture(scope="module")
def learn():
    build_lib.build()
    from paper_2410_22347_gb300 import learn as L
    return L


def _moments(seed, D, nq=300, nx=2500):
    rng = np.random.default_rng(seed)
    Q = rng.standard_normal((nq, D)) * np.arange(1, D + 1) ** -0.25
    Q = Q @ np.linalg.qr(rng.standard_normal((D, D)))[0].T
    X = rng.standard_normal((nx, D)) * np.arange(1, D + 1) ** -0.6
    X = X @ np.linalg.qr(rng.standard_normal((D, D)))[0].T
    return Q.T @ Q, X.T @ X


def _loss(KQ, KX, A, B):
    """sum over all pairs of (q^T x - (A q)^T (B x))^2 = tr((I - M)^T K_Q (I - M) K_X), M = A^T B."""
    R = np.eye(KQ.shape[0]) - A.T @ B
    return float(np.trace(R.T @ KQ @ R @ KX))


@pytest.mark.parametrize("D,d", [(24, 6), (40, 13), (33, 33)])
def test_sphering_factors_identities(learn, D, d):
    KQ, KX = _moments(D * 7 + d, D)
    A, B, W, lam = learn.sphering_factors(KQ, KX, d)
    assert A.shape == (d, D) and B.shape == (d, D)
    np.testing.assert_allclose(W.T @ W, KQ, rtol=0, atol=1e-12 * np.abs(KQ).max())
    np.testing.assert_allclose(A @ B.T, np.eye(d), rtol=0, atol=1e-10)
    ev = np.sort(np.linalg.eigvals(KQ @ KX).real)
    np.testing.assert_allclose(np.sort(lam), ev, rtol=1e-9, atol=1e-12 * ev.max())
    tail = float(ev[: D - d].sum())
    assert abs(_loss(KQ, KX, A, B) - tail) <= 1e-9 * float(ev.sum())
    if d == D:
        np.testing.assert_allclose(A.T @ B, np.eye(D), rtol=0, atol=1e-9)


def test_sphering_factors_agree_with_the_oracle_up_to_row_signs(learn):
    D, d = 36, 9
    KQ, KX = _moments(5, D)
    A, B, _, _ = learn.sphering_factors(KQ, KX, d)
    Ao, Bo, _, _ = oracle.sphering_from_moments(KQ, KX, d)
    sgn = np.sign(np.sum(A * Ao, axis=1))
    np.testing.assert_allclose(A * sgn[:, None], Ao, rtol=0, atol=1e-9 * np.abs(Ao).max())
    np.testing.assert_allclose(B * sgn[:, None], Bo, rtol=0, atol=1e-9 * np.abs(Bo).max())


def test_sphering_factors_reject_a_singular_query_moment(learn):
    D = 20
    rng = np.random.default_rng(3)
    Q = rng.standard_normal((10, D))          # 10 queries span only 10 of 20 dimensions
    _, KX = _moments(4, D)
    with pytest.raises(ValueError):
        learn.sphering_factors(Q.T @ Q, KX, 5)
