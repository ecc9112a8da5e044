"""Host checks of the seeded synthetic inputs (no GPU): the generators hold none of the
method's arithmetic, but every test and benchmark input comes from them, so their stated
properties are checked here -- unit rows, orthonormal projections, well-formed CSR candidate
lists with distinct ids per list, lognormal lengths with the requested arithmetic mean and
clipping, and reproducibility from the seed."""
import math

import numpy as np
import pytest
import torch

from paper_2410_22347_gb300 import synth


def _g(seed):
    g = torch.Generator()
    g.manual_seed(seed)
    return g


def test_row_orthonormal_and_haar():
    P = synth.row_orthonormal(24, 96, 3, _g(1), "cpu").double()
    for c in range(3):
        np.testing.assert_allclose((P[c] @ P[c].T).numpy(), np.eye(24), atol=1e-5)
    R = synth.haar_orthogonal(16, 2, _g(2), "cpu").double()
    np.testing.assert_allclose((R[0] @ R[0].T).numpy(), np.eye(16), atol=1e-5)


def test_mixture_rows_are_unit_vectors():
    means = torch.randn(4, 32, generator=_g(3))
    X = synth.mixture(500, 32, means, 1.0, _g(4), "cpu", chunk=128)
    np.testing.assert_allclose(X.double().norm(dim=1).numpy(), 1.0, atol=1e-5)


def test_candidate_lists_are_well_formed():
    lengths = torch.tensor([0, 1, 50, 300, 500, 7])
    off, ids = synth.candidate_lists(6, 1000, lengths, _g(5), "cpu")
    assert off.dtype == torch.int64 and ids.dtype == torch.int32
    np.testing.assert_array_equal(off.numpy(), np.concatenate([[0], np.cumsum(lengths.numpy())]))
    o, i = off.numpy(), ids.numpy()
    assert i.min() >= 0 and i.max() < 1000
    for q in range(6):
        lst = i[o[q]:o[q + 1]]
        assert len(np.unique(lst)) == len(lst)  # distinct within a list
    with pytest.raises(ValueError):
        synth.candidate_lists(1, 10, torch.tensor([11]), _g(6), "cpu")


def _clipped_lognormal_mean(mean, sigma, lo, hi):
    """E[clip(X, lo, hi)] for ln X ~ N(mu, sigma^2), mu = ln mean - sigma^2 / 2, in closed form:
    lo P(X < lo) + hi P(X > hi) + e^(mu + sigma^2/2) [Phi(b - sigma) - Phi(a - sigma)] with
    a, b the standardised ln lo, ln hi."""
    mu = math.log(mean) - 0.5 * sigma * sigma
    Phi = lambda z: 0.5 * (1.0 + math.erf(z / math.sqrt(2.0)))
    a, b = (math.log(lo) - mu) / sigma, (math.log(hi) - mu) / sigma
    return lo * Phi(a) + hi * (1.0 - Phi(b)) + mean * (Phi(b - sigma) - Phi(a - sigma))


def test_lognormal_lengths_mean_and_clipping():
    L = synth.lognormal_lengths(2000000, 2000.0, 1.2, 64, 32768, _g(7), "cpu").double()
    assert L.min() >= 64 and L.max() <= 32768
    # the clipped heavy tail pulls the mean below the requested 2000: compare with the closed
    # form of the clipped lognormal's mean (rounding to integers changes it by < 0.5; the
    # standard error of the sample mean is about 0.15% here)
    want = _clipped_lognormal_mean(2000.0, 1.2, 64, 32768)
    assert abs(L.mean().item() / want - 1.0) < 0.006
    U = synth.lognormal_lengths(200000, 500.0, 0.5, 1, 10 ** 9, _g(8), "cpu").double()
    assert abs(U.mean().item() / 500.0 - 1.0) < 0.01
    assert abs(torch.log(U).std().item() - 0.5) < 0.01


def test_workloads_are_reproducible_from_their_seed():
    a = synth.make_workload(N=400, D=32, d=8, C=3, nq=5, K_db=4, cands=20, kappa=10, k=5, cfg=91)
    b = synth.make_workload(N=400, D=32, d=8, C=3, nq=5, K_db=4, cands=20, kappa=10, k=5, cfg=91)
    c = synth.make_workload(N=400, D=32, d=8, C=3, nq=5, K_db=4, cands=20, kappa=10, k=5, cfg=92)
    for t in ("X", "Q", "A", "B", "mu", "off", "ids"):
        assert torch.equal(getattr(a, t), getattr(b, t)), t
    assert not torch.equal(a.X, c.X)
    assert a.off[-1].item() == 5 * 20 and math.isclose(a.X.double().norm(dim=1).mean().item(), 1.0, rel_tol=1e-5)
