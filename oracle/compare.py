"""Comparison rules between a GPU result and the oracle's (test infrastructure only).

Where several results are correct -- the order of near-equal scores, which of two nearly
tied candidates fills the last slot -- these helpers compare what is unique and check that
the rest is valid, using only oracle-computed scores:

* ``scores_close``: |s_gpu - s_ref| <= tol * max(|s_ref|, scale), where ``scale`` is the
  Cauchy-Schwarz bound of the dot product (||q_c|| ||x_i||), so near-zero scores are judged
  on the magnitude of the vectors that formed them;
* ``topk_equivalent``: the id lists are equal, or every id in their symmetric difference has
  an oracle score within ``window`` of the oracle's last kept score, and any reordering is
  between entries whose oracle scores are within ``window`` of each other;
* ``search_equivalent``: as above for the final top k of a multi-step search, where an id may
  also differ because the reduced-space top-kappa boundary was a near tie.
"""
from __future__ import annotations

import math

import numpy as np


def scores_close(got, ref, scale, tol=1e-5):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.broadcast_to(np.asarray(scale, np.float64), ref.shape)
    both_inf = np.isinf(got) & np.isinf(ref) & (np.sign(got) == np.sign(ref))
    with np.errstate(invalid="ignore"):  # inf - inf where both are the same infinity
        err = np.where(both_inf, 0.0, np.abs(got - ref))
    lim = tol * np.maximum(np.abs(np.where(np.isinf(ref), 0.0, ref)), scale)
    bad = ~(err <= lim)
    return not bad.any(), (np.nanmax(err / np.maximum(lim / tol, 1e-300)) if err.size else 0.0), np.flatnonzero(bad)


def topk_equivalent(got_ids, ref_ids, ref_scores, score_of, window=1e-6):
    """One query.  ``ref_scores``: the oracle's scores for ``ref_ids`` (sorted, padded with
    -inf / id -1).  ``score_of(id)``: the oracle's score of any id the GPU returned."""
    got = [int(i) for i in got_ids]
    ref = [int(i) for i in ref_ids]
    if got == ref:
        return True, ""
    valid = [s for s, i in zip(ref_scores, ref) if i >= 0]
    kth = valid[-1] if valid else -math.inf
    gs, rs = set(got) - {-1}, set(ref) - {-1}
    if len([i for i in got if i >= 0]) != len([i for i in ref if i >= 0]):
        return False, f"different counts {got} vs {ref}"
    for i in gs ^ rs:
        if abs(score_of(i) - kth) > window:
            return False, f"id {i} (score {score_of(i)!r}) vs k-th {kth!r}"
    # order: each position's oracle score must match the reference score at that position
    for t, (g, r) in enumerate(zip(got, ref)):
        if g == r or g < 0 or r < 0:
            continue
        if abs(score_of(g) - ref_scores[t]) > window:
            return False, f"position {t}: {g} ({score_of(g)!r}) vs {r} ({ref_scores[t]!r})"
    return True, ""


def search_equivalent(got_ids, ref_ids, ref_scores, exact_of, reduced_of, reduced_kappa_th,
                      window=1e-6, reduced_window=1e-6):
    """Final top-k of a multi-step search.  An id present on one side only is accepted when
    its exact score ties the k-th within ``window``, or when its reduced score ties the
    kappa-th reduced score within ``reduced_window`` (the survivor sets may then differ)."""
    got = [int(i) for i in got_ids]
    ref = [int(i) for i in ref_ids]
    if got == ref:
        return True, ""
    valid = [s for s, i in zip(ref_scores, ref) if i >= 0]
    kth = valid[-1] if valid else -math.inf
    for i in (set(got) ^ set(ref)) - {-1}:
        if abs(exact_of(i) - kth) <= window:
            continue
        if abs(reduced_of(i) - reduced_kappa_th) <= reduced_window:
            continue
        return False, f"id {i}: exact {exact_of(i)!r} vs k-th {kth!r}, reduced {reduced_of(i)!r} vs kappa-th {reduced_kappa_th!r}"
    for t, (g, r) in enumerate(zip(got, ref)):
        if g == r or g < 0 or r < 0:
            continue
        if abs(exact_of(g) - ref_scores[t]) > window and g in ref:
            return False, f"position {t}: {g} vs {r}"
    return True, ""
