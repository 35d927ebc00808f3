"""Factor-match score between two CP models (Sec. 4.2).

The paper uses the score to check whether a computed CP model recovers the
planted one, but gives no formula.  The reading used here: with unit columns,
a pair (r of model 1, p of model 2) scores

    (1 - |lambda_r - mu_p| / max(lambda_r, mu_p)) * prod_n |cos(a_r^(n), b_p^(n))|,

and the score is the mean over r of the best one-to-one matching, found as a
linear assignment (the Hungarian method, scipy) instead of trying every
permutation.  Signs are absorbed by the absolute cosines.  A score of 1 means
the two models are equal up to permutation and column signs.
"""
from __future__ import annotations

import numpy as np


def pair_scores(lam1, A1, lam2, A2) -> np.ndarray:
    """R1 x R2 matrix of the per-pair scores."""
    lam1 = np.asarray(lam1, dtype=np.float64)
    lam2 = np.asarray(lam2, dtype=np.float64)
    lm = np.maximum(lam1[:, None], lam2[None, :])
    with np.errstate(invalid="ignore", divide="ignore"):
        w = np.where(lm > 0, 1.0 - np.abs(lam1[:, None] - lam2[None, :]) / lm, 1.0)
    S = w.copy()
    for a, b in zip(A1, A2):
        a = np.asarray(a, dtype=np.float64)
        b = np.asarray(b, dtype=np.float64)
        na = np.linalg.norm(a, axis=0)
        nb = np.linalg.norm(b, axis=0)
        with np.errstate(invalid="ignore", divide="ignore"):
            cos = np.abs(a.T @ b) / np.outer(na, nb)
        S *= np.where(np.isfinite(cos), cos, 0.0)
    return S


def factor_match_score(lam1, A1, lam2, A2) -> float:
    """Mean pair score of the best matching of the components of model 1 to model 2."""
    from scipy.optimize import linear_sum_assignment
    S = pair_scores(lam1, A1, lam2, A2)
    rows, cols = linear_sum_assignment(S, maximize=True)
    return float(S[rows, cols].sum() / S.shape[0])
