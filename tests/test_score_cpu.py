"""The bench's factor-match score (Sec. 4.2 metric, matched by a linear
assignment) against the oracle's brute-force score over every permutation,
on the CPU.

Both read the score the same way: unit columns, per pair
(1 - |lambda - mu| / max) times the product of absolute cosines, averaged over
the best one-to-one matching. The assignment solver must find the same
optimum as trying every permutation. The cases are random models, a model
against a permuted, sign-flipped, rescaled and slightly perturbed copy of
itself, and models with a zero weight or a zero column.
"""
import numpy as np
import pytest

import oracle
from paper_2112_10855_gb300.score import factor_match_score


def model(rng, dims, R):
    return rng.uniform(0.1, 3.0, R), [rng.standard_normal((d, R)) for d in dims]


@pytest.mark.parametrize("dims,R", [((5, 4), 1), ((6, 5, 4), 3), ((7, 6, 5), 5), ((4, 5, 3, 4), 6),
                                    ((8, 7, 6), 7)])
def test_assignment_equals_brute_force_on_random_models(dims, R):
    rng = np.random.default_rng(R * 31 + len(dims))
    for _ in range(5):
        l1, A1 = model(rng, dims, R)
        l2, A2 = model(rng, dims, R)
        s = factor_match_score(l1, A1, l2, A2)
        assert abs(s - oracle.score(dims, l1, A1, l2, A2)) < 1e-12
        assert 0.0 <= s <= 1.0


@pytest.mark.parametrize("R", [2, 4, 7])
def test_assignment_equals_brute_force_on_near_copies(R):
    rng = np.random.default_rng(100 + R)
    dims = (9, 8, 7)
    l1, A1 = model(rng, dims, R)
    perm = rng.permutation(R)
    signs = np.where(rng.random(R) < 0.5, -1.0, 1.0)
    A2 = [a[:, perm] * signs[None, :] * 1.7 + 1e-3 * rng.standard_normal(a.shape) for a in A1]
    l2 = l1[perm] * (1 + 1e-3 * rng.standard_normal(R))
    s = factor_match_score(l1, A1, l2, A2)
    assert abs(s - oracle.score(dims, l1, A1, l2, A2)) < 1e-12
    assert s > 0.98
    # the exact copy scores 1
    A3 = [a[:, perm] * signs[None, :] * 1.7 for a in A1]
    assert abs(factor_match_score(l1, A1, l1[perm], A3) - 1.0) < 1e-14


def test_zero_weight_and_zero_column():
    rng = np.random.default_rng(7)
    dims, R = (6, 5, 4), 3
    l1, A1 = model(rng, dims, R)
    l2, A2 = model(rng, dims, R)
    l1[0] = 0.0
    l2[0] = 0.0
    A2[1][:, 2] = 0.0
    s = factor_match_score(l1, A1, l2, A2)
    assert abs(s - oracle.score(dims, l1, A1, l2, A2)) < 1e-12
