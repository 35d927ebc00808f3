"""The largest order a handle takes (N = 12) against the FP64 oracle.

Ragged dims of 2 and 3 at rank 2, so that every per-mode array of the handle
is used to its full length and V_n has 2^11 rows: three CP-ALS-QR sweeps
(dimension tree, Kronecker fold of V_n) and three CP-ALS sweeps (MTTKRP along
the tree, Cholesky), fits per sweep within 1e-10 and factors within 1e-9 of
the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2112_10855_gb300 import cpals, inputs

pytestmark = pytest.mark.gpu

DIMS = (3, 2, 3, 2, 2, 3, 2, 3, 3, 2, 2, 3)
OSOLVE = {"qr": oracle.QR, "normal": oracle.NORMAL}


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("solve", ["qr", "normal"])
def test_order_twelve_sweeps_match_oracle(cuda_lib, solve):
    R = 2
    p = inputs.planted(DIMS, R, seed=12, init_seed=13, noise=0.02)
    o = oracle.OracleCPALS(p.X, p.dims, R)
    o.set_factors(p.init_factors)
    k, fits_o = o.iterate(3, solve=OSOLVE[solve])
    assert k == 3
    h = cpals.CPALS(p.dims, R, "f64")
    h.set_tensor(torch.from_numpy(np.ascontiguousarray(p.X)).cuda())
    h.set_factors([np.asfortranarray(a) for a in p.init_factors])
    fits = h.iterate(3, solve=solve)
    assert np.abs(np.asarray(fits) - fits_o).max() <= 1e-10
    A, lam = h.get_factors()
    for m in range(len(DIMS)):
        assert rel(A[m], o.factor(m)) <= 1e-9, m
    assert rel(lam, o.lam()) <= 1e-9
