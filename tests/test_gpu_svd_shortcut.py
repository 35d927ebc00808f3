"""The SVD solve's truncation test (CPALS_OPT_SVD_SHORTCUT).

When ||R0||_F ||R0^-1||_F svd_rtol <= 1/4 no singular value of R0 can fall
below the truncation threshold, and the truncated solve W U pinv(Sigma) V^T
equals W R0^-T; the handle then skips the Jacobi SVD.  Checked here:
- well-conditioned problems (ranks 1..64): the update with the shortcut
  agrees with the Jacobi SVD path and with the FP64 oracle's SVD solve;
- an exactly rank-deficient R0 (two equal columns in every factor): the
  bound fails, the Jacobi SVD runs, and the result is the same bit for bit
  as with the shortcut off.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2112_10855_gb300 import cpals

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def pair(dims, R, X, A):
    hs = []
    for on in (True, False):
        h = cpals.CPALS(dims, R, "f64")
        h.set_svd_shortcut(on)
        h.set_tensor(torch.from_numpy(X).cuda())
        h.set_factors(A)
        hs.append(h)
    return hs


@pytest.mark.parametrize("dims,R", [((30, 28, 26), 1), ((37, 29, 41), 5), ((50, 45, 40), 10),
                                    ((45, 44, 43), 33), ((70, 66, 65), 64)])
def test_shortcut_matches_jacobi_and_oracle(cuda_lib, dims, R):
    rng = np.random.default_rng(R * 11 + 1)
    X = rng.standard_normal(int(np.prod(dims)))
    A = [np.asfortranarray(rng.standard_normal((d, R))) for d in dims]
    on, off = pair(dims, R, X, A)
    o = oracle.OracleCPALS(X, dims, R)
    o.set_factors(A)
    for n in range(3):
        for h in (on, off):
            h.solve_mode(n, "svd", 1e-10)
            h.sync()
        o.update_mode(n, oracle.SVD, 1e-10)
        A1, l1 = on.get_factors()
        A2, l2 = off.get_factors()
        assert rel(A1[n] * l1, A2[n] * l2) <= 1e-11, (n, rel(A1[n] * l1, A2[n] * l2))
        assert rel(A1[n] * l1, o.factor(n) * o.lam()) <= 1e-10


def test_rank_deficient_r0_takes_the_jacobi_svd(cuda_lib):
    dims, R = (40, 38, 36), 6
    rng = np.random.default_rng(4)
    X = rng.standard_normal(int(np.prod(dims)))
    A = [np.asfortranarray(rng.standard_normal((d, R))) for d in dims]
    for m in range(3):
        A[m][:, 5] = A[m][:, 4]
    on, off = pair(dims, R, X, A)
    for h in (on, off):
        h.solve_mode(0, "svd", 1e-10)
        h.sync()
    A1, l1 = on.get_factors()
    A2, l2 = off.get_factors()
    np.testing.assert_array_equal(A1[0], A2[0])
    np.testing.assert_array_equal(l1, l2)
