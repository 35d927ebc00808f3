"""The fused mode tail (one thread-block cluster: solve, normalisation,
Gram and CholeskyQR2 of the factor) against the separate kernels and the
FP64 oracle.

- Every solve kind at ranks 1..64 (rank 33 and 64 take the GPU-wide solve
  before the cluster): A_n and lambda within 1e-12 of the unfused path and
  1e-10 of the oracle; Q_n, R_n within 1e-12 of the unfused Householder QR
  (the thin QR with a positive diagonal is unique); Q_n orthonormal.
- An ill-conditioned factor (two columns 1e-9 apart): CholeskyQR2 is refused
  and the Householder QR takes over, so Q_n stays orthonormal to FP64
  rounding and A_n = Q_n R_n.
- Sweeps: fits per sweep within 1e-12 of the unfused path.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2112_10855_gb300 import cpals

pytestmark = pytest.mark.gpu

OSOLVE = {"qr": oracle.QR, "svd": oracle.SVD, "normal": oracle.NORMAL, "normal_pinv": oracle.NORMAL_PINV}


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def handles(dims, R, X, A, fused_first=True):
    out = []
    for fused in (True, False):
        h = cpals.CPALS(dims, R, "f64")
        h.set_fused_tail(fused)
        h.set_tensor(torch.from_numpy(X).cuda())
        h.set_factors(A)
        out.append(h)
    return out


CASES = [((50, 33, 41), 1), ((50, 33, 41), 4), ((50, 33, 41), 10), ((37, 29, 41), 20),
         ((12, 11, 10, 13), 3), ((70, 65, 66), 33), ((70, 65, 66), 64), ((400, 37, 9), 9)]


@pytest.mark.parametrize("solve", ["qr", "svd", "normal", "normal_pinv"])
@pytest.mark.parametrize("dims,R", CASES)
def test_fused_tail_matches_unfused_and_oracle(cuda_lib, dims, R, solve):
    rng = np.random.default_rng(sum(dims) * 7 + R)
    X = rng.standard_normal(int(np.prod(dims)))
    A = [np.asfortranarray(rng.standard_normal((d, R))) for d in dims]
    hf, hu = handles(dims, R, X, A)
    o = oracle.OracleCPALS(X, dims, R)
    o.set_factors(A)
    for n in range(len(dims)):
        for h in (hf, hu):
            h.solve_mode(n, solve, 1e-10)
            h.sync()
        o.update_mode(n, OSOLVE[solve], 1e-10)
        Af, lf = hf.get_factors()
        Au, lu = hu.get_factors()
        assert rel(Af[n], Au[n]) <= 1e-12 and rel(lf, lu) <= 1e-12, (n, rel(Af[n], Au[n]), rel(lf, lu))
        assert rel(Af[n], o.factor(n)) <= 1e-10 and rel(lf, o.lam()) <= 1e-10
        if solve in ("qr", "svd"):
            Qf, Rf = hf.get_factor_qr(n)
            Qu, Ru = hu.get_factor_qr(n)
            assert rel(Qf, Qu) <= 1e-12 and rel(Rf, Ru) <= 1e-12, (n, rel(Qf, Qu), rel(Rf, Ru))
            assert np.abs(Qf.T @ Qf - np.eye(R)).max() <= 1e-13
            assert np.all(np.diag(Rf) > 0) and np.allclose(np.tril(Rf, -1), 0.0)


def test_ill_conditioned_factor_falls_back_to_householder(cuda_lib):
    # mode 0's least-squares solution is the planted factor, whose columns 0
    # and 1 are 1e-9 apart: cond(A_0) ~ 1e9, beyond what CholeskyQR2 accepts
    dims, R = (60, 50, 40), 4
    rng = np.random.default_rng(5)
    F = [np.linalg.qr(rng.standard_normal((d, R)))[0] for d in dims]
    F[0][:, 1] = F[0][:, 0] + 1e-9 * rng.standard_normal(dims[0])
    F = [np.asfortranarray(f) for f in F]
    from paper_2112_10855_gb300 import inputs
    X = inputs.cp_full(dims, F, np.ones(R))
    hf, hu = handles(dims, R, X, F)
    for h in (hf, hu):
        h.solve_mode(0, "qr")
        h.sync()
    Af, lf = hf.get_factors()
    Qf, Rf = hf.get_factor_qr(0)
    Qu, Ru = hu.get_factor_qr(0)
    assert np.abs(Qf.T @ Qf - np.eye(R)).max() <= 1e-13          # Householder's orthogonality
    assert rel(Qf @ Rf, Af[0]) <= 1e-14
    assert np.all(np.diag(Rf) >= 0)
    # the same Householder QR on (up to rounding) the same A_0: column 0 of Q
    # and R agree closely (the later columns of Q carry the 1e-9 difference of
    # columns 0 and 1, amplified to ~1e-7)
    assert rel(Qf[:, 0], Qu[:, 0]) <= 1e-12 and rel(Rf, Ru) <= 1e-6


@pytest.mark.parametrize("solve", ["qr", "svd", "normal"])
@pytest.mark.parametrize("dims,R", [((40, 36, 32), 8), ((24, 22, 20, 18), 5), ((60, 58, 56), 20)])
def test_fused_tail_sweeps_match_unfused(cuda_lib, dims, R, solve):
    rng = np.random.default_rng(R + len(dims))
    X = rng.standard_normal(int(np.prod(dims)))
    A = [np.asfortranarray(rng.standard_normal((d, R))) for d in dims]
    hf, hu = handles(dims, R, X, A)
    ff = np.asarray(hf.iterate(5, solve=solve, svd_rtol=1e-10))
    fu = np.asarray(hu.iterate(5, solve=solve, svd_rtol=1e-10))
    assert np.abs(ff - fu).max() <= 1e-12, (ff, fu)


def test_newton_reciprocals_within_two_ulp(cuda_lib):
    # the fused tail's 1/x and 1/sqrt(x) (hardware seed + one third-order FP64
    # Newton step, resp. two Newton-Raphson steps) against the correctly
    # rounded FP64 results, over 40 decades
    rng = np.random.default_rng(3)
    x = np.concatenate([10.0 ** rng.uniform(-40, 40, 200000), rng.uniform(0.5, 2.0, 100000),
                        [1.0, 2.0, 0.5, 3.0, 1e-36, 1e36, 1.5e-36, 7e35]])
    xd = torch.from_numpy(x).cuda()
    rcp, rsq = cpals.test_newton_recip(xd)
    rcp, rsq = rcp.cpu().numpy(), rsq.cpu().numpy()
    ref_r = 1.0 / x
    ref_s = 1.0 / np.sqrt(x)
    ulp_r = np.abs(rcp - ref_r) / np.spacing(ref_r)
    ulp_s = np.abs(rsq - ref_s) / np.spacing(ref_s)
    assert ulp_r.max() <= 2.0, ulp_r.max()
    assert ulp_s.max() <= 2.0, ulp_s.max()
    neg = torch.tensor([-2.0, -1e-10, -1e20], dtype=torch.float64, device="cuda")
    r, _ = cpals.test_newton_recip(neg)
    np.testing.assert_allclose(r.cpu().numpy(), 1.0 / neg.cpu().numpy(), rtol=5e-16)


@pytest.mark.parametrize("solve", ["qr", "svd", "normal"])
def test_profiled_sweeps_match_graph_sweeps(cuda_lib, solve):
    # cpals_profile_sweeps runs the same sweeps eagerly on one stream: the
    # factors it leaves equal those of cpals_iterate bit for bit, and every
    # bucket it reports is a non-negative time
    dims, R = (40, 36, 32), 6
    rng = np.random.default_rng(12)
    X = rng.standard_normal(int(np.prod(dims)))
    A = [np.asfortranarray(rng.standard_normal((d, R))) for d in dims]
    h1, _ = handles(dims, R, X, A)
    h2, _ = handles(dims, R, X, A)
    h1.iterate(2, solve=solve, svd_rtol=1e-10)
    b = h2.profile_sweeps(2, solve=solve, svd_rtol=1e-10)
    assert set(b) == {"multi_ttm_or_mttkrp", "factor_qr_or_gram", "compute_q0", "apply_q0", "other"}
    assert all(v >= 0.0 for v in b.values()) and b["multi_ttm_or_mttkrp"] > 0.0
    if solve != "normal":
        assert b["compute_q0"] > 0.0 and b["apply_q0"] > 0.0
    for a1, a2 in zip(h1.get_factors()[0], h2.get_factors()[0]):
        np.testing.assert_array_equal(a1, a2)
