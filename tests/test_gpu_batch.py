"""Batched path (cpals_batch_*): many independent 3-way problems of uneven
dims and ranks; per sweep two passes over all tensors (dimension tree) and
one kernel per mode update.  Checked against the FP64 oracle run on each
problem separately, from the same initial factors.

The factor QRs run CholeskyQR2 with its acceptance check and fall back to
Householder (an ill-conditioned factor checks that path).

Bars: the Multi-TTM and W = Y_(n) Q0 run in FP32 (relative error
~sqrt(I) * 2^-24 per contraction), everything else in FP64.  After one sweep the factors agree with
the oracle to 1e-4 relative (FP32 error amplified by the solve's
conditioning).  At convergence (150 sweeps) the direct fit of the factors the
batch found (FP64 residual against the tensor) agrees with the oracle's to
1e-6 relative.  The batch's own efficient fit is computed from FP32 data.
At fit 0.99 the residual identity of Sec. 3.3.1 cancels ~1e-4 of ||X||^2,
so that value carries ~5e-6 absolute error and is checked to 2e-5 only.
Before convergence the ALS trajectory is sensitive to rounding, so a
mid-trajectory fit is not compared.
"""
import numpy as np
import pytest

import oracle
from paper_2112_10855_gb300 import cpals, inputs

pytestmark = pytest.mark.gpu


def problems(count, seed=77, lo=16, hi=40, rlo=2, rhi=8):
    dims, ranks = inputs.batch_shapes(count, seed=seed, lo=lo, hi=hi, rlo=rlo, rhi=rhi)
    out = []
    for p in range(count):
        pr = inputs.planted(tuple(dims[p]), int(ranks[p]), seed=seed + p, init_seed=seed + 1000 + p, noise=0.01)
        out.append(pr)
    return out


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def small_batch():
    return problems(9)


def make_batch(probs):
    b = cpals.CPALSBatch([p.dims for p in probs], [p.rank for p in probs])
    b.set_tensors([p.X.astype(np.float32) for p in probs])
    b.set_factors([p.init_factors for p in probs])
    return b


def test_batch_one_sweep_matches_oracle(cuda_lib, small_batch):
    b = make_batch(small_batch)
    fits, st = b.iterate(1)
    assert (st == 0).all()
    A, lam = b.get_factors()
    for p, pr in enumerate(small_batch):
        o = oracle.OracleCPALS(pr.X.astype(np.float32).astype(np.float64), pr.dims, pr.rank)
        o.set_factors(pr.init_factors)
        o.iterate(1, solve=oracle.QR)
        for m in range(3):
            assert rel(A[p][m], o.factor(m)) <= 1e-4, (p, m, rel(A[p][m], o.factor(m)))
        assert rel(lam[p], o.lam()) <= 1e-4
        assert abs(fits[p] - o.fit_last()) <= 1e-5


def test_batch_ill_conditioned_factor_takes_householder(cuda_lib, small_batch):
    # a problem whose mode-0 factor has two columns 1e-9 apart, started from
    # the true factors: after mode 0's update cond(A_0) ~ 1e9, past what the
    # factorisation kernel's CholeskyQR2 accepts, so its Householder QR runs.
    # A wrongly accepted CholeskyQR2 would leave Q_0 far from orthonormal and
    # the next modes' updates far from the oracle's.
    dims, R = (40, 36, 32), 4
    rng = np.random.default_rng(11)
    F = [np.linalg.qr(rng.standard_normal((d, R)))[0] for d in dims]
    F[0][:, 1] = F[0][:, 0] + 1e-9 * rng.standard_normal(dims[0])
    F = [np.asfortranarray(f) for f in F]
    X = inputs.cp_full(dims, F, np.ones(R))
    probs = list(small_batch[:2])
    b = cpals.CPALSBatch([p.dims for p in probs] + [dims], [p.rank for p in probs] + [R])
    b.set_tensors([p.X.astype(np.float32) for p in probs] + [X.astype(np.float32)])
    b.set_factors([p.init_factors for p in probs] + [F])
    fits, st = b.iterate(1)
    assert (st == 0).all()
    A, lam = b.get_factors()
    o = oracle.OracleCPALS(X.astype(np.float32).astype(np.float64), dims, R)
    o.set_factors(F)
    o.iterate(1, solve=oracle.QR)
    # (no fit check: at fit ~1 on a noise-free tensor the efficient fit's
    # residual identity cancels to the FP32 rounding level, ~3e-4)
    for m in range(3):
        assert rel(A[2][m], o.factor(m)) <= 1e-4, (m, rel(A[2][m], o.factor(m)))


def test_batch_converged_fits_match_oracle(cuda_lib, small_batch):
    b = make_batch(small_batch)
    fits, st = b.iterate(150)
    assert (st == 0).all()
    A, lam = b.get_factors()
    for p, pr in enumerate(small_batch):
        X = pr.X.astype(np.float32).astype(np.float64)
        o = oracle.OracleCPALS(X, pr.dims, pr.rank)
        o.set_factors(pr.init_factors)
        _, f = o.iterate(150, solve=oracle.QR)
        fit_b = 1.0 - oracle.residual_direct(X, pr.dims, lam[p], A[p]) / np.linalg.norm(X)
        fit_o = o.fit_direct()
        assert abs(fit_b - fit_o) <= 1e-6 * abs(fit_o), (p, fit_b, fit_o)
        assert abs(fits[p] - f[-1]) <= 2e-5, (p, fits[p], f[-1])


def test_batch_matches_single_problem_f32_path(cuda_lib, small_batch):
    import torch
    b = make_batch(small_batch)
    b.iterate(2)
    A, lam = b.get_factors()
    for p in (0, 4, 8):
        pr = small_batch[p]
        h = cpals.CPALS(pr.dims, pr.rank, "f32")
        h.set_tensor(torch.from_numpy(pr.X.astype(np.float32)).cuda())
        h.set_factors([np.asfortranarray(a) for a in pr.init_factors])
        h.iterate(2)
        As, ls = h.get_factors()
        for m in range(3):
            assert rel(A[p][m], As[m]) <= 1e-4


def test_batch_singular_problem_is_isolated(cuda_lib):
    probs = problems(4, seed=91)
    bad = probs[2]
    for m in range(3):
        bad.init_factors[m][:, 1] = bad.init_factors[m][:, 0]
    b = make_batch(probs)
    fits, st = b.iterate(1)
    assert st[2] == cpals.ERR_SINGULAR
    assert (np.delete(st, 2) == 0).all()
    A, _ = b.get_factors()
    # the failed problem keeps its factors; the others move
    np.testing.assert_array_equal(A[2][0], np.asfortranarray(bad.init_factors[0]))
    assert rel(A[0][0], probs[0].init_factors[0]) > 1e-3


def test_batch_autotuner_and_graph(cuda_lib, small_batch):
    b = make_batch(small_batch)
    b.iterate(1)
    g, t = b.launch_shape()
    assert g >= 1 and t in (128, 256)
    l0 = b.launch_count()
    b.iterate(3)
    assert b.launch_count() - l0 == 36    # twelve kernels per replayed sweep


def test_batch_rejects_bad_shapes(cuda_lib):
    with pytest.raises(cpals.CPALSError):
        cpals.CPALSBatch([(10, 10, 10)], [17])
    with pytest.raises(cpals.CPALSError):
        cpals.CPALSBatch([(10, 4, 10)], [5])
