"""The GPU-wide CholeskyQR2 (rank above 32): the factor QRs after the solve
and the Khatri-Rao fold steps of the QR of V_n, run as a chain of kernels over
every SM, against the one-cluster kernel (CPALS_OPT_WIDE_TAIL = 0) and the
FP64 oracle.

- Mode updates with every solve at ranks 33, 40 and 64, on factors of 70 to
  10000 rows: the last spans every row block with several 32-row chunks
  each, and the others have ragged splits. A_n and lambda are within 1e-12 of
  the cluster kernel and 1e-10 of the oracle. Q_n and R_n are within 1e-12 of
  the cluster kernel (the thin QR with a positive diagonal is unique), and
  Q_n is orthonormal to 1e-13.
- A factor set from the A_n that a mode update wrote gets the same Q_n and R_n
  bit for bit (the same row split and summation order), so a resumed run
  repeats the uninterrupted one.
- QR of V_n through wide fold steps (ranks 33..64, three and four modes):
  Q0 and R0 within 1e-12 of the oracle.
- Two columns 1e-9 apart: the check refuses CholeskyQR2 and the Householder
  QR takes over, so Q_n stays orthonormal and A_n = Q_n R_n.
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


def problem(dims, R, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal(int(np.prod(dims)))
    A = [np.asfortranarray(rng.standard_normal((d, R))) for d in dims]
    return X, A


def handle(dims, R, X, A, wide):
    h = cpals.CPALS(dims, R, "f64")
    h.set_wide_tail(wide)
    h.set_tensor(torch.from_numpy(X).cuda())
    h.set_factors(A)
    return h


@pytest.mark.parametrize("solve", ["qr", "svd", "normal", "normal_pinv"])
@pytest.mark.parametrize("dims,R", [((70, 65, 66), 33), ((700, 45, 44), 40), ((300, 70, 66), 64)])
def test_wide_tail_matches_cluster_and_oracle(cuda_lib, dims, R, solve):
    X, A = problem(dims, R, sum(dims) + R)
    hw, hc = handle(dims, R, X, A, True), handle(dims, R, X, A, False)
    o = oracle.OracleCPALS(X, dims, R)
    o.set_factors(A)
    for n in range(len(dims)):
        for h in (hw, hc):
            h.solve_mode(n, solve, 1e-10)
            h.sync()
        o.update_mode(n, OSOLVE[solve], 1e-10)
        Aw, lw = hw.get_factors()
        Ac, lc = hc.get_factors()
        assert rel(Aw[n], Ac[n]) <= 1e-12 and rel(lw, lc) <= 1e-12, (n, rel(Aw[n], Ac[n]), rel(lw, lc))
        assert rel(Aw[n], o.factor(n)) <= 1e-10 and rel(lw, o.lam()) <= 1e-10
        if solve in ("qr", "svd"):
            Qw, Rw = hw.get_factor_qr(n)
            Qc, Rc = hc.get_factor_qr(n)
            assert rel(Qw, Qc) <= 1e-12 and rel(Rw, Rc) <= 1e-12, (n, rel(Qw, Qc), rel(Rw, Rc))
            assert np.abs(Qw.T @ Qw - np.eye(R)).max() <= 1e-13
            assert np.all(np.diag(Rw) > 0) and np.allclose(np.tril(Rw, -1), 0.0)
            assert rel(Qw @ Rw, Aw[n]) <= 1e-13


def test_wide_tail_many_chunks_per_block(cuda_lib):
    # 10000 rows: every one of the (at most 2 x SMs) row blocks takes more
    # than one 32-row chunk, and the last chunks are ragged
    dims, R = (10000, 40, 36), 33
    X, A = problem(dims, R, 11)
    hw, hc = handle(dims, R, X, A, True), handle(dims, R, X, A, False)
    o = oracle.OracleCPALS(X, dims, R)
    o.set_factors(A)
    for h in (hw, hc):
        h.solve_mode(0, "qr", 0.0)
        h.sync()
    o.update_mode(0, oracle.QR, 0.0)
    Aw, lw = hw.get_factors()
    Ac, lc = hc.get_factors()
    assert rel(Aw[0], Ac[0]) <= 1e-12 and rel(lw, lc) <= 1e-12
    assert rel(Aw[0], o.factor(0)) <= 1e-10
    Qw, Rw = hw.get_factor_qr(0)
    Qc, Rc = hc.get_factor_qr(0)
    assert rel(Qw, Qc) <= 1e-12 and rel(Rw, Rc) <= 1e-12
    assert np.abs(Qw.T @ Qw - np.eye(R)).max() <= 1e-13


@pytest.mark.parametrize("dims,R", [((300, 70, 66), 64), ((700, 45, 44), 40)])
def test_factor_set_from_mode_update_repeats_its_qr(cuda_lib, dims, R):
    X, A = problem(dims, R, 7 * R)
    h = handle(dims, R, X, A, True)
    h.iterate(2, solve="qr")
    h.solve_mode(1, "qr", 0.0)
    h.sync()
    F, lam = h.get_factors()
    Q1, R1 = h.get_factor_qr(1)
    h2 = handle(dims, R, X, F, True)
    Q2, R2 = h2.get_factor_qr(1)
    np.testing.assert_array_equal(Q1, Q2)
    np.testing.assert_array_equal(R1, R2)


@pytest.mark.parametrize("dims,R", [((40, 36, 34), 33), ((50, 49, 48), 48), ((70, 66, 65), 64),
                                    ((36, 35, 34, 33), 33)])
def test_wide_fold_steps_match_oracle(cuda_lib, dims, R):
    X, A = problem(dims, R, 3 + R)
    o = oracle.OracleCPALS(X, dims, R)
    o.set_factors(A)
    hw, hc = handle(dims, R, X, A, True), handle(dims, R, X, A, False)
    for n in range(len(dims)):
        Q0, R0 = hw.krp_qr(n)
        Qc, Rc = hc.krp_qr(n)
        Q0o, R0o = o.krp_qr(n)
        assert rel(Q0, Q0o) <= 1e-12 and rel(R0, R0o) <= 1e-12, (n, rel(Q0, Q0o), rel(R0, R0o))
        assert rel(Q0, Qc) <= 1e-12 and rel(R0, Rc) <= 1e-12


def test_ill_conditioned_factor_falls_back_to_householder(cuda_lib):
    dims, R = (200, 60, 50), 40
    X, A = problem(dims, R, 19)
    # mode 1's factor with two columns 1e-9 apart: cond(A_1) near 1e9, past
    # what CholeskyQR2 accepts
    A[1][:, 7] = A[1][:, 3] + 1e-9 * np.random.default_rng(2).standard_normal(dims[1])
    h = handle(dims, R, X, A, True)
    Q, Rm = h.get_factor_qr(1)
    F, _ = h.get_factors()
    assert np.abs(Q.T @ Q - np.eye(R)).max() <= 1e-13
    assert rel(Q @ Rm, F[1]) <= 1e-14
    assert np.all(np.diag(Rm) >= 0) and np.allclose(np.tril(Rm, -1), 0.0)
