"""Pins for the CPU oracle: each check is against something other than the
oracle itself.  The references are LAPACK through numpy, explicit
Kronecker/Khatri-Rao matrix forms built with numpy, exact integer arithmetic,
closed forms, and identities the paper states.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2112_10855_gb300 import inputs
from tests import npforms as F

RNG = np.random.default_rng(2112)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- QR (Sec. 2.1)
@pytest.mark.parametrize("m,n", [(7, 3), (30, 10), (100, 10), (5, 5), (64, 20), (1, 1)])
def test_qr_matches_lapack_with_sign_convention(m, n):
    A = RNG.standard_normal((m, n))
    Q, R = oracle.qr(A)
    Qn, Rn = F.qr_pos(A)
    assert np.abs(np.tril(R, -1)).max() == 0.0
    assert (np.diag(R) >= 0).all()
    assert rel(Q @ R, A) < 1e-14
    assert np.abs(Q.T @ Q - np.eye(n)).max() < 1e-14 * max(m, 8)
    assert rel(Q, Qn) < 1e-12 and rel(R, Rn) < 1e-12


@pytest.mark.parametrize("m,n", [(1, 1), (12, 5), (36, 6), (64, 4), (400, 10), (125, 5), (33, 33)])
def test_qr_flop_count(m, n):
    # Eq. QRcost and the factor-QR cost of Sec. 3.2: a Householder QR of an
    # m x n matrix with Q formed explicitly costs 4 m n^2 + O(n^3) flops; with
    # V_n (m = R^{N-1}, n = R) that is 4 R^{N+1} + O(R^3), with a factor
    # (m = I_n, n = R) 4 I_n R^2 + O(R^3).  Counted exactly (one multiply-add =
    # 2 flops): reflector j updates n-1-j columns of A and n-j columns of Q,
    # each over m-j rows with a dot product and an update, so
    # flops = 4 m n^2 - (4/3) n^3 + 2 n^2 - (2/3) n.
    A = RNG.standard_normal((m, n))
    Q, R, madds = oracle.qr(A, return_madds=True)
    assert 3 * (2 * madds) == 12 * m * n * n - 4 * n ** 3 + 6 * n * n - 2 * n
    assert abs(2 * madds - 4 * m * n * n) <= 4 * n ** 3
    assert rel(Q @ R, A) < 1e-14


def test_qr_flop_count_skips_identity_reflectors():
    # a zero column gives H_j = I, which is neither applied nor counted
    m, n, z = 9, 4, 2
    A = RNG.standard_normal((m, n))
    A[:, z] = 0.0
    _, _, madds = oracle.qr(A, return_madds=True)
    full = sum(2 * (2 * n - 1 - 2 * j) * (m - j) for j in range(n))
    assert madds == full - 2 * (2 * n - 1 - 2 * z) * (m - z)


def test_qr_zero_column():
    A = RNG.standard_normal((9, 4))
    A[:, 2] = 0.0
    Q, R = oracle.qr(A)
    assert rel(Q @ R, A) < 1e-14
    assert R[2, 2] == 0.0


# ---------------------------------------------------- Kronecker / Khatri-Rao (Sec. 2.2)
def test_numpy_kron_follows_paper_index_rule():
    # [A (x) B](K(i-1)+k, M(j-1)+l) = A(i,j) B(k,l), written with 1-based loops
    A = RNG.standard_normal((2, 3))
    B = RNG.standard_normal((4, 5))
    K, M = B.shape
    Kr = np.kron(A, B)
    for i in range(1, 3):
        for j in range(1, 4):
            for k in range(1, K + 1):
                for l in range(1, M + 1):
                    assert Kr[K * (i - 1) + k - 1, M * (j - 1) + l - 1] == A[i - 1, j - 1] * B[k - 1, l - 1]


@pytest.mark.parametrize("rows", [[3], [2, 3], [4, 1, 3], [2, 2, 2, 3]])
def test_krp_columnwise_kronecker(rows):
    R = 4
    mats = [RNG.standard_normal((r, R)) for r in rows]
    K = oracle.krp(mats)
    for r in range(R):
        np.testing.assert_array_equal(K[:, r], F.kron_chain([m[:, r] for m in mats]))


def test_kr_identity():
    # Eq. kr-id: (C (x) D)(A (.) B) = (CA) (.) (DB)
    A = RNG.standard_normal((5, 3))
    B = RNG.standard_normal((4, 3))
    Cm = RNG.standard_normal((6, 5))
    D = RNG.standard_normal((2, 4))
    lhs = np.kron(Cm, D) @ oracle.krp([A, B])
    rhs = oracle.krp([Cm @ A, D @ B])
    assert rel(lhs, rhs) < 1e-14


# ---------------------------------------------------- unfolding and TTM (Sec. 2.2)
@pytest.mark.parametrize("dims", [(3, 4), (2, 3, 4), (3, 2, 2, 3), (2, 3, 1, 2, 2)])
def test_unfold_columns_are_fibers(dims):
    X = RNG.standard_normal(int(np.prod(dims)))
    T = F.tensor(X, dims)
    for n in range(len(dims)):
        Xn = oracle.unfold(X, dims, n)
        np.testing.assert_array_equal(Xn, F.unfold(X, dims, n))
        # pure-python check of the column index rule
        for idx in itertools.product(*[range(d) for d in dims]):
            col, s = 0, 1
            for m in range(len(dims)):
                if m == n:
                    continue
                col += idx[m] * s
                s *= dims[m]
            assert Xn[idx[n], col] == T[idx]


@pytest.mark.parametrize("dims,mode", [((4, 5, 6), 0), ((4, 5, 6), 1), ((4, 5, 6), 2), ((3, 2, 4, 2), 2)])
def test_ttm_matches_tensordot(dims, mode):
    X = RNG.standard_normal(int(np.prod(dims)))
    U = RNG.standard_normal((3, dims[mode]))
    Y = oracle.ttm(X, dims, mode, U)
    T = np.moveaxis(np.tensordot(U, F.tensor(X, dims), axes=([1], [mode])), 0, mode)
    assert rel(Y, T.reshape(-1, order="F")) < 1e-14


# ---------------------------------------------------- Multi-TTM (Eq. multittm)
CASES = [((5, 6), 2), ((4, 5, 6), 3), ((3, 4, 5), 2), ((2, 3, 4, 5), 2), ((3, 2, 4, 2, 3), 2),
         ((7, 3, 2), 4), ((2, 2, 2, 2, 2), 1)]


@pytest.mark.parametrize("dims,R", CASES)
def test_multi_ttm_matches_explicit_kronecker(dims, R):
    X = RNG.standard_normal(int(np.prod(dims)))
    Q = [RNG.standard_normal((d, R)) for d in dims]
    for n in range(len(dims)):
        Y = oracle.multi_ttm(X, dims, n, Q)
        assert Y.shape == (dims[n], R ** (len(dims) - 1))
        assert rel(Y, F.multi_ttm_explicit(X, dims, n, Q)) < 1e-13


@pytest.mark.parametrize("dims,R", [((3, 4, 5), 2), ((2, 3, 4, 3), 2)])
def test_multi_ttm_order_independent(dims, R):
    # Sec. 2.2: the single TTMs of a Multi-TTM can run in any order.
    X = RNG.standard_normal(int(np.prod(dims)))
    Q = [RNG.standard_normal((d, R)) for d in dims]
    for n in range(len(dims)):
        others = [m for m in range(len(dims)) if m != n]
        ref = oracle.multi_ttm(X, dims, n, Q)
        for order in itertools.permutations(others):
            assert rel(oracle.multi_ttm(X, dims, n, Q, order=list(order)), ref) < 1e-14


@pytest.mark.parametrize("dims,R", [((5, 4, 3), 2), ((3, 4, 2, 3), 3)])
def test_multi_ttm_integer_bit_exact(dims, R):
    # integer X and 0/1 factors: every sum is exact, compare bit for bit
    P = int(np.prod(dims))
    Xi = (np.arange(P) * 37 % 97 - 48).astype(np.int64)
    Qi = [(RNG.random((d, R)) < 0.5).astype(np.int64) for d in dims]
    for n in range(len(dims)):
        Y = oracle.multi_ttm(Xi.astype(np.float64), dims, n, [q.astype(np.float64) for q in Qi])
        ref = F.unfold(Xi, dims, n) @ F.kron_chain([Qi[m] for m in F.others_desc(len(dims), n)])
        np.testing.assert_array_equal(Y, ref.astype(np.float64))


def test_multi_ttm_closed_form():
    # X(i,j,k) = 1 + i + 2j + 4k on 2x2x2; all-ones Q_2, Q_3 sum each mode-1 slice:
    # Y_(1)(0) = 1+3+5+7 = 16, Y_(1)(1) = 2+4+6+8 = 20.  Selecting Q = e_1 picks X(:,0,0).
    X = np.arange(1.0, 9.0)
    ones = np.ones((2, 1))
    Y = oracle.multi_ttm(X, (2, 2, 2), 0, [ones, ones, ones])
    np.testing.assert_array_equal(Y[:, 0], [16.0, 20.0])
    e1 = np.array([[1.0], [0.0]])
    Y = oracle.multi_ttm(X, (2, 2, 2), 0, [ones, e1, e1])
    np.testing.assert_array_equal(Y[:, 0], [1.0, 2.0])
    Y = oracle.multi_ttm(X, (2, 2, 2), 2, [e1, ones, ones])     # sum over j of X(0,j,k)
    np.testing.assert_array_equal(Y[:, 0], [1.0 + 3.0, 5.0 + 7.0])


@pytest.mark.parametrize("dims,R,n", [((9, 7, 5), 3, 0), ((6, 8, 5, 7), 2, 2), ((5, 4, 6, 3, 4), 2, 4),
                                      ((5, 5, 5, 4), 2, 3)])
def test_multi_ttm_flop_count(dims, R, n):
    # Eq. TTMcost: with the contracted dims in decreasing order d_1 >= d_2 >= ...,
    # the TTMs cost P*R, P*R^2/d_1, P*R^3/(d_1 d_2), ... multiply-adds, i.e.
    # P * R * (1 + R/d_1 + R^2/(d_1 d_2) + ...) over the N-1 contracted modes.
    X = RNG.standard_normal(int(np.prod(dims)))
    Q = [RNG.standard_normal((d, R)) for d in dims]
    _, madds = oracle.multi_ttm(X, dims, n, Q, return_madds=True)
    d = sorted([dims[m] for m in range(len(dims)) if m != n], reverse=True)
    P = int(np.prod(dims))
    expect, frac = 0.0, 1.0
    for k in range(len(d)):
        expect += P * R * frac
        frac *= R / d[k]
    assert madds == round(expect)
    assert oracle.ttm_order(dims, n) == sorted([m for m in range(len(dims)) if m != n],
                                               key=lambda m: (-dims[m], -m))


# ---------------------------------------------------- structured QR (Eq. Z_qr)
@pytest.mark.parametrize("dims,R", [((6, 5, 7), 3), ((4, 5, 3, 4), 3), ((3, 4, 3, 3, 2), 2)])
def test_structured_qr_of_khatri_rao(dims, R):
    N = len(dims)
    A = [RNG.standard_normal((d, R)) for d in dims]
    QR = [oracle.qr(a) for a in A]
    for n in range(N):
        order = F.others_desc(N, n)
        V = oracle.krp([QR[m][1] for m in order])
        # V_n has R^{N-1} rows; column i (1-based) has i^{N-1} nonzeros (Sec. 3.3.3)
        assert V.shape == (R ** (N - 1), R)
        nnz = (V != 0).sum(axis=0)
        np.testing.assert_array_equal(nnz, [(i + 1) ** (N - 1) for i in range(R)])
        Q0, R0 = oracle.qr(V)
        Qbig = F.kron_chain([QR[m][0] for m in order]) @ Q0
        Zn = F.Z(A, n)
        assert rel(Qbig @ R0, Zn) < 1e-13
        assert np.abs(Qbig.T @ Qbig - np.eye(R)).max() < 1e-13
        Qz, Rz = F.qr_pos(Zn)
        assert rel(Qbig, Qz) < 1e-11 and rel(R0, Rz) < 1e-11


# ---------------------------------------------------- solves (Sec. 2.1, Sec. 3.1)
def _problem(dims, R, seed=1):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal(int(np.prod(dims)))
    A = [rng.standard_normal((d, R)) for d in dims]
    return X, A


@pytest.mark.parametrize("dims,R", [((6, 5, 7), 3), ((4, 5, 3, 4), 3), ((5, 4, 3, 3, 4), 2)])
def test_qr_update_equals_lstsq_on_explicit_Z(dims, R):
    X, A = _problem(dims, R)
    for n in range(len(dims)):
        o = oracle.OracleCPALS(X, dims, R)
        o.set_factors(A)
        assert o.update_mode(n, oracle.QR) == 0
        Ahat = o.last(n)["Ahat"]
        # factors are kept as given at initialisation (lambda = 1)
        ref = np.linalg.lstsq(F.Z(A, n), F.unfold(X, dims, n).T, rcond=None)[0].T
        assert rel(Ahat, ref) < 1e-11
        # the SVD variant without truncation gives the same solution
        o2 = oracle.OracleCPALS(X, dims, R)
        o2.set_factors(A)
        o2.update_mode(n, oracle.SVD, 0.0)
        assert rel(o2.last(n)["Ahat"], ref) < 1e-11


@pytest.mark.parametrize("dims,R", [((6, 5, 7), 3), ((4, 5, 3, 4), 3), ((5, 4, 3, 3, 4), 2)])
def test_sweeps_equal_alternating_lstsq(dims, R):
    # three whole sweeps against ALS written with numpy alone: each mode in
    # order solved by lstsq on the explicit Khatri-Rao product of the current
    # (normalised) factors, its columns then normalised, lambda the last
    # mode's norms -- the sequencing that single-update pins leave open
    X, A0 = _problem(dims, R, seed=11)
    A = [np.array(a) for a in A0]
    lam = np.ones(R)
    for _ in range(3):
        for n in range(len(dims)):
            Ahat = np.linalg.lstsq(F.Z(A, n), F.unfold(X, dims, n).T, rcond=None)[0].T
            lam = np.linalg.norm(Ahat, axis=0)
            A[n] = Ahat / np.where(lam > 0, lam, 1.0)
    o = oracle.OracleCPALS(X, dims, R)
    o.set_factors(A0)
    k, _ = o.iterate(3, solve=oracle.QR)
    assert k == 3
    for n in range(len(dims)):
        assert rel(o.factor(n), A[n]) < 1e-10, (n, rel(o.factor(n), A[n]))
    assert rel(o.lam(), lam) < 1e-10


def test_normal_update_equals_qr_update_well_conditioned():
    dims, R = (8, 7, 6), 3
    X, A = _problem(dims, R, seed=3)
    for n in range(3):
        a = oracle.OracleCPALS(X, dims, R); a.set_factors(A); a.update_mode(n, oracle.QR)
        b = oracle.OracleCPALS(X, dims, R); b.set_factors(A); b.update_mode(n, oracle.NORMAL)
        assert rel(a.factor(n), b.factor(n)) < 1e-10
        assert rel(a.lam(), b.lam()) < 1e-10
        # MTTKRP against the explicit X_(n) Z_n
        M, S = b.last_mttkrp(n)
        assert rel(M, F.unfold(X, dims, n) @ F.Z(A, n)) < 1e-13
        assert rel(S, F.Z(A, n).T @ F.Z(A, n)) < 1e-13


def test_normal_pinv_update_equals_normal_and_solve():
    # CP-ALS-PINV (Sec. 2.3): Ahat = M pinv(S); for a well-conditioned S it is
    # the Cholesky solution and numpy's solve of Ahat S = M
    dims, R = (8, 7, 6), 3
    X, A = _problem(dims, R, seed=4)
    for n in range(3):
        a = oracle.OracleCPALS(X, dims, R); a.set_factors(A); a.update_mode(n, oracle.NORMAL)
        b = oracle.OracleCPALS(X, dims, R); b.set_factors(A); b.update_mode(n, oracle.NORMAL_PINV, 1e-12)
        assert rel(a.factor(n), b.factor(n)) < 1e-10
        M, S = b.last_mttkrp(n)
        ref = np.linalg.solve(S.T, M.T).T
        assert rel(b.last(n)["Ahat"], ref) < 1e-10


def test_normal_pinv_on_singular_gram_matches_numpy_pinv():
    # columns 0 and 1 equal in every factor but mode n make the Hadamard Gram S
    # exactly rank-deficient; CP-ALS-PINV (Sec. 2.3) then gives M pinv(S) with
    # the relative cut, where the Cholesky form (Alg. cp-als) fails
    dims, R = (7, 6, 5), 3
    X, A = _problem(dims, R, seed=9)
    for n in range(3):
        B = [a.copy() for a in A]
        for m in range(3):
            if m != n:
                B[m][:, 1] = B[m][:, 0]
        o = oracle.OracleCPALS(X, dims, R); o.set_factors(B)
        o.update_mode(n, oracle.NORMAL_PINV, 1e-10)
        M, S = o.last_mttkrp(n)
        assert np.linalg.matrix_rank(S) == R - 1
        ref = M @ np.linalg.pinv(S, rcond=1e-10)
        assert rel(o.last(n)["Ahat"], ref) < 1e-9
        assert np.abs(o.last(n)["Ahat"][:, 0] - o.last(n)["Ahat"][:, 1]).max() < 1e-9 * np.abs(ref).max()


def test_trsm_against_solve():
    R0 = np.triu(RNG.standard_normal((6, 6))) + 4 * np.eye(6)
    W = RNG.standard_normal((11, 6))
    A = oracle.trsm_qr(W, R0)
    assert rel(A @ R0.T, W) < 1e-14
    with pytest.raises(np.linalg.LinAlgError):
        R1 = R0.copy(); R1[3, 3] = 0.0
        oracle.trsm_qr(W, R1)


def test_trsm_singularity_threshold():
    # the reading of the QR solve's singularity test: R0 is singular when some
    # |R0(k,k)| <= R * eps * max_j |R0(j,j)|; just above the bound it solves,
    # at or below it (or NaN) it refuses
    R = 6
    eps = np.finfo(np.float64).eps
    R0 = np.triu(RNG.standard_normal((R, R))) + 3 * np.eye(R)
    R0[1, 1] = 10.0
    dmax = np.abs(np.diag(R0)).max()
    W = RNG.standard_normal((5, R))
    bound = R * eps * dmax
    for k in (0, 4):
        ok = R0.copy(); ok[k, k] = 2.0 * bound
        A = oracle.trsm_qr(W, ok)
        # nearly singular: a small backward error, not a small residual
        assert np.isfinite(A).all()
        assert np.linalg.norm(A @ ok.T - W) <= 1e-13 * np.linalg.norm(A) * np.linalg.norm(ok)
        for v in (bound, 0.5 * bound, -0.5 * bound, 0.0, np.nan):
            bad = R0.copy(); bad[k, k] = v
            with pytest.raises(np.linalg.LinAlgError):
                oracle.trsm_qr(W, bad)


def test_jacobi_svd_against_lapack():
    for n in (1, 2, 5, 10, 17):
        A = RNG.standard_normal((n, n))
        U, S, V = oracle.jacobi_svd(A)
        assert rel(S, np.linalg.svd(A, compute_uv=False)) < 1e-13
        assert rel(U @ np.diag(S) @ V.T, A) < 1e-13
        assert np.abs(V.T @ V - np.eye(n)).max() < 1e-13
        assert np.abs(U.T @ U - np.eye(n)).max() < 1e-12


def test_svd_solve_truncation_matches_pinv():
    # rank-deficient R0 (two equal rows after a rotation): the truncated solve
    # equals W pinv(R0^T) with the same relative cut
    B = RNG.standard_normal((6, 4))
    R0 = np.linalg.qr(np.c_[B, B[:, 0] + 1e-13 * RNG.standard_normal(6), B[:, 1]])[1]
    W = RNG.standard_normal((9, 6))
    for rtol in (1e-10, 1e-6):
        A, kept = oracle.svd_solve(W, R0, rtol)
        assert kept == 4
        ref = W @ np.linalg.pinv(R0.T, rcond=rtol)
        assert rel(A, ref) < 1e-9


def test_cholesky_solve_against_numpy():
    B = RNG.standard_normal((10, 5))
    S = B.T @ B + np.eye(5)
    M = RNG.standard_normal((7, 5))
    A = oracle.cholesky_solve(M, S)
    assert rel(A, np.linalg.solve(S.T, M.T).T) < 1e-13
    with pytest.raises(np.linalg.LinAlgError):
        oracle.cholesky_solve(M, -S)


def test_normalize_two_norm():
    A = RNG.standard_normal((8, 3))
    A[:, 1] = 0.0
    An, lam = oracle.normalize(A)
    np.testing.assert_allclose(lam, np.linalg.norm(A, axis=0), rtol=1e-15)
    assert lam[1] == 0.0
    np.testing.assert_allclose(np.linalg.norm(An[:, [0, 2]], axis=0), 1.0, rtol=1e-15)


# ---------------------------------------------------- error and convergence (Sec. 3.3.1)
def test_efficient_fit_matches_direct():
    p = inputs.planted((9, 8, 7), 3, seed=5, init_seed=6, noise=0.05)
    o = oracle.OracleCPALS(p.X, p.dims, 3)
    o.set_factors(p.init_factors)
    for solve in (oracle.QR, oracle.NORMAL):
        k, fits = o.iterate(5, solve=solve)
        assert k == 5
        direct = o.fit_direct()
        # the efficient form is accurate to about sqrt(eps) relative
        assert abs(fits[-1] - direct) < 1e-7
        assert rel(oracle.residual_direct(p.X, p.dims, o.lam(), o.factors()),
                   np.linalg.norm(p.X - F.full(o.lam(), o.factors()))) < 1e-12


def test_noiseless_exact_rank_converges():
    p = inputs.planted((10, 9, 8), 3, seed=11, init_seed=12, noise=0.0)
    for solve in (oracle.QR, oracle.SVD):
        o = oracle.OracleCPALS(p.X, p.dims, 3)
        o.set_factors(p.init_factors)
        # fixed sweep count: the efficient fit saturates near sqrt(eps) (Sec. 3.3.1),
        # so a fit-change stop would end the run early
        o.iterate(200, tol=0.0, solve=solve, rtol=1e-12)
        assert 1.0 - o.fit_direct() < 1e-12
        assert oracle.score(p.dims, p.true_weights * np.prod(
            [np.linalg.norm(a, axis=0) for a in p.true_factors], axis=0), p.true_factors,
            o.lam(), o.factors()) > 0.999999


def test_singular_qr_solve_reported():
    # duplicate columns make V_n rank deficient: the QR solve refuses, SVD truncates
    dims, R = (6, 5, 4), 3
    X, A = _problem(dims, R, seed=9)
    for m in range(3):
        A[m][:, 2] = A[m][:, 1]
    o = oracle.OracleCPALS(X, dims, R)
    o.set_factors(A)
    assert o.update_mode(0, oracle.QR) == 1
    o2 = oracle.OracleCPALS(X, dims, R)
    o2.set_factors(A)
    assert o2.update_mode(0, oracle.SVD, 1e-10) == 0
    ref = np.linalg.lstsq(F.Z(A, 0), F.unfold(X, dims, 0).T, rcond=1e-10)[0].T
    assert rel(o2.last(0)["Ahat"], ref) < 1e-9


# ---------------------------------------------------- score (Sec. 4.2 metric)
def test_score_invariances():
    dims, R = (6, 5, 4), 4
    A = [RNG.standard_normal((d, R)) for d in dims]
    lam = np.array([3.0, 2.0, 1.0, 0.5])
    assert abs(oracle.score(dims, lam, A, lam, A) - 1.0) < 1e-14
    perm = [2, 0, 3, 1]
    B = [a[:, perm] * np.array([1, -1, 1, -1])[None, :] * 2.5 for a in A]
    assert abs(oracle.score(dims, lam, A, lam[perm], B) - 1.0) < 1e-14
    C = [RNG.standard_normal((d, R)) for d in dims]
    assert oracle.score(dims, lam, A, lam, C) < 0.5
    assert abs(oracle.score(dims, lam, A, 2 * lam, A) - 0.5) < 1e-14


@pytest.mark.parametrize("N,n", [(2, 9), (3, 8), (4, 7), (5, 6), (6, 5), (10, 3)])
def test_sine_of_sums_representations(N, n):
    # Sec. 4.3: the 2^{N-1}-term expansion and the rank-N representation of
    # Eq. sinsum_rkd both reproduce sin(x_1 + ... + x_N) on the grid
    # 2 pi k / n; this pins the Kruskal inputs of the sine-of-sums workload
    # (and cp_full, which expands them for the oracle)
    from paper_2112_10855_gb300 import inputs
    x = inputs.sine_grid(n)
    grids = np.meshgrid(*([x] * N), indexing="ij")
    ref = np.sin(sum(grids)).reshape(-1, order="F")
    dims = (n,) * N
    mu, V = inputs.sine_of_sums_expanded(N, n)
    assert len(mu) == 2 ** (N - 1)
    assert np.abs(inputs.cp_full(dims, V, mu) - ref).max() <= 1e-14 * N
    mu, V = inputs.sine_of_sums_rank_n(N, n)
    assert len(mu) == N
    assert np.abs(inputs.cp_full(dims, V, mu) - ref).max() <= 1e-13 * N


def test_package_score_equals_oracle_brute_force():
    # the package's factor-match score (linear assignment) against the
    # oracle's brute force over permutations, on random and on permuted,
    # sign-flipped and rescaled copies of a model
    from paper_2112_10855_gb300.score import factor_match_score
    rng = np.random.default_rng(5)
    for R in (1, 2, 4, 6):
        dims = (7, 6, 5)
        A1 = [rng.standard_normal((d, R)) for d in dims]
        A2 = [rng.standard_normal((d, R)) for d in dims]
        l1, l2 = rng.random(R) + 0.5, rng.random(R) + 0.5
        assert abs(factor_match_score(l1, A1, l2, A2) - oracle.score(dims, l1, A1, l2, A2)) < 1e-13
        perm = rng.permutation(R)
        A3 = [(-a[:, perm]) * 3.0 for a in A1]
        assert abs(factor_match_score(l1, A1, l1[perm], A3) - 1.0) < 1e-13
        assert abs(oracle.score(dims, l1, A1, l1[perm], A3) - 1.0) < 1e-13
