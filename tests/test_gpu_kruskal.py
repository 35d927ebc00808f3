"""Kruskal-tensor input (Sec. 3.3.2) against the FP64 oracle run on the dense
expansion of the same tensor.

The Kruskal path computes the same least-squares updates from the factors of
X (W_n from an MTTKRP of Q0 kept in factored form, the normal-equations
MTTKRP from Hadamard products of V_m^T A_m), so every quantity must match the
dense algorithm up to rounding: FP64 bars as in test_gpu_parity (1e-12 for
Y_(n), W_n and R0; 1e-10 for a mode update and for fits per sweep).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2112_10855_gb300 import cpals, inputs

pytestmark = pytest.mark.gpu

OSOLVE = {"qr": oracle.QR, "svd": oracle.SVD, "normal": oracle.NORMAL, "normal_pinv": oracle.NORMAL_PINV}


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def kruskal_handle(dims, R, mu, V, A=None, device=False):
    h = cpals.CPALS(dims, R, kruskal_rank=len(mu))
    if device:
        h.set_tensor_kruskal(torch.from_numpy(np.asarray(mu)).cuda(),
                             [torch.from_numpy(np.asfortranarray(v).T.copy()).cuda().t() for v in V])
    else:
        h.set_tensor_kruskal(np.asarray(mu, dtype=np.float64), [np.asfortranarray(v) for v in V])
    if A is not None:
        h.set_factors([np.asfortranarray(a) for a in A])
    return h


def init_factors(dims, R, seed):
    rng = np.random.default_rng(seed)
    return [np.asfortranarray(rng.standard_normal((d, R))) for d in dims]


# orders 2..6 with ragged dims; Kruskal ranks below, equal to and above R
CASES = [((30, 25), 4, 6), ((9, 8, 7), 3, 5), ((12, 11, 10, 9), 3, 2), ((7, 6, 5, 5, 4), 2, 7),
         ((6, 5, 5, 4, 4, 3), 2, 3), ((40, 35, 30), 10, 12)]


@pytest.mark.parametrize("dims,R,S", CASES)
def test_multi_ttm_w_and_r0_match_dense_oracle(cuda_lib, dims, R, S):
    mu, V = inputs.random_kruskal(dims, S, seed=7)
    X = inputs.cp_full(dims, V, mu)
    A = init_factors(dims, R, 8)
    h = kruskal_handle(dims, R, mu, V, A)
    for n in range(len(dims)):
        o = oracle.OracleCPALS(X, dims, R)
        o.set_factors(A)
        o.update_mode(n, oracle.QR)
        ref = o.last(n)
        _, R0 = h.krp_qr(n)
        assert rel(R0, ref["R0"]) <= 1e-12
        Y, W = h.multi_ttm(n, want_W=True)
        assert rel(Y, ref["Y"]) <= 1e-12, n
        assert rel(W, ref["W"]) <= 1e-12, n


@pytest.mark.parametrize("solve", ["qr", "svd", "normal", "normal_pinv"])
@pytest.mark.parametrize("dims,R,S", [((9, 8, 7), 3, 5), ((12, 11, 10, 9), 3, 4), ((40, 35, 30), 10, 12)])
def test_mode_update_matches_dense_oracle(cuda_lib, solve, dims, R, S):
    mu, V = inputs.random_kruskal(dims, S, seed=17)
    X = inputs.cp_full(dims, V, mu)
    A = init_factors(dims, R, 18)
    for n in range(len(dims)):
        o = oracle.OracleCPALS(X, dims, R)
        o.set_factors(A)
        assert o.update_mode(n, OSOLVE[solve], 1e-12) == 0
        h = kruskal_handle(dims, R, mu, V, A)
        h.solve_mode(n, solve, 1e-12)
        Ag, lam = h.get_factors()
        assert rel(Ag[n], o.factor(n)) <= 1e-10, (n, rel(Ag[n], o.factor(n)))
        assert rel(lam, o.lam()) <= 1e-10


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_kruskal_mttkrp_matches_dense(cuda_lib, mode):
    dims, R, S = (21, 17, 13), 4, 6
    mu, V = inputs.random_kruskal(dims, S, seed=27)
    X = inputs.cp_full(dims, V, mu)
    A = init_factors(dims, R, 28)
    h = kruskal_handle(dims, R, mu, V, A)
    assert rel(h.mttkrp(mode), oracle.mttkrp(X, dims, mode, A)) <= 1e-12


@pytest.mark.parametrize("solve", ["qr", "svd", "normal", "normal_pinv"])
def test_sweeps_match_dense_oracle(cuda_lib, solve):
    dims, R, S = (14, 13, 12, 11), 3, 5
    mu, V = inputs.random_kruskal(dims, S, seed=37)
    X = inputs.cp_full(dims, V, mu)
    A = init_factors(dims, R, 38)
    o = oracle.OracleCPALS(X, dims, R)
    o.set_factors(A)
    _, fo = o.iterate(8, solve=OSOLVE[solve], rtol=1e-12)
    h = kruskal_handle(dims, R, mu, V, A, device=True)
    fg = h.iterate(8, solve=solve, svd_rtol=1e-12)
    assert np.abs(fg - fo).max() <= 1e-10
    Ag, _ = h.get_factors()
    for m in range(len(dims)):
        assert rel(Ag[m], o.factor(m)) <= 1e-8
    assert abs(h.fit(direct=True) - o.fit_direct()) <= 1e-10


def test_kruskal_handle_equals_dense_handle(cuda_lib):
    # the same tensor through the dense path (Multi-TTM over X) and the
    # Kruskal path: only rounding differs
    dims, R, S = (30, 28, 26), 6, 9
    mu, V = inputs.random_kruskal(dims, S, seed=47)
    X = inputs.cp_full(dims, V, mu)
    A = init_factors(dims, R, 48)
    hd = cpals.CPALS(dims, R)
    hd.set_tensor(torch.from_numpy(X).cuda())
    hd.set_factors(A)
    hk = kruskal_handle(dims, R, mu, V, A)
    fd = hd.iterate(10, solve="qr")
    fk = hk.iterate(10, solve="qr")
    assert np.abs(fd - fk).max() <= 1e-11
    assert abs(hd.fit(direct=True) - hk.fit(direct=True)) <= 1e-11


def test_sine_of_sums_four_way(cuda_lib):
    # Sec. 4.3: sin(x_1 + ... + x_4) on a 16-point grid, input in its rank-8
    # expanded form, target rank 4 (the exact rank); QR and SVD sweeps
    N, n = 4, 16
    mu, V = inputs.sine_of_sums_expanded(N, n)
    dims = (n,) * N
    X = inputs.cp_full(dims, V, mu)
    A = init_factors(dims, N, 57)
    for solve in ("qr", "svd"):
        o = oracle.OracleCPALS(X, dims, N)
        o.set_factors(A)
        _, fo = o.iterate(6, solve=OSOLVE[solve], rtol=1e-12)
        h = kruskal_handle(dims, N, mu, V, A)
        fg = h.iterate(6, solve=solve, svd_rtol=1e-12)
        assert np.abs(fg - fo).max() <= 1e-10
        assert abs(h.fit(direct=True) - o.fit_direct()) <= 1e-10


def test_ten_way_rank_n_representation(cuda_lib):
    # order 10 (Sec. 4.3's higher-order case) at a size the oracle can expand:
    # 4^10 entries, the rank-10 representation of Eq. sinsum_rkd as input,
    # target rank 3 (V_n has 3^9 rows)
    N, n, R = 10, 4, 3
    mu, V = inputs.sine_of_sums_rank_n(N, n)
    dims = (n,) * N
    X = inputs.cp_full(dims, V, mu)
    A = init_factors(dims, R, 67)
    o = oracle.OracleCPALS(X, dims, R)
    o.set_factors(A)
    _, fo = o.iterate(3, solve=oracle.QR)
    h = kruskal_handle(dims, R, mu, V, A)
    fg = h.iterate(3, solve="qr")
    assert np.abs(fg - fo).max() <= 1e-9
    Ag, _ = h.get_factors()
    for m in range(N):
        assert rel(Ag[m], o.factor(m)) <= 1e-7


def gram_fit(mu, V, lam, A):
    """1 - ||X - Xhat|| / ||X|| from Gram matrices (host, for sizes no dense check reaches)."""
    H = np.ones((len(mu), len(mu)))
    K = np.ones((len(mu), len(lam)))
    G = np.ones((len(lam), len(lam)))
    for v, a in zip(V, A):
        H *= v.T @ v
        K *= v.T @ a
        G *= a.T @ a
    x2 = mu @ H @ mu
    r2 = x2 - 2 * mu @ K @ lam + lam @ G @ lam
    return 1.0 - np.sqrt(max(r2, 0.0)) / np.sqrt(x2)


def test_rank_power_beyond_dense_storage(cuda_lib):
    # order 10, rank 10 on a 12-point grid: the dense tensor would hold 12^10
    # entries and Q0 10^9 x 10, neither of which the Kruskal path forms; the
    # efficient fit must equal the fit from Gram matrices of the returned factors
    N, n, R = 10, 12, 10
    mu, V = inputs.sine_of_sums_rank_n(N, n)
    dims = (n,) * N
    A = init_factors(dims, R, 77)
    h = kruskal_handle(dims, R, mu, V, A)
    fits = h.iterate(5, solve="qr")
    Ag, lam = h.get_factors()
    assert np.all(np.isfinite(fits))
    assert abs(fits[-1] - gram_fit(mu, V, lam, Ag)) <= 1e-8


def test_kruskal_handle_rejects_dense_calls(cuda_lib):
    dims, R, S = (6, 5, 4), 2, 3
    mu, V = inputs.random_kruskal(dims, S, seed=1)
    h = kruskal_handle(dims, R, mu, V, init_factors(dims, R, 2))
    with pytest.raises(cpals.CPALSError):
        h.set_tensor(np.zeros(int(np.prod(dims))))
    with pytest.raises(cpals.CPALSError):
        h.ttm_first(0)
