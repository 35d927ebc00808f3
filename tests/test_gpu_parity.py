"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle.

Every case feeds both sides identical seeded inputs.  FP64 bars:
  - Multi-TTM Y_(n), W_n, Q0/R0 and factor QR: relative Frobenius <= 1e-12;
  - one mode update (A_n, lambda): <= 1e-10;
  - fit per sweep: |gpu - oracle| <= 1e-10.
Integer-valued inputs make the index bookkeeping bit-exact.  FP32 bars are
stated per test (the error bound of an FP32 dot product of length K).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2112_10855_gb300 import cpals, inputs
from tests import npforms as F

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def gaussian_problem(dims, R, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal(int(np.prod(dims)))
    A = [np.asfortranarray(rng.standard_normal((d, R))) for d in dims]
    return X, A


def gpu_handle(dims, R, X, A=None, precision="f64", device_x=True):
    h = cpals.CPALS(dims, R, precision)
    if device_x:
        h.set_tensor(torch.from_numpy(np.ascontiguousarray(X)).cuda())
    else:
        h.set_tensor(np.ascontiguousarray(X))
    if A is not None:
        h.set_factors([np.asfortranarray(a) for a in A])
    return h


# shapes spanning several 256-row tiles with ragged tails, all orders 2..5
SHAPES = [((50, 33), 4), ((37, 29, 41), 5), ((23, 19, 17), 3), ((12, 11, 10, 9), 3), ((7, 6, 5, 4, 3), 2),
          ((64, 64, 64), 16), ((40, 35, 30), 20), ((9, 8, 7), 7)]


@pytest.mark.parametrize("dims,R", SHAPES)
def test_multi_ttm_matches_oracle(cuda_lib, dims, R):
    X, A = gaussian_problem(dims, R, seed=sum(dims) + R)
    QR = [oracle.qr(a) for a in A]
    h = gpu_handle(dims, R, X)
    h.set_factor_qr([q for q, _ in QR], [r for _, r in QR])
    for n in range(len(dims)):
        Y, _ = h.multi_ttm(n)
        ref = oracle.multi_ttm(X, dims, n, [q for q, _ in QR])
        assert Y.shape == ref.shape
        assert rel(Y, ref) <= 1e-12, (n, rel(Y, ref))


# the later TTMs of the FP32 Multi-TTM run through shared-memory tiles: the
# last four shapes give them L = 1, L = 3 and L = 6 (staged along k), L >= 16
# (staged along rows), ragged 128-row tiles, K of 20 to 70 (one to three
# chunks of 32) and R = 33 (two column blocks)
@pytest.mark.parametrize("dims,R", [((5, 4, 3), 2), ((3, 4, 3, 3), 3), ((40, 30, 20), 6), ((300, 7), 5),
                                    ((70, 150, 12), 12), ((45, 40, 70), 3), ((30, 20, 25), 6),
                                    ((40, 36, 34, 33), 33)])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_multi_ttm_index_bookkeeping_bit_exact(cuda_lib, dims, R, precision):
    # integer X and 0/1 Q: every partial sum is an integer below 2^24, exact in
    # FP64 and FP32, so the two sides must agree bit for bit
    P = int(np.prod(dims))
    X = (np.arange(P) * 37 % 97 - 48).astype(np.float64)
    rng = np.random.default_rng(7)
    Q = [np.asfortranarray((rng.random((d, R)) < 0.5).astype(np.float64)) for d in dims]
    Rm = [np.asfortranarray(np.triu(np.ones((R, R)))) for _ in dims]
    h = gpu_handle(dims, R, X, precision=precision)
    h.set_factor_qr(Q, Rm)
    for n in range(len(dims)):
        Y, _ = h.multi_ttm(n)
        np.testing.assert_array_equal(Y, oracle.multi_ttm(X, dims, n, Q))


# (m, R): one Householder CTA, and the multi-launch TSQR (leaves of >= R rows
# and the tree of triangle pairs) for the taller or wider shapes
@pytest.mark.parametrize("m,R", [(10, 10), (50, 5), (400, 10), (1000, 10), (3000, 20), (500, 64), (1, 1), (129, 64),
                                 (21, 10), (120, 20), (64, 32), (300, 32), (2000, 32), (2500, 32), (67, 8)])
def test_factor_qr_matches_oracle(cuda_lib, m, R):
    rng = np.random.default_rng(m + R)
    A = np.asfortranarray(rng.standard_normal((m, R)))
    dims = (m, R, R)
    X = np.zeros(m * R * R)
    h = gpu_handle(dims, R, X)
    h.set_factors([A, np.asfortranarray(np.eye(R)), np.asfortranarray(np.eye(R))])
    Q, Rm = h.get_factor_qr(0)
    Qo, Ro = oracle.qr(A)
    assert rel(Q, Qo) <= 1e-12 and rel(Rm, Ro) <= 1e-12
    assert (np.diag(Rm) >= 0).all()


def test_factor_qr_rank_deficient(cuda_lib):
    # a zero column and a repeated column: the thin QR is not unique there, so
    # check the factorisation itself (Q R = A, Q^T Q = I, R upper triangular
    # with diag(R) >= 0) and the R entries the rank fixes
    m, R = 400, 10
    rng = np.random.default_rng(5)
    A = rng.standard_normal((m, R))
    A[:, 3] = 0.0
    A[:, 7] = A[:, 1]
    A = np.asfortranarray(A)
    h = gpu_handle((m, R, R), R, np.zeros(m * R * R))
    h.set_factors([A, np.asfortranarray(np.eye(R)), np.asfortranarray(np.eye(R))])
    Q, Rm = h.get_factor_qr(0)
    assert np.abs(Q @ Rm - A).max() <= 1e-13 * np.abs(A).max() * m
    assert np.abs(Q.T @ Q - np.eye(R)).max() <= 1e-13
    assert np.allclose(np.tril(Rm, -1), 0.0) and (np.diag(Rm) >= 0).all()
    _, Ro = oracle.qr(np.asfortranarray(A[:, :3]))
    assert rel(Rm[:3, :3], Ro) <= 1e-12


# R <= 32 goes through the staircase QR of each Khatri-Rao step (rows ordered
# by max(i, j)); R = 1 and R = 32 are its edges; R = 48 the dense TSQR
@pytest.mark.parametrize("dims,R", [((6, 5, 7), 3), ((20, 20, 20), 10), ((12, 11, 10, 9), 5), ((30, 30, 30), 16),
                                    ((7, 6, 5, 4, 3), 3), ((20, 20, 20, 20), 20), ((5, 4, 3), 1),
                                    ((40, 36, 34), 32), ((10, 9, 8, 7), 7), ((50, 49, 48), 48)])
def test_krp_qr_matches_oracle(cuda_lib, dims, R):
    X, A = gaussian_problem(dims, R, seed=3)
    o = oracle.OracleCPALS(X, dims, R)
    o.set_factors(A)
    h = gpu_handle(dims, R, X, A)
    for n in range(len(dims)):
        Q0, R0 = h.krp_qr(n)
        Q0o, R0o = o.krp_qr(n)
        assert rel(Q0, Q0o) <= 1e-12 and rel(R0, R0o) <= 1e-12, n


@pytest.mark.parametrize("dims,R", [((37, 29, 41), 5), ((12, 11, 10, 9), 3), ((50, 33), 4)])
def test_apply_q0_matches_oracle(cuda_lib, dims, R):
    X, A = gaussian_problem(dims, R, seed=5)
    for n in range(len(dims)):
        o = oracle.OracleCPALS(X, dims, R)
        o.set_factors(A)
        o.update_mode(n, oracle.QR)
        ref = o.last(n)
        h = gpu_handle(dims, R, X, A)
        h.krp_qr(n)
        Y, W = h.multi_ttm(n, want_W=True)
        assert rel(Y, ref["Y"]) <= 1e-12
        assert rel(W, ref["W"]) <= 1e-12


OSOLVE = {"qr": oracle.QR, "svd": oracle.SVD, "normal": oracle.NORMAL, "normal_pinv": oracle.NORMAL_PINV}


@pytest.mark.parametrize("solve", ["qr", "svd", "normal", "normal_pinv"])
@pytest.mark.parametrize("dims,R", [((37, 29, 41), 5), ((12, 11, 10, 9), 3), ((60, 50, 40), 10),
                                    ((70, 66, 64), 64)])
def test_mode_update_matches_oracle(cuda_lib, solve, dims, R):
    # rank 64: V_n (4096 x 64) goes through the TSQR tree of triangle pairs,
    # the SVD and pseudo-inverse solves through the 64 x 64 Jacobi SVD
    X, A = gaussian_problem(dims, R, seed=11)
    osolve = OSOLVE[solve]
    for n in range(len(dims)):
        o = oracle.OracleCPALS(X, dims, R)
        o.set_factors(A)
        assert o.update_mode(n, osolve, 1e-12) == 0
        h = gpu_handle(dims, R, X, A)
        h.solve_mode(n, solve, 1e-12)
        Ag, lam = h.get_factors()
        assert rel(Ag[n], o.factor(n)) <= 1e-10, (n, rel(Ag[n], o.factor(n)))
        assert rel(lam, o.lam()) <= 1e-10
        Qg, Rg = h.get_factor_qr(n)
        Qo, Ro = o.qr_factor(n)
        assert rel(Rg, Ro) <= 1e-10


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_mttkrp_matches_oracle(cuda_lib, mode):
    dims, R = (33, 27, 45), 6
    X, A = gaussian_problem(dims, R, seed=13)
    h = gpu_handle(dims, R, X, A)
    M = h.mttkrp(mode)
    assert rel(M, oracle.mttkrp(X, dims, mode, A)) <= 1e-12


@pytest.mark.parametrize("solve", ["qr", "svd", "normal", "normal_pinv"])
def test_sweeps_match_oracle_c1_shape(cuda_lib, solve):
    # 50^3, rank 5, N(0,1) factors, unit weights, 1% noise, 20 sweeps
    p = inputs.workload_c1()
    osolve = OSOLVE[solve]
    o = oracle.OracleCPALS(p.X, p.dims, p.rank)
    o.set_factors(p.init_factors)
    k, fits_o = o.iterate(20, solve=osolve, rtol=1e-10)
    assert k == 20
    h = gpu_handle(p.dims, p.rank, p.X, p.init_factors)
    fits = h.iterate(20, solve=solve, svd_rtol=1e-10)
    assert len(fits) == 20
    assert np.abs(fits - fits_o).max() <= 1e-10
    Ag, lam = h.get_factors()
    for m in range(3):
        assert rel(Ag[m], o.factor(m)) <= 1e-8
    assert abs(h.fit(direct=True) - o.fit_direct()) <= 1e-10


@pytest.mark.parametrize("dims,R", [((24, 22, 20), 4), ((14, 13, 12, 11), 3), ((9, 8, 8, 7, 6), 2),
                                    ((30, 30, 30), 6)])
@pytest.mark.parametrize("solve", ["qr", "svd", "normal", "normal_pinv"])
def test_dimension_tree_sweeps_match_oracle(cuda_lib, dims, R, solve):
    # sweeps with the dimension tree (two passes over X per sweep) against the
    # oracle's per-mode Multi-TTMs: only rounding differs
    p = inputs.planted(dims, R, seed=31, init_seed=32, noise=0.02)
    osolve = OSOLVE[solve]
    o = oracle.OracleCPALS(p.X, p.dims, R)
    o.set_factors(p.init_factors)
    _, fits_o = o.iterate(6, solve=osolve, rtol=1e-12)
    h = gpu_handle(p.dims, R, p.X, p.init_factors)
    fits = h.iterate(6, solve=solve, svd_rtol=1e-12)
    assert np.abs(fits - fits_o).max() <= 1e-10
    A, lam = h.get_factors()
    for m in range(len(dims)):
        assert rel(A[m], o.factor(m)) <= 1e-8
    # and against the same library without the tree
    h2 = gpu_handle(p.dims, R, p.X, p.init_factors)
    h2.set_dimtree(False)
    fits2 = h2.iterate(6, solve=solve, svd_rtol=1e-12)
    assert np.abs(fits - fits2).max() <= 1e-11


@pytest.mark.parametrize("dims,R", [((30, 30, 30), 6), ((14, 13, 12, 11), 3), ((9, 8, 8, 7, 6), 2),
                                    ((6, 6, 5, 5, 4, 4), 2), ((36, 35, 34, 33), 33)])
@pytest.mark.parametrize("solve", ["qr", "svd"])
def test_tree_qr_of_vn_sweeps_match_oracle(cuda_lib, dims, R, solve):
    # the QR of V_n from per-half QRs (Kronecker apply of the other half's Q)
    # against the oracle's QR of the formed V_n and against the same library
    # folding all N-1 factors per mode; R = 33 takes the Householder step path
    p = inputs.planted(dims, R, seed=33, init_seed=34, noise=0.02)
    o = oracle.OracleCPALS(p.X, p.dims, R)
    o.set_factors(p.init_factors)
    _, fits_o = o.iterate(3, solve=OSOLVE[solve], rtol=1e-12)
    h = gpu_handle(p.dims, R, p.X, p.init_factors)
    fits = h.iterate(3, solve=solve, svd_rtol=1e-12)
    assert np.abs(fits - fits_o).max() <= 1e-10
    A, lam = h.get_factors()
    for m in range(len(dims)):
        assert rel(A[m], o.factor(m)) <= 1e-8
    h2 = gpu_handle(p.dims, R, p.X, p.init_factors)
    h2.set_krp_tree(False)
    fits2 = h2.iterate(3, solve=solve, svd_rtol=1e-12)
    assert np.abs(fits - fits2).max() <= 1e-11
    A2, _ = h2.get_factors()
    for m in range(len(dims)):
        assert rel(A[m], A2[m]) <= 1e-9


def test_direct_fit_and_resume(cuda_lib):
    # 10 + 10 sweeps equal 20 sweeps bit for bit (checkpoint = get/set factors)
    p = inputs.workload_c1(size=24, rank=4)
    h1 = gpu_handle(p.dims, p.rank, p.X, p.init_factors)
    h1.iterate(20)
    A20, l20 = h1.get_factors()
    h2 = gpu_handle(p.dims, p.rank, p.X, p.init_factors)
    h2.iterate(10)
    A10, l10 = h2.get_factors()
    h3 = gpu_handle(p.dims, p.rank, p.X)
    h3.set_factors(A10, l10)
    h3.iterate(10)
    A, l = h3.get_factors()
    for m in range(3):
        np.testing.assert_array_equal(A[m], A20[m])
    np.testing.assert_array_equal(l, l20)
    o = oracle.OracleCPALS(p.X, p.dims, p.rank)
    o.set_factors(A20, l20)
    assert abs(h1.fit(direct=True) - o.fit_direct()) <= 1e-12


def test_singular_qr_solve_is_reported_and_factor_kept(cuda_lib):
    dims, R = (16, 15, 14), 3
    X, A = gaussian_problem(dims, R, seed=9)
    for m in range(3):
        A[m][:, 2] = A[m][:, 1]
    h = gpu_handle(dims, R, X, A)
    before, _ = h.get_factors()
    h.solve_mode(0, "qr")
    with pytest.raises(cpals.SingularError):
        h.sync()
    after, _ = h.get_factors()
    np.testing.assert_array_equal(after[0], before[0])
    # the SVD solve truncates the rank-deficient direction: min-norm lstsq
    h.solve_mode(0, "svd", 1e-10)
    h.sync()
    Ag, lam = h.get_factors()
    o = oracle.OracleCPALS(X, dims, R)
    o.set_factors(A)
    o.update_mode(0, oracle.SVD, 1e-10)
    assert rel(Ag[0] * lam[None, :], o.factor(0) * o.lam()[None, :]) <= 1e-8
    # CP-ALS-PINV on the exactly rank-deficient Hadamard Gram: M pinv(S)
    h = gpu_handle(dims, R, X, A)
    h.solve_mode(0, "normal_pinv", 1e-10)
    h.sync()
    Ag, lam = h.get_factors()
    o = oracle.OracleCPALS(X, dims, R)
    o.set_factors(A)
    o.update_mode(0, oracle.NORMAL_PINV, 1e-10)
    assert rel(Ag[0] * lam[None, :], o.factor(0) * o.lam()[None, :]) <= 1e-8


def test_host_tensor_path_and_edge_shapes(cuda_lib):
    # host X (copied by the library), rank 1, order 2, rank == a dim
    for dims, R in [((9, 1 + 8), 1), ((5, 5), 5), ((3, 4, 5), 3)]:
        X, A = gaussian_problem(dims, R, seed=17)
        h = gpu_handle(dims, R, X, A, device_x=False)
        o = oracle.OracleCPALS(X, dims, R)
        o.set_factors(A)
        for n in range(len(dims)):
            h.solve_mode(n, "qr")
            o.update_mode(n, oracle.QR)
        h.sync()
        Ag, lam = h.get_factors()
        for n in range(len(dims)):
            assert rel(Ag[n], o.factor(n)) <= 1e-9


@pytest.mark.parametrize("dims,R", [((37, 29, 41), 5), ((40, 35, 30), 20), ((12, 11, 10, 9), 3)])
def test_f32_multi_ttm_error_bound(cuda_lib, dims, R):
    # FP32 copy of X and FP32 accumulation: each entry of Y is a sum of
    # prod_{m != n} I_m products; relative Frobenius error stays below
    # ~sqrt(K) * 2^-24 per TTM, bounded here by 2e-6.
    X, A = gaussian_problem(dims, R, seed=19)
    QR = [oracle.qr(a) for a in A]
    h = gpu_handle(dims, R, X, precision="f32")
    h.set_factor_qr([q for q, _ in QR], [r for _, r in QR])
    for n in range(len(dims)):
        Y, _ = h.multi_ttm(n)
        assert rel(Y, oracle.multi_ttm(X, dims, n, [q for q, _ in QR])) <= 2e-6


# the FP32 TTMs with L % 4 == 0 run through the TMA-fed CUDA-core pipeline:
# boxes of 128 rows (BL = 128, or BL = L < 128 with 128 / L t slices),
# ragged row tiles and K chunks of 64, Q resident in shared memory or streamed
# per chunk (K = 400 at R = 64), and every column width up to 64.  Each output
# is summed in order of k; the row kernels do the same within a K split and
# add the splits in a fixed order, so the two paths differ by FP32 rounding
# only (the integer-valued cases of test_multi_ttm_index_bookkeeping_bit_exact
# pin both exactly)
@pytest.mark.parametrize("dims,R", [((64, 40, 36), 20), ((128, 30, 20, 12), 12), ((12, 70, 66), 9),
                                    ((68, 64, 66), 64), ((36, 400, 44), 33), ((52, 50, 49), 48)])
def test_f32_pipeline_matches_row_kernels(cuda_lib, dims, R):
    X, A = gaussian_problem(dims, R, seed=23)
    QR = [oracle.qr(a) for a in A]
    hs = []
    for pipe in (True, False):
        h = gpu_handle(dims, R, X, precision="f32")
        h.set_f32_pipeline(pipe)
        h.set_factor_qr([q for q, _ in QR], [r for _, r in QR])
        hs.append(h)
    for n in range(len(dims)):
        Y1, _ = hs[0].multi_ttm(n)
        Y0, _ = hs[1].multi_ttm(n)
        assert rel(Y1, Y0) <= 1e-6
        assert rel(Y1, oracle.multi_ttm(X, dims, n, [q for q, _ in QR])) <= 2e-6
    for h in hs:
        h.set_factors(A)
    f1 = hs[0].iterate(3, solve="qr")
    f0 = hs[1].iterate(3, solve="qr")
    assert np.abs(f1 - f0).max() <= 1e-6


def test_full_size_multi_ttm_c2(cuda_lib):
    # 400^3 FP64 rank 10 (the benchmark configuration), same launch path:
    # full parity of Y_(n) for every mode against the oracle
    p = inputs.workload_c2()
    QR = [oracle.qr(a) for a in p.init_factors]
    h = gpu_handle(p.dims, p.rank, p.X)
    h.set_factor_qr([q for q, _ in QR], [r for _, r in QR])
    for n in range(3):
        Y, _ = h.multi_ttm(n)
        ref = oracle.multi_ttm(p.X, p.dims, n, [q for q, _ in QR])
        assert rel(Y, ref) <= 1e-12


def test_full_size_sweep_c2(cuda_lib):
    # one full QR sweep at 400^3 rank 10 from the same start: factors and fit
    p = inputs.workload_c2()
    o = oracle.OracleCPALS(p.X, p.dims, p.rank)
    o.set_factors(p.init_factors)
    o.iterate(1, solve=oracle.QR)
    h = gpu_handle(p.dims, p.rank, p.X, p.init_factors)
    fits = h.iterate(1, solve="qr")
    assert abs(fits[0] - o.fit_last()) <= 1e-10
    Ag, lam = h.get_factors()
    for m in range(3):
        assert rel(Ag[m], o.factor(m)) <= 1e-9


# ---------------------------------------------------------------- tensor cores (BF16X3, TF32X3)
# shapes cover the 128-bit load path (L % 4 == 0: (40,30,20) mode 0, (64,48,40),
# (36,36,36,36)) and the scalar path (L = 1 fibers, odd L such as (70,45,33))
# The persistent TMA pipeline takes every first TTM whose row stride L (the
# product of the dims before the contracted mode) is a multiple of 4: here
# L = 40, 64 (row tiles of several t slices), 300, 46656, 1296 (ragged
# 128-row tiles, more tiles than SMs), 2400 with K = 150 (several ragged
# K-chunks at R = 48), the increasing dims (16, 20, 24, 28) (every mode), and
# L = 4096 with K = 300 at R = 64, whose Q tiles (80 KB in bf16, 160 KB in
# tf32) stream through the operand slots instead of staying resident.
TC_SHAPES = [((40, 30, 20), 16), ((300, 20), 16), ((20, 18, 17, 16), 16), ((70, 45, 33), 20), ((129, 64, 40), 32),
             ((64, 48, 40), 32), ((36, 36, 36, 36), 16), ((66, 65, 64), 64), ((48, 50, 150), 48),
             ((16, 20, 24, 28), 16), ((64, 64, 300), 64)]
# relative error per split product: ~2^-16 with bf16 parts, ~2^-21 with tf32 parts;
# over a contraction of length K the relative Frobenius error stays below
# 2 * u * sqrt(K_max) (K_max = the largest contracted dim)
TC_U = {"bf16x3": 2.0 ** -16, "tf32x3": 2.0 ** -21}


@pytest.mark.parametrize("pipeline", [True, False])
@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3"])
@pytest.mark.parametrize("dims,R", TC_SHAPES)
def test_split_tc_index_bookkeeping_bit_exact(cuda_lib, dims, R, precision, pipeline):
    # integers |x| <= 48 are exact in bf16 and tf32 (lo parts are zero) and 0/1
    # factors keep every product and partial sum exact in FP32, so the
    # tensor-core path must agree bit for bit with the oracle; a wrong operand
    # layout cannot pass
    P = int(np.prod(dims))
    X = (np.arange(P) * 37 % 97 - 48).astype(np.float64)
    rng = np.random.default_rng(R + len(dims))
    Q = [np.asfortranarray((rng.random((d, R)) < 0.5).astype(np.float64)) for d in dims]
    Rm = [np.asfortranarray(np.triu(np.ones((R, R)))) for _ in dims]
    h = gpu_handle(dims, R, X, precision=precision)
    h.set_tc_pipeline(pipeline)
    h.set_factor_qr(Q, Rm)
    for n in range(len(dims)):
        Y, _ = h.multi_ttm(n)
        np.testing.assert_array_equal(Y, oracle.multi_ttm(X, dims, n, Q))


@pytest.mark.parametrize("pipeline", [True, False])
@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3"])
@pytest.mark.parametrize("dims,R", TC_SHAPES)
def test_split_tc_multi_ttm_error_bound(cuda_lib, dims, R, precision, pipeline):
    # hi*hi + hi*lo + lo*hi drops lo*lo and rounds the lo parts
    X, A = gaussian_problem(dims, R, seed=23)
    QR = [oracle.qr(a) for a in A]
    h = gpu_handle(dims, R, X, precision=precision)
    h.set_tc_pipeline(pipeline)
    h.set_factor_qr([q for q, _ in QR], [r for _, r in QR])
    tol = 2.0 * TC_U[precision] * np.sqrt(max(dims))
    for n in range(len(dims)):
        Y, _ = h.multi_ttm(n)
        err = rel(Y, oracle.multi_ttm(X, dims, n, [q for q, _ in QR]))
        assert err <= tol, (n, err, tol)


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3"])
def test_split_tc_sweeps_track_oracle(cuda_lib, precision):
    # dimension-tree sweeps whose passes over X run on the tensor cores: the
    # first pass contracts mode 3 (L = 48*52*56), the second mode 1 (L = 48,
    # two t slices per row tile); fit per sweep against the FP64 oracle, and
    # the persistent pipeline against the per-tile kernel
    p = inputs.planted((48, 52, 56, 60), 16, seed=5, init_seed=6, noise=0.01)
    o = oracle.OracleCPALS(p.X, p.dims, p.rank)
    o.set_factors(p.init_factors)
    _, ofits = o.iterate(4, solve=oracle.QR)
    fits = {}
    for pipeline in (True, False):
        h = gpu_handle(p.dims, p.rank, p.X, p.init_factors, precision=precision)
        h.set_tc_pipeline(pipeline)
        fits[pipeline] = np.asarray(h.iterate(4, solve="qr"))
    tol = 1e-4 if precision == "bf16x3" else 1e-5
    assert np.abs(fits[True] - np.asarray(ofits)).max() <= tol, (fits[True], ofits)
    assert np.abs(fits[True] - fits[False]).max() <= tol / 10


def test_mixed_precisions_recover_planted_factors_like_fp64(cuda_lib):
    # the mixed precisions (FP32, and 3 x bf16 / 3 x tf32 on the tensor cores at
    # rank 16) recover the planted model as FP64 does: factor-match score
    # (Sec. 4.2) against the planted factors within 1e-3 of FP64's
    from paper_2112_10855_gb300.score import factor_match_score
    p = inputs.planted((64, 60, 56), 16, seed=41, init_seed=42, congruence=0.5, noise=0.01)
    Xd = torch.from_numpy(p.X).cuda()
    scores = {}
    for prec in ["f64", "f32", "bf16x3", "tf32x3"]:
        h = cpals.CPALS(p.dims, p.rank, prec)
        h.set_tensor(Xd)
        h.set_factors([np.asfortranarray(a) for a in p.init_factors])
        h.iterate(150, tol=1e-10, solve="qr")
        A, lam = h.get_factors()
        scores[prec] = factor_match_score(lam, A, p.true_weights, p.true_factors)
    assert scores["f64"] >= 0.95, scores
    for prec in ["f32", "bf16x3", "tf32x3"]:
        assert abs(scores[prec] - scores["f64"]) <= 1e-3, scores


@pytest.mark.parametrize("precision", ["f32", "bf16x3", "tf32x3"])
def test_mixed_mttkrp_error_bound(cuda_lib, precision):
    # the MTTKRP of the normal equations with FP32 passes over X; at rank 16
    # its first contraction runs on the tensor cores (split products)
    dims, R = (40, 36, 32), 16
    X, A = gaussian_problem(dims, R, seed=19)
    h = gpu_handle(dims, R, X, A, precision=precision)
    u = {"f32": 2.0 ** -24, **TC_U}[precision]
    tol = 2.0 * u * np.sqrt(max(dims)) + 4.0 * 2.0 ** -24 * np.sqrt(max(dims))
    for n in range(len(dims)):
        err = rel(h.mttkrp(n), oracle.mttkrp(X, dims, n, A))
        assert err <= tol, (n, err, tol)


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3"])
def test_full_size_tensor_core_multi_ttm_sampled_rows(cuda_lib, precision):
    # the 1000^3 rank-64 workload's size and launch configuration: the
    # persistent TMA pipeline over 7813 row tiles with Q tiles streamed
    # through the operand ring (K = 1000); rows of Y_(0) (1000 x 4096) against
    # Q_1^T X_i Q_2 in FP64 from the sampled slices of X, under the split
    # products' error bound
    n = 1000
    R = 64
    g = torch.Generator(device="cuda").manual_seed(7)
    X = torch.randn(n * n * n, dtype=torch.float64, device="cuda", generator=g)
    rng = np.random.default_rng(8)
    A = [np.asfortranarray(rng.standard_normal((n, R))) for _ in range(3)]
    h = cpals.CPALS((n, n, n), R, precision)
    h.set_tensor(X)
    h.set_factors(A)
    Y, _ = h.multi_ttm(0)
    Q = [h.get_factor_qr(m)[0] for m in range(3)]
    X3 = X.view(n, n, n)                  # [i2][i1][i0]: mode 0 fastest
    tol = 2.0 * TC_U[precision] * np.sqrt(n) + 4.0 * 2.0 ** -24 * np.sqrt(n)
    for i in (0, 1, 517, 998, 999):
        Xi = X3[:, :, i].cpu().numpy().T  # (i1, i2)
        ref = Q[1].T @ Xi @ Q[2]          # (r1, r2); Y_(0) column r1 + R r2
        got = Y[i].reshape((R, R), order="F")
        assert rel(got, ref) <= tol, (i, rel(got, ref), tol)
    del X, X3


@pytest.mark.parametrize("precision", ["bf16x3", "f32"])
def test_full_size_mixed_multi_ttm_c3(cuda_lib, precision):
    # the 4-way 120^4 rank-20 workload at full size: one Multi-TTM per mode
    # against the FP64 oracle with the same Q_m
    p = inputs.workload_c3()
    Q = [oracle.qr(a)[0] for a in p.init_factors]
    h = gpu_handle(p.dims, p.rank, p.X, precision=precision)
    h.set_factor_qr(Q, [oracle.qr(a)[1] for a in p.init_factors])
    u = {"f32": 2.0 ** -24, **TC_U}[precision]
    tol = 2.0 * u * np.sqrt(120) + 4.0 * 2.0 ** -24 * np.sqrt(120)
    for n in (0, 3):
        Y, _ = h.multi_ttm(n)
        err = rel(Y, oracle.multi_ttm(p.X, p.dims, n, Q))
        assert err <= tol, (n, err, tol)


@pytest.mark.parametrize("solve", ["svd", "normal_pinv"])
def test_truncated_solves_at_rank_40_match_oracle(cuda_lib, solve):
    # rank >= 32 takes the FP32-preconditioned Jacobi SVD; with columns 38
    # and 39 equal in every factor, R0 (and S) lose one rank exactly and the
    # truncated solve must match the oracle's minimum-norm update
    dims, R = (45, 44, 43), 40
    X, A = gaussian_problem(dims, R, seed=29)
    for m in range(3):
        A[m][:, 39] = A[m][:, 38]
    h = gpu_handle(dims, R, X, A)
    h.solve_mode(0, solve, 1e-10)
    h.sync()
    Ag, lam = h.get_factors()
    o = oracle.OracleCPALS(X, dims, R)
    o.set_factors(A)
    o.update_mode(0, OSOLVE[solve], 1e-10)
    assert rel(Ag[0] * lam[None, :], o.factor(0) * o.lam()[None, :]) <= 1e-8
