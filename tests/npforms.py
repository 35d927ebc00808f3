"""Explicit matrix forms written with numpy, used to pin the oracle.

These build the paper's objects in their matrix form (explicit Kronecker and
Khatri-Rao products, explicit unfoldings via numpy reshapes), which is a
different computation from the oracle's TTM sequences and loops.
"""
from functools import reduce

import numpy as np


def tensor(X, dims):
    return np.asarray(X).reshape(tuple(dims), order="F")


def unfold(X, dims, n):
    """X_(n): rows i_n, columns the other indices with the lowest mode fastest."""
    T = tensor(X, dims)
    return np.moveaxis(T, n, 0).reshape(dims[n], -1, order="F")


def kron_chain(mats):
    return reduce(np.kron, mats)


def khatri_rao(mats):
    R = mats[0].shape[1]
    return np.stack([kron_chain([m[:, r] for m in mats]) for r in range(R)], axis=1)


def others_desc(N, n):
    """Modes N..1 without n (0-based), the order of the Kronecker/KRP chains."""
    return [m for m in range(N - 1, -1, -1) if m != n]


def multi_ttm_explicit(X, dims, n, Q):
    """Y_(n) = X_(n) (Q_N (x) ... (x) Q_1), skipping n (Eq. multittm with U_m = Q_m^T)."""
    return unfold(X, dims, n) @ kron_chain([Q[m] for m in others_desc(len(dims), n)])


def Z(A, n):
    """Z_n = A_N (.) ... (.) A_1, skipping n (Eq. cp_mat)."""
    return khatri_rao([A[m] for m in others_desc(len(A), n)])


def full(lam, A):
    """Dense sum_r lambda_r a_r^(1) o ... o a_r^(N), flat, mode 1 fastest."""
    N = len(A)
    Xn = (A[0] * lam[None, :]) @ khatri_rao([A[m] for m in range(N - 1, 0, -1)]).T
    return Xn.reshape(-1, order="F")


def qr_pos(A):
    """numpy (LAPACK) thin QR with the diag(R) >= 0 convention."""
    Q, R = np.linalg.qr(A)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :], R * s[:, None]
