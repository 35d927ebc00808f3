"""Seeded synthetic inputs for CP-ALS-QR workloads.

This module only draws random numbers and assembles the synthetic tensors the
paper's experiments describe (Sec. 4.1-4.2): planted CP tensors with Gaussian or
collinear factors, weights, Gaussian noise and random initial factors.  It
holds none of the method's arithmetic (no QR of Khatri-Rao products, no
Multi-TTM, no solves), so both the CUDA path and the CPU oracle can take their
inputs from it without sharing any computation.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based generator:
draw k of stream s is mix64(key(seed, s) + (k + 1) * GOLDEN).  Uniforms take the
top 53 bits, normals use the Box-Muller transform on pairs of uniforms.

Layout conventions (shared with the C-ABI): a tensor of dims (I_1..I_N) is a
flat float64 array with mode 1 fastest, element (i_1..i_N) at
sum_m i_m * prod_{k<m} I_k; matrices are column-major (numpy order='F').
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    base = np.array([(seed * 0xD1B54A32D192ED03 + stream * 0x9E3779B97F4A7C15 + 1) & _MASK],
                    dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(base)[0]


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniforms in (0, 1) from draws offset..offset+n-1 of (seed, stream)."""
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix64(_key(seed, stream) + k * _GOLDEN)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int, chunk: int = 1 << 22) -> np.ndarray:
    """n i.i.d. N(0,1) draws: Box-Muller on uniform pairs (2k, 2k+1).

    Chunks are filled by a thread pool (numpy releases the GIL); each chunk
    writes its own slice, so the result does not depend on the thread count.
    """
    out = np.empty(n, dtype=np.float64)

    def fill(s):
        m = min(chunk, n - s)
        u = uniform(seed, stream, 2 * m, offset=2 * s)
        out[s:s + m] = np.sqrt(-2.0 * np.log(u[0::2])) * np.cos(2.0 * math.pi * u[1::2])

    starts = list(range(0, n, chunk))
    if len(starts) <= 1:
        for s in starts:
            fill(s)
    else:
        import concurrent.futures as cf
        import os
        with cf.ThreadPoolExecutor(max_workers=min(len(starts), os.cpu_count() or 1)) as ex:
            list(ex.map(fill, starts))
    return out


def randint(seed: int, stream: int, n: int, lo: int, hi: int) -> np.ndarray:
    """n integers uniform on {lo..hi} (inclusive)."""
    u = uniform(seed, stream, n)
    return lo + np.minimum((u * (hi - lo + 1)).astype(np.int64), hi - lo)


def gaussian_matrix(seed: int, stream: int, rows: int, cols: int) -> np.ndarray:
    return normal(seed, stream, rows * cols).reshape((rows, cols), order="F")


def collinear_matrix(seed: int, stream: int, rows: int, cols: int, congruence: float) -> np.ndarray:
    """rows x cols matrix with unit columns of pairwise congruence c.

    C = (1-c) I + c 11^T = L L^T, A = Q L^T with Q the orthonormal factor of a
    Gaussian matrix, so A^T A = C (the collinearity recipe the paper borrows for
    its Sec. 4.2 experiment, which it cites but does not spell out).
    """
    if rows < cols:
        raise ValueError("collinear factors need rows >= cols")
    c = float(congruence)
    C = (1.0 - c) * np.eye(cols) + c * np.ones((cols, cols))
    L = np.linalg.cholesky(C)
    G = gaussian_matrix(seed, stream, rows, cols)
    Q, _ = np.linalg.qr(G)
    return np.asfortranarray(Q @ L.T)


def cp_full(dims, factors, weights) -> np.ndarray:
    """Dense tensor sum_r w_r a_r^(1) o ... o a_r^(N), flat with mode 1 fastest."""
    N = len(dims)
    R = factors[0].shape[1]
    # columns of the Kronecker chain a^(N) (x) ... (x) a^(2), built with einsum
    tail = np.ones((1, R))
    for m in range(1, N):
        a = factors[m]
        tail = np.einsum("jr,ir->jir", a, tail).reshape(-1, R)   # new (slower) index outermost
    head = factors[0] * np.asarray(weights)[None, :]
    return np.ascontiguousarray((head @ tail.T).reshape(-1, order="F"))


@dataclass
class Problem:
    dims: tuple
    rank: int
    X: np.ndarray                     # flat float64, mode 1 fastest
    true_factors: list
    true_weights: np.ndarray
    init_factors: list = field(default_factory=list)
    meta: dict = field(default_factory=dict)


def planted(dims, rank, *, seed=2112, init_seed=10855, congruence=0.0, unit_columns=False,
            weights=None, noise=0.01, init_rank=None) -> Problem:
    """Planted CP tensor plus Gaussian noise scaled to `noise` * ||X_true||_F.

    congruence == 0 draws factor entries i.i.d. N(0,1) (unless unit_columns);
    congruence > 0 uses collinear_matrix.  weights: None -> ones, or an array.
    Initial factors (for modes 2..N; mode 1 is solved first) are i.i.d. N(0,1)
    from init_seed, with rank init_rank (default: rank).
    """
    dims = tuple(int(d) for d in dims)
    N = len(dims)
    facs = []
    for m in range(N):
        if congruence > 0.0:
            facs.append(collinear_matrix(seed, 100 + m, dims[m], rank, congruence))
        else:
            A = gaussian_matrix(seed, 100 + m, dims[m], rank)
            if unit_columns:
                A = A / np.linalg.norm(A, axis=0, keepdims=True)
            facs.append(np.asfortranarray(A))
    w = np.ones(rank) if weights is None else np.asarray(weights, dtype=np.float64)
    X = cp_full(dims, facs, w)
    if noise > 0.0:
        E = normal(seed, 7, X.size)
        X += noise * np.linalg.norm(X) / np.linalg.norm(E) * E
        del E
    R0 = rank if init_rank is None else int(init_rank)
    init = [gaussian_matrix(init_seed, 200 + m, dims[m], R0) for m in range(N)]
    return Problem(dims, R0, X, facs, w, init,
                   {"seed": seed, "init_seed": init_seed, "congruence": congruence,
                    "noise": noise, "true_rank": rank})


def logspace_weights(rank: int, wmin: float) -> np.ndarray:
    return np.logspace(0.0, math.log10(wmin), rank)


# Workload recipes (sizes, distributions) of the synthetic benchmark tensors.
def workload_c1(seed=2112, init_seed=10855, size=50, rank=5, noise=0.01):
    """3-way size^3, rank 5, N(0,1) factors, unit weights, 1% noise."""
    return planted((size,) * 3, rank, seed=seed, init_seed=init_seed, noise=noise)


def workload_c2(seed=2112, init_seed=10855, size=400, rank=10):
    """3-way size^3, rank 10, congruence 0.99, weights logspace 1..1e-4, 0.1% noise."""
    return planted((size,) * 3, rank, seed=seed, init_seed=init_seed, congruence=0.99,
                   weights=logspace_weights(rank, 1e-4), noise=1e-3)


def workload_c3(seed=2112, init_seed=10855, size=120, rank=20):
    """4-way size^4, rank 20, congruence 0.9, 1% noise."""
    return planted((size,) * 4, rank, seed=seed, init_seed=init_seed, congruence=0.9,
                   noise=0.01)


def workload_c5a(seed=2112, init_seed=10855, size=1000, rank=64, noise=1e-3):
    """3-way size^3, rank 64, congruence 0.999, weights logspace 1..1e-6, 0.1% noise."""
    return planted((size,) * 3, rank, seed=seed, init_seed=init_seed, congruence=0.999,
                   weights=logspace_weights(rank, 1e-6), noise=noise)


def sine_grid(n: int) -> np.ndarray:
    """n points 2 pi k / n, k = 0..n-1, on [0, 2 pi) (the discretisation of Sec. 4.3)."""
    return 2.0 * math.pi * np.arange(n) / n


def sine_of_sums_expanded(N: int, n: int):
    """sin(x_1 + ... + x_N) on the grid as a Kruskal tensor of rank 2^{N-1}.

    Expanding with sin(a + b) = sin a cos b + cos a sin b mode by mode leaves
    one term per subset T of the modes with |T| odd: prod_{j in T} sin(x_j)
    prod_{j not in T} cos(x_j), with sign (-1)^{(|T|-1)/2}.  Returns (mu, V):
    weights (2^{N-1},) and N factor matrices (n x 2^{N-1}, column-major).
    """
    x = sine_grid(n)
    terms = [t for t in range(1 << N) if bin(t).count("1") % 2 == 1]
    S = len(terms)
    mu = np.array([(-1.0) ** ((bin(t).count("1") - 1) // 2) for t in terms])
    V = []
    for j in range(N):
        Vj = np.empty((n, S), order="F")
        for c, t in enumerate(terms):
            Vj[:, c] = np.sin(x) if (t >> j) & 1 else np.cos(x)
        V.append(Vj)
    return mu, V


def sine_of_sums_rank_n(N: int, n: int, alpha=None):
    """sin(x_1 + ... + x_N) on the grid as the rank-N Kruskal tensor of Eq.
    sinsum_rkd: term j has sin(x_j) in mode j and
    sin(x_k + alpha_k - alpha_j) / sin(alpha_k - alpha_j) in every mode k != j.
    alpha defaults to alpha_j = j pi / N (every difference a non-multiple of pi).
    Returns (mu = ones, V)."""
    x = sine_grid(n)
    a = np.arange(N) * math.pi / N if alpha is None else np.asarray(alpha, dtype=np.float64)
    V = []
    for k in range(N):
        Vk = np.empty((n, N), order="F")
        for j in range(N):
            Vk[:, j] = np.sin(x) if k == j else np.sin(x + a[k] - a[j]) / math.sin(a[k] - a[j])
        V.append(Vk)
    return np.ones(N), V


def random_kruskal(dims, S, seed=2112, stream=300):
    """A Kruskal tensor with N(0,1) factors (I_m x S) and weights U(0.5, 1.5)."""
    V = [gaussian_matrix(seed, stream + m, d, S) for m, d in enumerate(dims)]
    mu = 0.5 + uniform(seed, stream + 99, S)
    return mu, [np.asfortranarray(v) for v in V]


def batch_shapes(count=512, seed=2112, lo=16, hi=128, rlo=2, rhi=16, order=3):
    """Per-problem dims ~ U{lo..hi} and ranks ~ U{rlo..rhi} for the batched workload."""
    dims = randint(seed, 11, count * order, lo, hi).reshape(count, order)
    ranks = randint(seed, 12, count, rlo, rhi)
    return dims, ranks
