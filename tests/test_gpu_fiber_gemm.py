"""FP32 TTM over the contiguous mode (L = 1) above rank 16: the tiled GEMM
kernel (128 fibers x 32 or 64 columns per CTA, K in chunks of 32, K split
over CTAs when the fibers are few).

- Two-way tensors, whose mode-1 Multi-TTM is the single L = 1 contraction
  X x_0 Q_0^T. They use integer X and 0/1 Q, so every sum is an integer below
  2^24 and exact in FP32. The result must equal the oracle bit for bit, at
  ranks 17..64 (both column widths, padded and full), K with ragged 32-chunks,
  ragged 128-fiber tiles, and a single-CTA case that splits K.
- A Gaussian three-way tensor against the FP64 oracle, at the FP32 rounding
  level of a length-1000 sum.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2112_10855_gb300 import cpals

pytestmark = pytest.mark.gpu


def handle(dims, R, X, Q):
    h = cpals.CPALS(dims, R, "f32")
    h.set_tensor(torch.from_numpy(np.ascontiguousarray(X)).cuda())
    h.set_factor_qr(Q, [np.asfortranarray(np.triu(np.ones((R, R)))) for _ in dims])
    return h


@pytest.mark.parametrize("dims,R", [((1000, 600), 20), ((130, 9030), 64), ((96, 2000), 33), ((200, 4500), 17),
                                    ((64, 3300), 32), ((4000, 40), 40), ((1000, 64), 64), ((36, 1000), 24)])
def test_fiber_gemm_bit_exact(cuda_lib, dims, R):
    P = int(np.prod(dims))
    X = (np.arange(P) * 37 % 97 - 48).astype(np.float64)
    rng = np.random.default_rng(R + dims[0])
    Q = [np.asfortranarray((rng.random((d, R)) < 0.5).astype(np.float64)) for d in dims]
    h = handle(dims, R, X, Q)
    Y, _ = h.multi_ttm(1)
    np.testing.assert_array_equal(Y, oracle.multi_ttm(X, dims, 1, Q))


def test_fiber_gemm_gaussian_against_fp64(cuda_lib):
    dims, R = (1000, 30, 40), 20
    rng = np.random.default_rng(5)
    X = rng.standard_normal(int(np.prod(dims)))
    Q = [np.asfortranarray(np.linalg.qr(rng.standard_normal((d, R)))[0]) for d in dims]
    h = handle(dims, R, X, Q)
    for n in (1, 2):
        Y, _ = h.multi_ttm(n)
        ref = oracle.multi_ttm(X, dims, n, Q)
        assert np.linalg.norm(Y - ref) / np.linalg.norm(ref) <= 1e-5
