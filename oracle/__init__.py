"""FP64 CPU oracle for CP-ALS-QR (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
binding) never imports it and never falls back to it.

The arithmetic lives in ``cpals_oracle.c`` (plain C, FP64).  This module
compiles it with gcc and exposes numpy-friendly wrappers.
"""
from .oracle import (  # noqa: F401
    build, lib, qr, krp, unfold, ttm, ttm_order, multi_ttm, trsm_qr, jacobi_svd, svd_solve,
    normalize, mttkrp, cholesky_solve, residual_direct, fit_efficient_qr, score, OracleCPALS,
    use_library, compile_variant, source_text,
    QR, SVD, NORMAL, NORMAL_PINV,
)
