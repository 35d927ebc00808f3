"""Robustness on ill-conditioned problems (Sec. 4.2), on the GPU.

A 50^3 rank-5 tensor from unit-norm factors with pairwise column congruence
1 - 1e-7 and 1e-10 relative noise makes every Z_n nearly rank deficient.
The QR-based solves reach a small residual, and the normal equations (which
square the condition number) do no better: CP-ALS-PINV stays at or above the
QR solves, CP-ALS at or above them or loses positive definiteness.  The
handle factors well-conditioned matrices by CholeskyQR2 and falls back to
Householder when its check fails, so the QR solve must do as well with those
paths on as with Householder everywhere (CPALS_OPT_FUSED_TAIL = 0).
"""
import numpy as np
import pytest
import torch

from paper_2112_10855_gb300 import cpals, inputs

pytestmark = pytest.mark.gpu


def relerr(h):
    return 1.0 - h.fit(direct=True)


def run(p, solve, fused=True, sweeps=100):
    h = cpals.CPALS(p.dims, p.rank, "f64")
    h.set_fused_tail(fused)
    h.set_tensor(torch.from_numpy(p.X).cuda())
    h.set_factors([np.asfortranarray(a) for a in p.init_factors])
    try:
        h.iterate(sweeps, solve=solve)
    except cpals.SingularError:
        return None
    return relerr(h)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_qr_solves_beat_normal_equations_on_collinear_factors(cuda_lib, seed):
    p = inputs.planted((50, 50, 50), 5, seed=5000 + 97 * seed, init_seed=6000 + seed, congruence=1 - 1e-7,
                       unit_columns=True, noise=1e-10)
    e_qr = run(p, "qr")
    e_svd = run(p, "svd")
    e_pinv = run(p, "normal_pinv")
    e_ne = run(p, "normal")
    e_qr_hh = run(p, "qr", fused=False)
    vals = dict(qr=e_qr, svd=e_svd, pinv=e_pinv, normal=e_ne, qr_householder=e_qr_hh)
    assert e_qr is not None and e_svd is not None and e_qr_hh is not None, vals
    assert e_qr <= 1e-6 and e_svd <= 1e-6, vals
    # the CholeskyQR2 paths (with their fallbacks) lose nothing against Householder everywhere
    assert e_qr <= 2 * max(e_qr_hh, 1e-12), vals
    # the normal equations do no better than the QR solves (or fail outright)
    assert e_pinv is None or e_pinv >= 0.5 * e_qr, vals
    assert e_ne is None or e_ne >= 0.5 * e_qr, vals
