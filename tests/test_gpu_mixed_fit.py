"""The mixed precisions reach the FP64 oracle's fit.

The passes over X read an FP32 copy of X (FP32 FMA, or 3 x bf16 / 3 x tf32
split products on the tensor cores at rank >= 16) while every small factor
stays FP64.  From the oracle's initial factors, each mixed-precision handle
runs as many sweeps as the FP64 oracle (which stops once the fit changes by
less than 1e-10, or after 300 sweeps) and its direct fit (Sec. 3.3.1, one
FP64 pass over the FP64 X) must lie within 1e-6 relative of the oracle's.
Near a fit stationary point a small change of the factors changes the fit
only to second order, so the FP32 rounding of X (2^-24 relative) leaves the
converged fit far inside that bar.  The factors after one sweep are also
checked against the oracle's, with a bound from the precision of the passes
over X (amplified by the conditioning of the update).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2112_10855_gb300 import cpals, inputs

pytestmark = pytest.mark.gpu

MAX_SWEEPS = 300
TOL = 1e-10
# C3-like problems (column congruence 0.9, 1% noise), reduced so that the
# oracle finishes its sweeps in well under a minute
PROBLEMS = {
    "3way_60x64x68_r16": dict(dims=(60, 64, 68), rank=16, seed=31, init_seed=32),
    "4way_28x28x28x28_r20": dict(dims=(28, 28, 28, 28), rank=20, seed=33, init_seed=34),
}
# relative Frobenius error of lambda-scaled factors after one sweep
ONE_SWEEP_TOL = {"f32": 1e-4, "bf16x3": 1e-3, "tf32x3": 1e-4}

_cache = {}


def oracle_run(name):
    if name not in _cache:
        cfg = PROBLEMS[name]
        p = inputs.planted(cfg["dims"], cfg["rank"], seed=cfg["seed"], init_seed=cfg["init_seed"],
                           congruence=0.9, noise=0.01)
        o = oracle.OracleCPALS(p.X, p.dims, p.rank)
        o.set_factors(p.init_factors)
        o.iterate(1, solve=oracle.QR)
        one = ([a.copy() for a in o.factors()], o.lam().copy())
        k, fits = o.iterate(MAX_SWEEPS - 1, tol=TOL, solve=oracle.QR)
        _cache[name] = dict(problem=p, sweeps=1 + abs(k), fit_direct=o.fit_direct(), fits=fits, one_sweep=one)
    return _cache[name]


def scaled(A, lam):
    return np.concatenate([a * lam[None, :] ** (1.0 / len(A)) for a in A])


@pytest.mark.parametrize("precision", ["f32", "bf16x3", "tf32x3"])
@pytest.mark.parametrize("name", sorted(PROBLEMS))
def test_mixed_converged_fit_matches_fp64_oracle(cuda_lib, name, precision):
    ref = oracle_run(name)
    p = ref["problem"]
    h = cpals.CPALS(p.dims, p.rank, precision)
    h.set_tensor(torch.from_numpy(p.X).cuda())
    h.set_factors([np.asfortranarray(a) for a in p.init_factors])

    # one sweep: factors against the oracle's
    h.iterate(1, solve="qr")
    A1, lam1 = h.get_factors()
    oA, olam = ref["one_sweep"]
    err1 = np.linalg.norm(scaled(A1, lam1) - scaled(oA, olam)) / np.linalg.norm(scaled(oA, olam))
    assert err1 <= ONE_SWEEP_TOL[precision], (name, precision, err1)

    # the oracle's sweep count in total, then the direct fit
    h.iterate(ref["sweeps"] - 1, solve="qr")
    fit = h.fit(direct=True)
    gap = abs(fit - ref["fit_direct"]) / ref["fit_direct"]
    assert gap <= 1e-6, (name, precision, fit, ref["fit_direct"], gap, ref["sweeps"])


@pytest.mark.parametrize("precision", ["f32", "bf16x3", "tf32x3"])
def test_w_in_fp32_matches_fp64_w_after_one_sweep(cuda_lib, precision):
    # W = Y_(n) Q0 formed in FP32 (the default for the mixed precisions)
    # against the same handle forming it in FP64 from the widened Y_(n).  The
    # FP32 sum over R^{N-1} = 8000 terms carries ~sqrt(8000) 2^-24 = 5e-6
    # relative error, which the solve amplifies by the conditioning of R0
    # (~10 for these factors): the factors after one sweep agree to 1e-4
    cfg = PROBLEMS["4way_28x28x28x28_r20"]
    p = inputs.planted(cfg["dims"], cfg["rank"], seed=cfg["seed"], init_seed=cfg["init_seed"], congruence=0.9,
                       noise=0.01)
    out = {}
    for fp32_w in (True, False):
        h = cpals.CPALS(p.dims, p.rank, precision)
        h.set_apply_q0_fp32(fp32_w)
        h.set_tensor(torch.from_numpy(p.X).cuda())
        h.set_factors([np.asfortranarray(a) for a in p.init_factors])
        h.iterate(1, solve="qr")
        out[fp32_w] = h.get_factors()
    (A1, l1), (A2, l2) = out[True], out[False]
    err = max(np.linalg.norm(a - b) / np.linalg.norm(b) for a, b in zip(A1, A2))
    assert err <= 1e-4, err
    assert np.linalg.norm(l1 - l2) / np.linalg.norm(l2) <= 1e-4
