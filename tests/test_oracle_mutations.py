"""Planted mistakes in the oracle must fail a pin.

Each case compiles a copy of the C oracle with one plausible mistake (a dropped
term, a wrong sign or index, a transposed operand), on the CPU, and checks
that at least one pin of tests/test_oracle_pins.py fails against that copy.
Every planted mistake keeps its memory accesses in bounds.
"""
import numpy as np
import pytest

import oracle
from tests import test_oracle_pins as P

MUTATIONS = {
    "krp_kron_order": ("nxt[K * i + kk] = cur[i] * mats[k][kk + K * r];",
                       "nxt[i + len * kk] = cur[i] * mats[k][kk + K * r];"),
    "ttm_transposed_U": ("s += X[l + L * (k + K * t)] * U[j + J * k];",
                         "s += X[l + L * (k + K * t)] * U[k + K * j];"),
    "unfold_row_major": ("Xn[idx[n] + dims[n] * col] = X[lin];",
                         "Xn[idx[n] * (P / dims[n]) + col] = X[lin];"),
    "trsm_sign": ("for (int64_t j = k + 1; j < R; ++j) s -= R0[k + R * j] * x[j];",
                  "for (int64_t j = k + 1; j < R; ++j) s += R0[k + R * j] * x[j];"),
    "trsm_transposed_R0": ("for (int64_t j = k + 1; j < R; ++j) s -= R0[k + R * j] * x[j];",
                           "for (int64_t j = k + 1; j < R; ++j) s -= R0[j + R * k] * x[j];"),
    "qr_no_sign_fix": ("if (R[j + n * j] < 0.0) {", "if (0) {"),
    "fit_dropped_model_norm": ("double res2 = normX2 - 2.0 * inner + nrm;\n    if (res2 < 0.0) res2 = 0.0;\n    return 1.0 - sqrt(res2) / sqrt(normX2);\n}\n\n/* Efficient CP-ALS error",
                               "double res2 = normX2 - 2.0 * inner;\n    if (res2 < 0.0) res2 = 0.0;\n    return 1.0 - sqrt(res2) / sqrt(normX2);\n}\n\n/* Efficient CP-ALS error"),
    "jacobi_rotation_sign": ("B[i + n * p] = c * bp - s * bq;", "B[i + n * p] = c * bp + s * bq;"),
    "normalize_no_sqrt": ("double l = sqrt(s);", "double l = s;"),
    "mttkrp_includes_mode_n": ("if (m != n) p *= A[m][idx[m] + dims[m] * r];",
                               "p *= A[m][idx[m] + dims[m] * r];"),
    "cholesky_transposed_L": ("for (int64_t j = k + 1; j < R; ++j) s -= L[j + R * k] * Ahat[i + I * j];",
                              "for (int64_t j = k + 1; j < R; ++j) s -= L[k + R * j] * Ahat[i + I * j];"),
    "krp_qr_ascending_modes": ("for (int m = st->N - 1; m >= 0; --m)\n        if (m != n) { mats[cnt]",
                               "for (int m = 0; m < st->N; ++m)\n        if (m != n) { mats[cnt]"),
    "ttm_order_ties_low_mode": ("(dims[y] == dims[x] && y > x)", "(dims[y] == dims[x] && y < x)"),
    "apply_q0_skipped_in_update": ("orc_matmul(In, RN1, R, st->Y, st->Q0, st->W);",
                                   "orc_matmul(In, R, R, st->Y, st->R0, st->W);"),
    "factor_qr_left_stale": ("orc_qr(In, R, st->A[n], st->Q[n], st->Rf[n]);",
                             "/* factor QR not refreshed */"),
    "svd_no_truncation": ("int keep = S[j] > rtol * S[0] && S[j] > 0.0;", "int keep = S[j] > 0.0;"),
    "svd_U_in_place_of_V": ("for (int64_t j = 0; j < R; ++j) s += WU[i + I * j] * V[k + R * j];",
                            "for (int64_t j = 0; j < R; ++j) s += WU[i + I * j] * U[k + R * j];"),
    "hadamard_gram_summed": ("for (int64_t k = 0; k < R * R; ++k) st->S[k] *= st->G[m][k];",
                             "for (int64_t k = 0; k < R * R; ++k) st->S[k] += st->G[m][k];"),
    "direct_residual_drops_lambda": ("double p = lambda[r];", "double p = 1.0;"),
    "fit_qr_R0_not_transposed": ("for (int64_t j = 0; j < R; ++j) s += AhatN[i + IN * j] * R0[k + R * j];",
                                 "for (int64_t j = 0; j < R; ++j) s += AhatN[i + IN * j] * R0[j + R * k];"),
    "fit_normal_drops_one_lambda": ("nrm += SN[a + R * b] * lambda[a] * GN[a + R * b] * lambda[b];",
                                    "nrm += SN[a + R * b] * lambda[a] * GN[a + R * b];"),
    "lambda_accumulates_over_modes": ("        lambda[r] = l;\n", "        lambda[r] *= l;\n"),
    "score_keeps_sign": ("term *= (n1 > 0.0 && n2 > 0.0) ? fabs(d) / sqrt(n1 * n2) : 0.0;",
                         "term *= (n1 > 0.0 && n2 > 0.0) ? d / sqrt(n1 * n2) : 0.0;"),
    "score_identity_permutation_only": ("while (i < R) {", "while (0) {"),
    "qr_q_misses_reflector_column": ("for (int64_t k = j; k < n; ++k) {", "for (int64_t k = j + 1; k < n; ++k) {"),
    "singular_test_drops_rank_factor": ("if (!(fabs(R0[k + R * k]) > (double)R * 2.220446049250313e-16 * dmax)) return 1;",
                                        "if (!(fabs(R0[k + R * k]) > 2.220446049250313e-16 * dmax)) return 1;"),
}

PINS = [
    (P.test_qr_matches_lapack_with_sign_convention, (30, 10)),
    (P.test_krp_columnwise_kronecker, ([2, 3],)),
    (P.test_kr_identity, ()),
    (P.test_unfold_columns_are_fibers, ((2, 3, 4),)),
    (P.test_ttm_matches_tensordot, ((4, 5, 6), 1)),
    (P.test_multi_ttm_matches_explicit_kronecker, ((3, 4, 5), 2)),
    (P.test_multi_ttm_flop_count, ((6, 8, 5, 7), 2, 2)),
    (P.test_multi_ttm_flop_count, ((5, 5, 5, 4), 2, 3)),
    (P.test_structured_qr_of_khatri_rao, ((6, 5, 7), 3)),
    (P.test_qr_update_equals_lstsq_on_explicit_Z, ((6, 5, 7), 3)),
    (P.test_normal_update_equals_qr_update_well_conditioned, ()),
    (P.test_trsm_against_solve, ()),
    (P.test_jacobi_svd_against_lapack, ()),
    (P.test_cholesky_solve_against_numpy, ()),
    (P.test_normalize_two_norm, ()),
    (P.test_efficient_fit_matches_direct, ()),
    (P.test_sweeps_equal_alternating_lstsq, ((6, 5, 7), 3)),
    (P.test_svd_solve_truncation_matches_pinv, ()),
    (P.test_score_invariances, ()),
    (P.test_trsm_singularity_threshold, ()),
]


def _some_pin_fails():
    failed = []
    for fn, args in PINS:
        try:
            fn(*args)
        except (AssertionError, np.linalg.LinAlgError, ValueError, FloatingPointError, pytest.fail.Exception):
            failed.append(fn.__name__)
    return failed


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    before, after = MUTATIONS[name]
    src = oracle.source_text()
    assert src.count(before) == 1, f"mutation anchor for {name} not unique"
    so = oracle.compile_variant(src.replace(before, after), str(tmp_path / f"mut_{name}.so"))
    with oracle.use_library(so):
        failed = _some_pin_fails()
    assert failed, f"planted mistake {name} passed every pin"


def test_unmutated_oracle_passes_the_same_pins():
    assert _some_pin_fails() == []
