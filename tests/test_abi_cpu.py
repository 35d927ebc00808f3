"""CPU-only checks of the boundary: the C-ABI library builds for sm_103a, loads,
exports every entry point declared in include/cpals.h, and rejects bad
arguments before touching the GPU.  Without the library, or without a GPU,
the binding raises: there is no host fallback.  Also pins the seeded input
generator."""
import ctypes as C
import re

import numpy as np
import pytest

from paper_2112_10855_gb300 import _build, cpals, inputs


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return cpals.load()


def test_header_declares_the_boundary():
    names = cpals.exported_symbols()
    for required in ["cpals_create", "cpals_set_factors", "cpals_multi_ttm", "cpals_solve_mode",
                     "cpals_iterate", "cpals_fit", "cpals_krp_qr", "cpals_mttkrp", "cpals_set_tensor",
                     "cpals_destroy", "cpals_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in cpals.exported_symbols():
        assert hasattr(lib, name), f"{name} declared in include/cpals.h but not exported"


def test_exports_are_c_symbols():
    # the shared object exports unmangled names (extern "C")
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (cpals_[a-z0-9_]+)\b", out))
    assert set(cpals.exported_symbols()) <= exported


@pytest.mark.parametrize("dims,N,rank,prec", [
    ((10, 10, 10), 1, 3, 0),        # N < 2
    ((10, 10, 10), 3, 0, 0),        # rank 0
    ((10, 10, 10), 3, 65, 0),       # rank above the maximum
    ((10, 0, 10), 3, 2, 0),         # empty mode
    ((10, 4, 10), 3, 5, 0),         # rank above a dim
    ((10, 10, 10), 3, 3, 7),        # unknown precision
    ((3,) * 13, 13, 2, 0),          # N above the maximum
    ((64,) * 8, 8, 64, 0),          # R^N above what a dense handle holds
])
def test_create_rejects_bad_arguments_on_the_host(lib, dims, N, rank, prec):
    d = (C.c_int64 * len(dims))(*dims)
    h = C.c_void_p()
    rc = lib.cpals_create(d, N, rank, prec, C.byref(h))
    assert rc == cpals.ERR_ARG
    assert not h.value
    assert lib.cpals_last_error(None)


@pytest.mark.parametrize("dims,N,rank,S", [
    ((10, 10, 10), 3, 3, 0),        # Kruskal rank 0
    ((10, 10, 10), 3, 3, 5000),     # Kruskal rank above the maximum
    ((10, 4, 10), 3, 5, 3),         # rank above a dim
    ((3,) * 13, 13, 2, 2),          # N above the maximum
])
def test_create_kruskal_rejects_bad_arguments_on_the_host(lib, dims, N, rank, S):
    d = (C.c_int64 * len(dims))(*dims)
    h = C.c_void_p()
    rc = lib.cpals_create_kruskal(d, N, rank, S, C.byref(h))
    assert rc == cpals.ERR_ARG
    assert not h.value


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.cpals_set_stream(None, None) == cpals.ERR_ARG
    assert lib.cpals_solve_mode(None, 0, 0, 0.0) == cpals.ERR_ARG
    assert lib.cpals_destroy(None) == cpals.OK
    assert lib.cpals_launch_count(None) == -1


def test_options_match_the_header(lib):
    # the binding's option setters pass the enum values include/cpals.h declares
    import inspect
    import os
    hdr = open(os.path.join(_build.ROOT, "include", "cpals.h")).read()
    enum = dict((k, int(v)) for k, v in re.findall(r"(CPALS_OPT_[A-Z0-9_]+)\s*=\s*(\d+)", hdr))
    assert enum == {"CPALS_OPT_DIMTREE": 0, "CPALS_OPT_TC_PIPELINE": 1, "CPALS_OPT_KRP_TREE": 2,
                    "CPALS_OPT_F32_PIPELINE": 3, "CPALS_OPT_TEST_WITHHOLD_COPIES": 4,
                    "CPALS_OPT_FUSED_TAIL": 5, "CPALS_OPT_SVD_SHORTCUT": 6,
                    "CPALS_OPT_APPLY_Q0_FP32": 7, "CPALS_OPT_WIDE_TAIL": 8}
    setters = {"set_dimtree": "CPALS_OPT_DIMTREE", "set_tc_pipeline": "CPALS_OPT_TC_PIPELINE",
               "set_krp_tree": "CPALS_OPT_KRP_TREE", "set_f32_pipeline": "CPALS_OPT_F32_PIPELINE",
               "set_test_withhold_copies": "CPALS_OPT_TEST_WITHHOLD_COPIES",
               "set_fused_tail": "CPALS_OPT_FUSED_TAIL", "set_svd_shortcut": "CPALS_OPT_SVD_SHORTCUT",
               "set_apply_q0_fp32": "CPALS_OPT_APPLY_Q0_FP32", "set_wide_tail": "CPALS_OPT_WIDE_TAIL"}
    for name, opt in setters.items():
        src = inspect.getsource(getattr(cpals.CPALS, name))
        m = re.search(r"cpals_set_option\(self\._h, (\d+),", src)
        assert m and int(m.group(1)) == enum[opt], name
    # a null handle is rejected before the option is looked at
    for opt in enum.values():
        assert lib.cpals_set_option(None, opt, 1) == cpals.ERR_ARG


def test_splitmix64_matches_published_definition():
    # SplitMix64 seeded with 0: the first output is 0xE220A8397B1DCDAF
    z = inputs._mix64(np.array([0x9E3779B97F4A7C15], dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF


def test_generator_is_seeded_and_shaped():
    a = inputs.normal(5, 1, 1000)
    b = inputs.normal(5, 1, 1000)
    c = inputs.normal(6, 1, 1000)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)
    assert abs(a.mean()) < 0.15 and abs(a.std() - 1.0) < 0.1
    # chunked generation gives the same stream
    np.testing.assert_array_equal(inputs.normal(5, 1, 1000, chunk=97), a)


def test_collinear_generator_congruence():
    A = inputs.collinear_matrix(1, 2, 40, 6, 0.9)
    G = A.T @ A
    np.testing.assert_allclose(G, 0.1 * np.eye(6) + 0.9, atol=1e-13)


def test_planted_tensor_layout():
    p = inputs.planted((4, 3, 5), 2, noise=0.0)
    T = p.X.reshape((4, 3, 5), order="F")
    A = p.true_factors
    i, j, k = 3, 1, 4
    expect = sum(A[0][i, r] * A[1][j, r] * A[2][k, r] for r in range(2))
    assert abs(T[i, j, k] - expect) < 1e-13


def test_allocation_hook_rejects_negative_counts(lib):
    assert lib.cpals_test_fail_allocation(-1) == cpals.ERR_ARG
    assert lib.cpals_test_fail_allocation(0) == cpals.OK


def test_missing_library_raises(monkeypatch, tmp_path):
    monkeypatch.setattr(cpals, "_lib", None)
    with pytest.raises(RuntimeError, match="not found"):
        cpals.load(str(tmp_path / "libcpals.so"))


def test_no_host_fallback_without_a_gpu(lib):
    # valid arguments and no usable GPU: creation fails with the CUDA error
    # instead of computing anything on the host
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(cpals.CPALSError) as e:
        cpals.CPALS((4, 4, 4), 2, "f64")
    assert e.value.code == cpals.ERR_CUDA
    with pytest.raises(cpals.CPALSError) as e:
        cpals.CPALSBatch([(16, 16, 16)], [2])
    assert e.value.code == cpals.ERR_CUDA


def _static_call(lib, dims, N, rank, mode, null_q=None, null=None):
    d = (C.c_int64 * len(dims))(*dims)
    # non-null dummy addresses: every case here is rejected before any device access
    q = (C.c_void_p * len(dims))(*[0x1000 * (m + 1) for m in range(len(dims))])
    if null_q is not None:
        q[null_q] = None
    X, Y = C.c_void_p(0x100000), C.c_void_p(0x200000)
    args = {"dims": d, "X": X, "Q": q, "Y": Y}
    if null is not None:
        args[null] = None
    return lib.cpals_multi_ttm_static(args["dims"], N, rank, mode, args["X"], args["Q"], args["Y"], None)


@pytest.mark.parametrize("dims,N,rank,mode,null_q,null", [
    ((10, 10, 10), 1, 3, 0, None, None),         # N < 2
    ((3,) * 13, 13, 2, 0, None, None),           # N above the maximum
    ((10, 10, 10), 3, 0, 0, None, None),         # rank 0
    ((10, 10, 10), 3, 65, 0, None, None),        # rank above the maximum
    ((10, 10, 10), 3, 3, 3, None, None),         # mode out of range
    ((10, 10, 10), 3, 3, -1, None, None),        # negative mode
    ((10, 2, 10), 3, 3, 0, None, None),          # rank above a dim
    ((10, 10, 10), 3, 3, 0, 2, None),            # a Q_m the Multi-TTM needs is NULL
    ((10, 10, 10), 3, 3, 0, None, "X"),          # X NULL
    ((10, 10, 10), 3, 3, 0, None, "Y"),          # Y NULL
    ((10, 10, 10), 3, 3, 0, None, "Q"),          # Q array NULL
    ((10, 10, 10), 3, 3, 0, None, "dims"),       # dims NULL
    ((1 << 40, 1 << 30, 64), 3, 3, 2, None, None),   # prod(dims) overflows int64
])
def test_static_entry_rejects_bad_arguments_on_the_host(lib, dims, N, rank, mode, null_q, null):
    assert _static_call(lib, dims, N, rank, mode, null_q, null) == cpals.ERR_ARG
    assert lib.cpals_last_error(None)


@pytest.mark.parametrize("count,dims,ranks", [
    (0, [], []),                                  # no problems
    (1, [16, 16, 16], [0]),                       # rank 0
    (1, [16, 16, 16], [17]),                      # rank above the batched maximum
    (2, [16, 16, 16, 16, 3, 16], [4, 4]),         # a dim below the rank
    (1, [16, 5000, 16], [4]),                     # a dim above 4096
    (1, [4096, 4096, 4096], [16]),                # working set beyond one CTA's shared memory
])
def test_batch_create_rejects_bad_arguments_on_the_host(lib, count, dims, ranks):
    d = (C.c_int64 * max(len(dims), 1))(*dims)
    r = (C.c_int * max(len(ranks), 1))(*ranks)
    out = C.c_void_p()
    assert lib.cpals_batch_create(count, d, r, C.byref(out)) == cpals.ERR_ARG
    assert not out.value
    assert lib.cpals_last_error(None)
