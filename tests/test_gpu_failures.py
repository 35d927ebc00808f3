"""Failure paths, made without faulting the GPU.

- A bounded device wait that runs out: the test hook
  CPALS_OPT_TEST_WITHHOLD_COPIES makes the persistent tensor-core pass over X
  issue no copies, so its consumers' waits (1 ms limit) give up with nothing
  in flight.  The pass records CPALS_ERR_TIMEOUT; the factors stay as they
  were; after the hook is cleared the same update gives the result an
  untouched handle gives.
- A device allocation that fails (host-side hook): cpals_create returns
  CPALS_ERR_NOMEM and frees what it held; the next create succeeds.
- NaN or Inf in X: cpals_set_tensor refuses the tensor.
"""
import numpy as np
import pytest
import torch

from paper_2112_10855_gb300 import cpals

pytestmark = pytest.mark.gpu

DIMS, R = (48, 52, 56), 16       # first pass over X: L = 48 * 52 (a multiple of 4) -> persistent pipeline


def problem(seed=3):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal(int(np.prod(DIMS)))
    A = [np.asfortranarray(rng.standard_normal((d, R))) for d in DIMS]
    return X, A


def handle(X, A, precision="bf16x3"):
    h = cpals.CPALS(DIMS, R, precision)
    h.set_tensor(torch.from_numpy(X).cuda())
    h.set_factors(A)
    return h


@pytest.mark.parametrize("precision", ["bf16x3", "tf32x3"])
def test_timed_out_wait_reports_timeout_and_keeps_factors(cuda_lib, precision):
    X, A = problem()
    h = handle(X, A, precision)
    A0, lam0 = h.get_factors()
    h.set_test_withhold_copies(True)
    h.solve_mode(0, "qr")
    with pytest.raises(cpals.CPALSError) as e:
        h.sync()
    assert e.value.code == cpals.ERR_TIMEOUT
    A1, lam1 = h.get_factors()
    for a0, a1 in zip(A0, A1):
        np.testing.assert_array_equal(a0, a1)
    np.testing.assert_array_equal(lam0, lam1)
    # a sweep (captured graph) with the hook set fails the same way
    with pytest.raises(cpals.CPALSError) as e:
        h.iterate(2, solve="qr")
    assert e.value.code == cpals.ERR_TIMEOUT
    for a0, a1 in zip(A0, h.get_factors()[0]):
        np.testing.assert_array_equal(a0, a1)
    # cleared: the handle works again and agrees with an untouched handle
    h.set_test_withhold_copies(False)
    h.solve_mode(0, "qr")
    h.sync()
    ref = handle(X, A, precision)
    ref.solve_mode(0, "qr")
    ref.sync()
    for a, b in zip(h.get_factors()[0], ref.get_factors()[0]):
        np.testing.assert_array_equal(a, b)
    f1 = h.iterate(3, solve="qr")
    f2 = ref.iterate(3, solve="qr")
    np.testing.assert_array_equal(f1, f2)


@pytest.mark.parametrize("nth", [1, 2, 7, 20])
def test_failed_allocation_in_create_reports_nomem(cuda_lib, nth):
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    cpals.test_fail_allocation(nth)
    try:
        with pytest.raises(cpals.CPALSError) as e:
            cpals.CPALS(DIMS, R, "f32")
        assert e.value.code == cpals.ERR_NOMEM
    finally:
        cpals.test_fail_allocation(0)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (8 << 20)          # nothing held on to (allocator granularity aside)
    X, A = problem()
    h = handle(X, A, "f32")
    h.iterate(2, solve="qr")


def test_failed_allocation_of_the_owned_tensor_copy(cuda_lib):
    X, A = problem()
    h = cpals.CPALS(DIMS, R, "f32")
    cpals.test_fail_allocation(1)            # the FP32 copy of X is the handle's next allocation
    try:
        with pytest.raises(cpals.CPALSError) as e:
            h.set_tensor(torch.from_numpy(X).cuda())
        assert e.value.code == cpals.ERR_NOMEM
    finally:
        cpals.test_fail_allocation(0)
    h.set_tensor(torch.from_numpy(X).cuda())
    h.set_factors(A)
    h.iterate(2, solve="qr")


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_nan_or_inf_in_x_is_refused(cuda_lib, bad, precision):
    X, A = problem()
    X[12345] = bad
    h = cpals.CPALS(DIMS, R, precision)
    with pytest.raises(cpals.CPALSError) as e:
        h.set_tensor(torch.from_numpy(X).cuda())
    assert e.value.code == cpals.ERR_ARG
    h.set_factors(A)
    with pytest.raises(cpals.CPALSError) as e:
        h.solve_mode(0, "qr")
    assert e.value.code == cpals.ERR_STATE
    X[12345] = 0.0
    h.set_tensor(torch.from_numpy(X).cuda())
    h.solve_mode(0, "qr")
    h.sync()
