"""cpals_multi_ttm_static: the Multi-TTM entry point that allocates nothing.

It serves callers that must not allocate device memory (a framework whose
pool allocator owns all device memory, a hard device-memory budget, or a
latency-critical loop that cannot take cudaMalloc's implicit
synchronisation).  Its scratch is a fixed 16 MiB array inside the library.
This test calls it through the C-ABI, twice in a row, and checks each result
against cpals_multi_ttm on the same inputs, within the parity tolerance of
the other Multi-TTM tests (relative Frobenius 1e-12).  Two calls in a row
show that the contents the first call leaves in the shared array do not
leak into the second call's result.  The file's name makes pytest collect it
last.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2112_10855_gb300 import cpals

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("dims,R,modes", [
    ((120, 110, 100), 10, None), ((37, 29, 41), 5, None), ((12, 11, 10, 9), 3, None),
    # a long first mode: the first TTM splits its 40000 indices more than 16
    # ways (two-pass reduction) and the partials fill over 90% of the array
    # (tests/test_ttm_plan_cpu.py checks that plan on the CPU)
    ((40000, 10, 10), 10, (1, 2)),
])
def test_static_multi_ttm_matches_handle_path_twice(cuda_lib, dims, R, modes):
    rng = np.random.default_rng(sum(dims) * R)
    X = rng.standard_normal(int(np.prod(dims)))
    QR = [oracle.qr(rng.standard_normal((d, R))) for d in dims]
    Q = [np.asfortranarray(q) for q, _ in QR]
    Rm = [np.asfortranarray(r) for _, r in QR]
    Xd = torch.from_numpy(X).cuda()
    Qd = [torch.from_numpy(q).cuda() for q in Q]        # keeps the column-major strides
    assert all(q.stride() == (1, q.shape[0]) for q in Qd)
    h = cpals.CPALS(dims, R, "f64")
    h.set_tensor(Xd)
    h.set_factor_qr(Q, Rm)
    stream = torch.cuda.current_stream()
    for n in (range(len(dims)) if modes is None else modes):
        ref, _ = h.multi_ttm(n)
        for call in range(2):
            Y = torch.full((R ** (len(dims) - 1), dims[n]), float("nan"), dtype=torch.float64, device="cuda").t()
            cpals.multi_ttm_static(Xd, [None if m == n else Qd[m] for m in range(len(dims))], n, R, dims, Y,
                                   stream)
            torch.cuda.synchronize()
            got = Y.cpu().numpy()
            assert np.isfinite(got).all()
            assert rel(got, ref) <= 1e-12, (n, call, rel(got, ref))


def test_static_multi_ttm_rejects_oversize(cuda_lib):
    # 400^3 rank 64: the first intermediate alone is 160000*64 doubles > 2^21
    dims, R = (400, 400, 400), 64
    X = torch.zeros(1, dtype=torch.float64, device="cuda")
    Q = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in dims]
    Y = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(cpals.CPALSError) as e:
        cpals.multi_ttm_static(X, Q, 0, R, dims, Y)
    assert e.value.code == cpals.ERR_ARG
    assert "static scratch" in str(e.value)
