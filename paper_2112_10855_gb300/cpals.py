"""Thin Python binding of libcpals (include/cpals.h), by ctypes.

Only argument marshalling happens here.  Every step of CP-ALS-QR runs inside
the CUDA library.  There is no CPU fallback: if the library is missing or no
GPU is present, the calls raise.

Arrays: torch CUDA tensors are passed as device pointers (CPALS_MEM_DEVICE),
numpy arrays as host pointers (CPALS_MEM_HOST).  Matrices are column-major: an
I x R factor is a tensor of shape (I, R) with strides (1, I)
(``A.t().contiguous().t()``) or a numpy array with order='F'.  The data tensor
is a flat array with mode 0 fastest.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

OK, ERR_ARG, ERR_NOMEM, ERR_CUDA, ERR_SINGULAR, ERR_TIMEOUT, ERR_STATE = range(7)
F64, F32, BF16X3, TF32X3 = 0, 1, 2, 3
SOLVE_QR, SOLVE_SVD, SOLVE_NORMAL, SOLVE_NORMAL_PINV = 0, 1, 2, 3
MEM_DEVICE, MEM_HOST = 0, 1
ELEM_F64, ELEM_F32 = 0, 1

PRECISIONS = {"f64": F64, "f32": F32, "bf16x3": BF16X3, "tf32x3": TF32X3}
SOLVES = {"qr": SOLVE_QR, "svd": SOLVE_SVD, "normal": SOLVE_NORMAL, "normal_pinv": SOLVE_NORMAL_PINV}

_vp = C.c_void_p
_lib = None


class CPALSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"cpals error {code}: {msg}")
        self.code = code


class SingularError(CPALSError):
    pass


def load(path: str | None = None):
    """Load libcpals.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libcpals.so not found at {path}; build it first (python -c 'import "
                           "__graft_entry__ as g; g.build()')")
    L = C.CDLL(path)
    i64p = C.POINTER(C.c_int64)
    L.cpals_create.argtypes = [i64p, C.c_int, C.c_int, C.c_int, C.POINTER(_vp)]
    L.cpals_destroy.argtypes = [_vp]
    L.cpals_last_error.argtypes = [_vp]
    L.cpals_last_error.restype = C.c_char_p
    L.cpals_set_stream.argtypes = [_vp, _vp]
    L.cpals_workspace_bytes.argtypes = [_vp, C.POINTER(C.c_size_t)]
    L.cpals_set_tensor.argtypes = [_vp, _vp, C.c_int, C.c_int]
    L.cpals_create_kruskal.argtypes = [i64p, C.c_int, C.c_int, C.c_int, C.POINTER(_vp)]
    L.cpals_set_tensor_kruskal.argtypes = [_vp, _vp, C.POINTER(_vp), C.c_int]
    L.cpals_set_factors.argtypes = [_vp, C.POINTER(_vp), _vp, C.c_int]
    L.cpals_get_factors.argtypes = [_vp, C.POINTER(_vp), _vp, C.c_int]
    L.cpals_get_factor_qr.argtypes = [_vp, C.c_int, _vp, _vp, C.c_int]
    L.cpals_set_factor_qr.argtypes = [_vp, C.POINTER(_vp), C.POINTER(_vp), C.c_int]
    L.cpals_krp_qr.argtypes = [_vp, C.c_int, _vp, _vp, C.c_int]
    L.cpals_multi_ttm.argtypes = [_vp, C.c_int, _vp, _vp, C.c_int]
    L.cpals_mttkrp.argtypes = [_vp, C.c_int, _vp, C.c_int]
    L.cpals_ttm_first.argtypes = [_vp, C.c_int]
    L.cpals_solve_mode.argtypes = [_vp, C.c_int, C.c_int, C.c_double]
    L.cpals_iterate.argtypes = [_vp, C.c_int, C.c_double, C.c_int, C.c_double, C.POINTER(C.c_int),
                                C.POINTER(C.c_double)]
    L.cpals_fit.argtypes = [_vp, C.c_int, C.POINTER(C.c_double)]
    L.cpals_profile_sweeps.argtypes = [_vp, C.c_int, C.c_int, C.c_double, C.POINTER(C.c_double)]
    L.cpals_sync.argtypes = [_vp]
    L.cpals_set_option.argtypes = [_vp, C.c_int, C.c_int64]
    L.cpals_launch_count.argtypes = [_vp]
    L.cpals_launch_count.restype = C.c_int64
    L.cpals_test_fail_allocation.argtypes = [C.c_int]
    L.cpals_test_newton_recip.argtypes = [_vp, C.c_int64, _vp, _vp]
    L.cpals_multi_ttm_static.argtypes = [i64p, C.c_int, C.c_int, C.c_int, _vp, C.POINTER(_vp), _vp, _vp]
    L.cpals_batch_create.argtypes = [C.c_int, i64p, C.POINTER(C.c_int), C.POINTER(_vp)]
    L.cpals_batch_destroy.argtypes = [_vp]
    L.cpals_batch_set_stream.argtypes = [_vp, _vp]
    L.cpals_batch_set_tensors.argtypes = [_vp, C.POINTER(_vp), C.c_int]
    L.cpals_batch_set_factors.argtypes = [_vp, C.POINTER(_vp), C.c_int]
    L.cpals_batch_get_factors.argtypes = [_vp, C.POINTER(_vp), C.POINTER(_vp), C.c_int]
    L.cpals_batch_iterate.argtypes = [_vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)]
    L.cpals_batch_launch_count.argtypes = [_vp]
    L.cpals_batch_launch_count.restype = C.c_int64
    L.cpals_batch_launch_shape.argtypes = [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.cpals_probe_fma_peak.argtypes = [C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    _lib = L
    return L


def exported_symbols():
    """Names of the C-ABI entry points declared in include/cpals.h."""
    import re
    hdr = os.path.join(_build.ROOT, "include", "cpals.h")
    with open(hdr) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(cpals_[a-z0-9_]+)\s*\(", text)))


def _check(h, rc):
    if rc != OK:
        msg = load().cpals_last_error(h).decode(errors="replace")
        if rc == ERR_SINGULAR:
            raise SingularError(rc, msg)
        raise CPALSError(rc, msg)


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, mem flag) of a torch tensor or numpy array."""
    if x is None:
        return None, MEM_DEVICE
    if _is_torch(x):
        if x.is_cuda:
            return C.c_void_p(x.data_ptr()), MEM_DEVICE
        return C.c_void_p(x.data_ptr()), MEM_HOST
    if isinstance(x, np.ndarray):
        return C.c_void_p(x.ctypes.data), MEM_HOST
    raise TypeError(f"unsupported array type {type(x)}")


def _colmajor_ok(x, rows, cols):
    if _is_torch(x):
        return tuple(x.shape) == (rows, cols) and (cols == 1 or x.stride() == (1, rows) or rows == 1) \
            and x.dtype.is_floating_point and x.element_size() == 8
    return x.shape == (rows, cols) and x.dtype == np.float64 and (x.flags.f_contiguous or cols == 1)


class CPALS:
    """One CP-ALS(-QR) problem: cpals_create / cpals_destroy and the calls of include/cpals.h."""

    def __init__(self, dims, rank, precision="f64", kruskal_rank=None):
        """kruskal_rank=S: a handle for a tensor given in Kruskal form
        (cpals_create_kruskal, Sec. 3.3.2); set it with set_tensor_kruskal."""
        import torch  # noqa: F401  (the library shares the device and context with torch)
        L = load()
        self.dims = tuple(int(d) for d in dims)
        self.N = len(self.dims)
        self.R = int(rank)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.S = None if kruskal_rank is None else int(kruskal_rank)
        d = (C.c_int64 * self.N)(*self.dims)
        h = _vp()
        if self.S is None:
            rc = L.cpals_create(d, self.N, self.R, self.precision, C.byref(h))
        else:
            if self.precision != PRECISIONS["f64"]:
                raise ValueError("Kruskal input runs in FP64")
            rc = L.cpals_create_kruskal(d, self.N, self.R, self.S, C.byref(h))
        if rc != OK:
            raise CPALSError(rc, L.cpals_last_error(None).decode(errors="replace"))
        self._h = h
        self._keep = []

    def close(self):
        if getattr(self, "_h", None):
            load().cpals_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- plumbing
    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
        raw = getattr(stream, "cuda_stream", stream)
        _check(self._h, load().cpals_set_stream(self._h, C.c_void_p(raw or 0)))

    def workspace_bytes(self):
        b = C.c_size_t()
        _check(self._h, load().cpals_workspace_bytes(self._h, C.byref(b)))
        return b.value

    def launch_count(self):
        return load().cpals_launch_count(self._h)

    def set_dimtree(self, on: bool):
        """CPALS_OPT_DIMTREE: share Multi-TTM passes over X across modes in sweeps."""
        _check(self._h, load().cpals_set_option(self._h, 0, 1 if on else 0))

    def set_tc_pipeline(self, on: bool):
        """CPALS_OPT_TC_PIPELINE: persistent TMA-fed tensor-core kernel for the pass over X."""
        _check(self._h, load().cpals_set_option(self._h, 1, 1 if on else 0))

    def set_krp_tree(self, on: bool):
        """CPALS_OPT_KRP_TREE: per-half QR of the Khatri-Rao products in dimension-tree sweeps."""
        _check(self._h, load().cpals_set_option(self._h, 2, 1 if on else 0))

    def set_f32_pipeline(self, on: bool):
        """CPALS_OPT_F32_PIPELINE: TMA-fed CUDA-core kernel for the FP32 TTMs."""
        _check(self._h, load().cpals_set_option(self._h, 3, 1 if on else 0))

    def set_test_withhold_copies(self, on: bool):
        """CPALS_OPT_TEST_WITHHOLD_COPIES (test hook): the tensor-core pass over X
        issues no copies and its bounded waits run out after 1 ms."""
        _check(self._h, load().cpals_set_option(self._h, 4, 1 if on else 0))

    def set_fused_tail(self, on):
        """CPALS_OPT_FUSED_TAIL: solve, normalisation and CholeskyQR2 of the factor in the fused kernels
        (True / False force it; "auto", the default, takes them from rank 8 up)."""
        v = 2 if on == "auto" else (1 if on else 0)
        _check(self._h, load().cpals_set_option(self._h, 5, v))

    def set_svd_shortcut(self, on: bool):
        """CPALS_OPT_SVD_SHORTCUT: skip the Jacobi SVD when a norm bound proves nothing is truncated."""
        _check(self._h, load().cpals_set_option(self._h, 6, 1 if on else 0))

    def set_apply_q0_fp32(self, on: bool):
        """CPALS_OPT_APPLY_Q0_FP32: mixed precisions form W = Y_(n) Q0 in FP32."""
        _check(self._h, load().cpals_set_option(self._h, 7, 1 if on else 0))

    def set_wide_tail(self, on: bool):
        """CPALS_OPT_WIDE_TAIL: above rank 32, CholeskyQR2 of the factors and fold steps over every SM."""
        _check(self._h, load().cpals_set_option(self._h, 8, 1 if on else 0))

    def sync(self):
        _check(self._h, load().cpals_sync(self._h))

    # -- data
    def set_tensor(self, X):
        """X: flat float64/float32 array of prod(dims) entries, mode 0 fastest."""
        n = int(np.prod(self.dims))
        if _is_torch(X):
            if not X.is_contiguous() or X.numel() != n:
                raise ValueError("X must be a contiguous tensor with prod(dims) entries")
            elem = ELEM_F64 if X.element_size() == 8 else ELEM_F32
        else:
            X = np.ascontiguousarray(X)
            if X.size != n:
                raise ValueError("X must have prod(dims) entries")
            elem = ELEM_F64 if X.dtype == np.float64 else ELEM_F32
        p, mem = _ptr(X)
        self._X = X   # a borrowed device pointer must stay alive
        _check(self._h, load().cpals_set_tensor(self._h, p, elem, mem))

    def _mats_in(self, mats, rows, cols=None):
        cols = self.R if cols is None else cols
        ptrs, mem = [], None
        for m, A in enumerate(mats):
            if not _colmajor_ok(A, rows[m], cols):
                raise ValueError(f"matrix {m} must be a column-major float64 {rows[m]} x {cols} array")
            p, mm = _ptr(A)
            if mem is not None and mm != mem:
                raise ValueError("mix of host and device matrices")
            mem = mm
            ptrs.append(p)
        return (_vp * len(ptrs))(*ptrs), mem

    def set_factors(self, A, lam=None):
        arr, mem = self._mats_in(A, self.dims)
        lp = None
        if lam is not None:
            lp, lm = _ptr(lam)
            if lm != mem:
                raise ValueError("lambda must live where the factors live")
        _check(self._h, load().cpals_set_factors(self._h, arr, lp, mem))

    def set_tensor_kruskal(self, mu, V):
        """V: N column-major FP64 I_m x S arrays (numpy or CUDA torch); mu: S weights or None."""
        arr, mem = self._mats_in(V, self.dims, cols=self.S)
        mp = None
        if mu is not None:
            mp, mm = _ptr(mu)
            if mm != mem:
                raise ValueError("mu must live where the factors live")
        _check(self._h, load().cpals_set_tensor_kruskal(self._h, mp, arr, mem))

    def set_factor_qr(self, Q, R):
        qa, mem = self._mats_in(Q, self.dims)
        ra, mem2 = self._mats_in(R, [self.R] * self.N)
        if mem != mem2:
            raise ValueError("Q and R must live in the same memory")
        _check(self._h, load().cpals_set_factor_qr(self._h, qa, ra, mem))

    def _out(self, rows, cols, device):
        if device:
            import torch
            return torch.empty((cols, rows), dtype=torch.float64, device="cuda").t()
        return np.zeros((rows, cols), order="F")

    def get_factors(self, device=False):
        outs = [self._out(d, self.R, device) for d in self.dims]
        lam = self._out(self.R, 1, device)[:, 0] if device else np.zeros(self.R)
        ptrs = [_ptr(o)[0] for o in outs]
        lp, mem = _ptr(lam)
        _check(self._h, load().cpals_get_factors(self._h, (_vp * self.N)(*ptrs), lp, mem))
        return outs, lam

    def get_factor_qr(self, mode, device=False):
        Q = self._out(self.dims[mode], self.R, device)
        R = self._out(self.R, self.R, device)
        _check(self._h, load().cpals_get_factor_qr(self._h, mode, _ptr(Q)[0], _ptr(R)[0],
                                                   MEM_DEVICE if device else MEM_HOST))
        return Q, R

    # -- the hot path
    def krp_qr(self, mode, device=False):
        RN1 = self.R ** (self.N - 1)
        Q0 = None if self.S is not None else self._out(RN1, self.R, device)
        R0 = self._out(self.R, self.R, device)
        _check(self._h, load().cpals_krp_qr(self._h, mode, _ptr(Q0)[0], _ptr(R0)[0],
                                            MEM_DEVICE if device else MEM_HOST))
        return Q0, R0

    def multi_ttm(self, mode, want_Y=True, want_W=False, device=False):
        RN1 = self.R ** (self.N - 1)
        In = self.dims[mode]
        Y = self._out(In, RN1, device) if want_Y else None
        W = self._out(In, self.R, device) if want_W else None
        _check(self._h, load().cpals_multi_ttm(self._h, mode, _ptr(Y)[0], _ptr(W)[0],
                                               MEM_DEVICE if device else MEM_HOST))
        return Y, W

    def ttm_first(self, mode):
        _check(self._h, load().cpals_ttm_first(self._h, mode))

    def mttkrp(self, mode, device=False):
        M = self._out(self.dims[mode], self.R, device)
        _check(self._h, load().cpals_mttkrp(self._h, mode, _ptr(M)[0], MEM_DEVICE if device else MEM_HOST))
        return M

    def solve_mode(self, mode, solve="qr", svd_rtol=0.0):
        s = SOLVES[solve] if isinstance(solve, str) else int(solve)
        _check(self._h, load().cpals_solve_mode(self._h, mode, s, float(svd_rtol)))

    def iterate(self, iters, tol=0.0, solve="qr", svd_rtol=0.0, want_fits=True):
        s = SOLVES[solve] if isinstance(solve, str) else int(solve)
        done = C.c_int(0)
        fits = (C.c_double * max(int(iters), 1))() if want_fits else None
        _check(self._h, load().cpals_iterate(self._h, int(iters), float(tol), s, float(svd_rtol),
                                             C.byref(done), fits))
        return np.array(fits[:done.value]) if want_fits else done.value

    def profile_sweeps(self, sweeps=3, solve="qr", svd_rtol=0.0):
        """cpals_profile_sweeps: mean ms per sweep in the five buckets of Table its_parts
        (passes over X, factor QR or Gram, computing Q0, applying Q0, other)."""
        out = (C.c_double * 5)()
        _check(self._h, load().cpals_profile_sweeps(self._h, int(sweeps), SOLVES[solve], float(svd_rtol), out))
        return dict(zip(["multi_ttm_or_mttkrp", "factor_qr_or_gram", "compute_q0", "apply_q0", "other"], list(out)))

    def fit(self, direct=False):
        f = C.c_double()
        _check(self._h, load().cpals_fit(self._h, 1 if direct else 0, C.byref(f)))
        return f.value


class CPALSBatch:
    """Many independent 3-way problems: cpals_batch_create and the cpals_batch_* calls."""

    def __init__(self, dims, ranks):
        L = load()
        self.dims = [tuple(int(x) for x in d) for d in dims]
        self.ranks = [int(r) for r in ranks]
        self.count = len(self.dims)
        flat = (C.c_int64 * (3 * self.count))(*[x for d in self.dims for x in d])
        rk = (C.c_int * self.count)(*self.ranks)
        h = _vp()
        rc = L.cpals_batch_create(self.count, flat, rk, C.byref(h))
        if rc != OK:
            raise CPALSError(rc, L.cpals_last_error(None).decode(errors="replace"))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().cpals_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _rc(self, rc):
        if rc != OK:
            raise CPALSError(rc, load().cpals_last_error(None).decode(errors="replace"))

    def set_stream(self, stream):
        raw = getattr(stream, "cuda_stream", stream)
        self._rc(load().cpals_batch_set_stream(self._h, C.c_void_p(raw or 0)))

    def set_tensors(self, Xs):
        """Xs: count flat FP32 arrays (numpy: host; torch CUDA: device)."""
        arrs = [np.ascontiguousarray(x, dtype=np.float32) if isinstance(x, np.ndarray) else x for x in Xs]
        ptrs = [_ptr(a) for a in arrs]
        mem = ptrs[0][1]
        self._keepX = arrs
        self._rc(load().cpals_batch_set_tensors(self._h, (_vp * self.count)(*[p for p, _ in ptrs]), mem))

    def set_factors(self, A):
        """A: count lists of 3 column-major FP64 I_m x R_p arrays (numpy)."""
        mats = [np.asfortranarray(a, dtype=np.float64) for fs in A for a in fs]
        self._keepA = mats
        ptrs = (_vp * len(mats))(*[C.c_void_p(m.ctypes.data) for m in mats])
        self._rc(load().cpals_batch_set_factors(self._h, ptrs, MEM_HOST))

    def get_factors(self):
        outs = [[np.zeros((d[m], r), order="F") for m in range(3)] for d, r in zip(self.dims, self.ranks)]
        lams = [np.zeros(r) for r in self.ranks]
        aptr = (_vp * (3 * self.count))(*[C.c_void_p(o.ctypes.data) for fs in outs for o in fs])
        lptr = (_vp * self.count)(*[C.c_void_p(l.ctypes.data) for l in lams])
        self._rc(load().cpals_batch_get_factors(self._h, aptr, lptr, MEM_HOST))
        return outs, lams

    def iterate(self, iters):
        fits = (C.c_double * self.count)()
        st = (C.c_int * self.count)()
        self._rc(load().cpals_batch_iterate(self._h, int(iters), fits, st))
        return np.array(fits[:]), np.array(st[:])

    def launch_count(self):
        return load().cpals_batch_launch_count(self._h)

    def launch_shape(self):
        g, t = C.c_int(), C.c_int()
        load().cpals_batch_launch_shape(self._h, C.byref(g), C.byref(t))
        return g.value, t.value


def multi_ttm_static(X, Q, mode, rank, dims, Y, stream=None):
    """cpals_multi_ttm_static: Multi-TTM into the caller's device tensor Y
    (I_n x R^{N-1}, column-major), with no device allocation by the library.
    X: flat FP64 CUDA tensor; Q: list of N column-major FP64 CUDA tensors
    (Q[mode] may be None)."""
    L = load()
    dims = tuple(int(d) for d in dims)
    N = len(dims)
    d = (C.c_int64 * N)(*dims)
    ptrs = (_vp * N)(*[None if q is None else C.c_void_p(q.data_ptr()) for q in Q])
    raw = getattr(stream, "cuda_stream", stream) or 0
    rc = L.cpals_multi_ttm_static(d, N, int(rank), int(mode), C.c_void_p(X.data_ptr()), ptrs,
                                  C.c_void_p(Y.data_ptr()), C.c_void_p(raw))
    if rc != OK:
        raise CPALSError(rc, L.cpals_last_error(None).decode(errors="replace"))


def test_fail_allocation(nth):
    """cpals_test_fail_allocation (test hook): the nth device allocation of a
    handle from now on fails as if the device were out of memory (0 disables)."""
    L = load()
    rc = L.cpals_test_fail_allocation(int(nth))
    if rc != OK:
        raise CPALSError(rc, L.cpals_last_error(None).decode(errors="replace"))


def test_newton_recip(x):
    """cpals_test_newton_recip (test hook): (1/x, 1/sqrt(x)) as the fused mode
    tail computes them, for a float64 CUDA tensor x."""
    import torch
    rcp = torch.empty_like(x)
    rsq = torch.empty_like(x)
    L = load()
    rc = L.cpals_test_newton_recip(C.c_void_p(x.data_ptr()), x.numel(), C.c_void_p(rcp.data_ptr()),
                                   C.c_void_p(rsq.data_ptr()))
    if rc != OK:
        raise CPALSError(rc, L.cpals_last_error(None).decode(errors="replace"))
    return rcp, rsq


def probe_fma_peak(ms_target=50.0):
    """Measured FP64 and FP32 FMA throughput in TFLOP/s (dependent-chain probe)."""
    a, b = C.c_double(), C.c_double()
    rc = load().cpals_probe_fma_peak(float(ms_target), C.byref(a), C.byref(b))
    if rc != OK:
        raise CPALSError(rc, "FMA probe failed")
    return a.value, b.value
