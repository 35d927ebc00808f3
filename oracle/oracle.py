"""ctypes wrappers around the C oracle (test infrastructure only).

Arrays are float64.  Matrices are column-major (numpy order='F').  Tensors are
flat with mode 1 fastest.  Each wrapper allocates its outputs and returns them.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpals_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libcpals_oracle.so")
_lock = threading.Lock()
_lib = None

QR, SVD, NORMAL, NORMAL_PINV = 0, 1, 2, 3

_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, IEEE arithmetic, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class use_library:
    """Context manager: route the wrappers to another build of the oracle (a
    copy with a planted mistake, compiled by the tests)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        lib()
        self._saved = _lib
        _lib = _configure(C.CDLL(self.path))
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile oracle source text (e.g. with a planted mistake) to out_path."""
    c_path = out_path + ".c"
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                           "-ffp-contract=off", "-o", out_path, c_path, "-lm"])
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _configure(C.CDLL(_SO))
    return _lib


def _configure(L):
    L.orc_multi_ttm.restype = C.c_int64
    L.orc_qr_madds.restype = C.c_int64
    L.orc_trsm_qr.restype = C.c_int
    L.orc_svd_solve.restype = C.c_int
    L.orc_cholesky_solve.restype = C.c_int
    L.orc_residual_direct.restype = C.c_double
    L.orc_norm2.restype = C.c_double
    L.orc_fit_efficient_qr.restype = C.c_double
    L.orc_fit_efficient_normal.restype = C.c_double
    L.orc_score.restype = C.c_double
    L.orc_create.restype = C.c_void_p
    L.orc_create.argtypes = [C.c_int, _i64p, C.c_int64, _dp]
    L.orc_destroy.argtypes = [C.c_void_p]
    L.orc_set_factors.argtypes = [C.c_void_p, C.POINTER(_dp), _dp]
    L.orc_krp_qr.argtypes = [C.c_void_p, C.c_int]
    L.orc_update_mode.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double]
    L.orc_update_mode.restype = C.c_int
    L.orc_fit_last.argtypes = [C.c_void_p, C.c_int]
    L.orc_fit_last.restype = C.c_double
    L.orc_iterate.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_double, _dp]
    L.orc_iterate.restype = C.c_int
    L.orc_fit_direct.argtypes = [C.c_void_p]
    L.orc_fit_direct.restype = C.c_double
    L.orc_get_normX2.argtypes = [C.c_void_p]
    L.orc_get_normX2.restype = C.c_double
    L.orc_get_factor.argtypes = [C.c_void_p, C.c_int, _dp]
    L.orc_get_qr_factor.argtypes = [C.c_void_p, C.c_int, _dp, _dp]
    L.orc_get_lambda.argtypes = [C.c_void_p, _dp]
    L.orc_get_last.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp, _dp]
    L.orc_get_mttkrp.argtypes = [C.c_void_p, _dp, _dp]
    return L


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and (a.flags.f_contiguous or a.flags.c_contiguous)
    return a.ctypes.data_as(_dp)


def _f(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _dims(dims):
    d = np.asarray(dims, dtype=np.int64)
    return d, d.ctypes.data_as(_i64p)


def _ptr_array(mats):
    arr = (_dp * len(mats))(*[_p(m) for m in mats])
    return arr


def qr(A, return_madds=False):
    """Householder QR with explicit Q and diag(R) >= 0.  return_madds: also
    the multiply-adds of its two O(m n^2) loop nests (Eq. QRcost pin)."""
    A = _f(A)
    m, n = A.shape
    Q = np.zeros((m, n), order="F")
    R = np.zeros((n, n), order="F")
    L = lib()
    L.orc_qr_madds(1)
    L.orc_qr(C.c_int64(m), C.c_int64(n), _p(A), _p(Q), _p(R))
    madds = L.orc_qr_madds(1)
    return (Q, R, madds) if return_madds else (Q, R)


def krp(mats):
    mats = [_f(m) for m in mats]
    R = mats[0].shape[1]
    rows = np.array([m.shape[0] for m in mats], dtype=np.int64)
    out = np.zeros((int(np.prod(rows)), R), order="F")
    lib().orc_krp(C.c_int(len(mats)), rows.ctypes.data_as(_i64p), _ptr_array(mats),
                  C.c_int64(R), _p(out))
    return out


def unfold(X, dims, n):
    X = np.ascontiguousarray(X, dtype=np.float64)
    d, dp = _dims(dims)
    out = np.zeros((d[n], X.size // d[n]), order="F")
    lib().orc_unfold(C.c_int(len(d)), dp, _p(X), C.c_int(n), _p(out))
    return out


def ttm(X, dims, mode, U):
    X = np.ascontiguousarray(X, dtype=np.float64)
    U = _f(U)
    d, dp = _dims(dims)
    J = U.shape[0]
    out = np.zeros(X.size // d[mode] * J)
    lib().orc_ttm(C.c_int(len(d)), dp, _p(X), C.c_int(mode), C.c_int64(J), _p(U), _p(out))
    return out


def ttm_order(dims, n):
    d, dp = _dims(dims)
    order = (C.c_int * len(d))()
    lib().orc_ttm_order(C.c_int(len(d)), dp, C.c_int(n), order)
    return [order[k] for k in range(len(d) - 1)]


def multi_ttm(X, dims, n, Q, order=None, return_madds=False):
    """Y_(n) (I_n x R^{N-1}) of X x_{m != n} Q_m^T."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    Q = [_f(q) for q in Q]
    d, dp = _dims(dims)
    R = Q[(n + 1) % len(d)].shape[1]
    Y = np.zeros((d[n], R ** (len(d) - 1)), order="F")
    ordp = None
    if order is not None:
        ordp = (C.c_int * (len(d) - 1))(*order)
    madds = lib().orc_multi_ttm(C.c_int(len(d)), dp, _p(X), C.c_int(n), C.c_int64(R),
                                _ptr_array(Q), ordp, _p(Y))
    return (Y, madds) if return_madds else Y


def trsm_qr(W, R0):
    W, R0 = _f(W), _f(R0)
    I, R = W.shape
    A = np.zeros((I, R), order="F")
    rc = lib().orc_trsm_qr(C.c_int64(I), C.c_int64(R), _p(W), _p(R0), _p(A))
    if rc:
        raise np.linalg.LinAlgError("R0 is numerically singular")
    return A


def jacobi_svd(A):
    A = _f(A)
    n = A.shape[0]
    U = np.zeros((n, n), order="F")
    V = np.zeros((n, n), order="F")
    S = np.zeros(n)
    lib().orc_jacobi_svd(C.c_int64(n), _p(A), _p(U), _p(S), _p(V))
    return U, S, V


def svd_solve(W, R0, rtol):
    W, R0 = _f(W), _f(R0)
    I, R = W.shape
    A = np.zeros((I, R), order="F")
    kept = lib().orc_svd_solve(C.c_int64(I), C.c_int64(R), _p(W), _p(R0), C.c_double(rtol), _p(A))
    return A, kept


def normalize(Ahat):
    Ahat = _f(Ahat)
    I, R = Ahat.shape
    A = np.zeros((I, R), order="F")
    lam = np.zeros(R)
    lib().orc_normalize(C.c_int64(I), C.c_int64(R), _p(Ahat), _p(A), _p(lam))
    return A, lam


def mttkrp(X, dims, n, A):
    X = np.ascontiguousarray(X, dtype=np.float64)
    A = [_f(a) for a in A]
    d, dp = _dims(dims)
    R = A[0].shape[1]
    M = np.zeros((d[n], R), order="F")
    lib().orc_mttkrp(C.c_int(len(d)), dp, _p(X), C.c_int(n), C.c_int64(R), _ptr_array(A), _p(M))
    return M


def cholesky_solve(M, S):
    M, S = _f(M), _f(S)
    I, R = M.shape
    A = np.zeros((I, R), order="F")
    if lib().orc_cholesky_solve(C.c_int64(I), C.c_int64(R), _p(M), _p(S), _p(A)):
        raise np.linalg.LinAlgError("S is not positive definite")
    return A


def residual_direct(X, dims, lam, A):
    X = np.ascontiguousarray(X, dtype=np.float64)
    A = [_f(a) for a in A]
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    d, dp = _dims(dims)
    return lib().orc_residual_direct(C.c_int(len(d)), dp, _p(X), C.c_int64(A[0].shape[1]),
                                     _p(lam), _ptr_array(A))


def fit_efficient_qr(normX2, WN, AhatN, R0, RN, lam):
    WN, AhatN, R0, RN = _f(WN), _f(AhatN), _f(R0), _f(RN)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    IN, R = WN.shape
    return lib().orc_fit_efficient_qr(C.c_double(normX2), C.c_int64(IN), C.c_int64(R), _p(WN),
                                      _p(AhatN), _p(R0), _p(RN), _p(lam))


def score(dims, lam1, A1, lam2, A2):
    A1 = [_f(a) for a in A1]
    A2 = [_f(a) for a in A2]
    lam1 = np.ascontiguousarray(lam1, dtype=np.float64)
    lam2 = np.ascontiguousarray(lam2, dtype=np.float64)
    d, dp = _dims(dims)
    return lib().orc_score(C.c_int(len(d)), dp, C.c_int64(A1[0].shape[1]), _p(lam1),
                           _ptr_array(A1), _p(lam2), _ptr_array(A2))


class OracleCPALS:
    """Alg. cp-als-qr / Alg. cp-als driver state held by the C oracle."""

    def __init__(self, X, dims, rank):
        self.X = np.ascontiguousarray(X, dtype=np.float64)   # kept alive: the C side borrows it
        self.dims = tuple(int(x) for x in dims)
        self.N = len(self.dims)
        self.R = int(rank)
        self._d, dp = _dims(self.dims)
        self._h = lib().orc_create(C.c_int(self.N), dp, C.c_int64(self.R), _p(self.X))
        if not self._h:
            raise ValueError("invalid oracle problem")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def set_factors(self, A, lam=None):
        A = [_f(a) for a in A]
        self._keep = A
        lp = None
        if lam is not None:
            self._lam_keep = np.ascontiguousarray(lam, dtype=np.float64)
            lp = _p(self._lam_keep)
        lib().orc_set_factors(self._h, _ptr_array(A), lp)

    def update_mode(self, n, solve=QR, rtol=0.0):
        return lib().orc_update_mode(self._h, n, solve, rtol)

    def krp_qr(self, n):
        lib().orc_krp_qr(self._h, n)
        RN1 = self.R ** (self.N - 1)
        Q0 = np.zeros((RN1, self.R), order="F")
        R0 = np.zeros((self.R, self.R), order="F")
        lib().orc_get_last(self._h, _p(Q0), _p(R0), None, None, None)
        return Q0, R0

    def iterate(self, iters, tol=0.0, solve=QR, rtol=0.0):
        fits = np.zeros(max(iters, 1))
        k = lib().orc_iterate(self._h, iters, tol, solve, rtol, _p(fits))
        return k, fits[:abs(k) if k else 0]

    def fit_last(self, solve=QR):
        return lib().orc_fit_last(self._h, solve)

    def fit_direct(self):
        return lib().orc_fit_direct(self._h)

    @property
    def normX2(self):
        return lib().orc_get_normX2(self._h)

    def factor(self, m):
        A = np.zeros((self.dims[m], self.R), order="F")
        lib().orc_get_factor(self._h, m, _p(A))
        return A

    def factors(self):
        return [self.factor(m) for m in range(self.N)]

    def qr_factor(self, m):
        Q = np.zeros((self.dims[m], self.R), order="F")
        R = np.zeros((self.R, self.R), order="F")
        lib().orc_get_qr_factor(self._h, m, _p(Q), _p(R))
        return Q, R

    def lam(self):
        out = np.zeros(self.R)
        lib().orc_get_lambda(self._h, _p(out))
        return out

    def last(self, n):
        RN1 = self.R ** (self.N - 1)
        In = self.dims[n]
        Q0 = np.zeros((RN1, self.R), order="F")
        R0 = np.zeros((self.R, self.R), order="F")
        Y = np.zeros((In, RN1), order="F")
        W = np.zeros((In, self.R), order="F")
        Ah = np.zeros((In, self.R), order="F")
        lib().orc_get_last(self._h, _p(Q0), _p(R0), _p(Y), _p(W), _p(Ah))
        return {"Q0": Q0, "R0": R0, "Y": Y, "W": W, "Ahat": Ah}

    def last_mttkrp(self, n):
        M = np.zeros((self.dims[n], self.R), order="F")
        S = np.zeros((self.R, self.R), order="F")
        lib().orc_get_mttkrp(self._h, _p(M), _p(S))
        return M, S
