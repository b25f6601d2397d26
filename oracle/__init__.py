"""FP64 CPU oracle for TSQR -- TEST INFRASTRUCTURE ONLY.

A plain unblocked Householder QR of the whole matrix (no tree), thin-Q formation, Q^T B and
Q B, sign normalisation and the two accuracy metrics, in plain C (``tsqr_oracle.c``) behind
ctypes.  TSQR computes exactly this factorization up to the signs of diag(R) (Sec. 2), so the
oracle is the definition itself.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the CUDA library never does, and the two
share no code.

Every array is row-major FP64 (numpy C order).
"""
import ctypes

import numpy as np

from .build import build as _build

_libs = {}
_variant = "serial"
_dp = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.c_int64


def set_variant(name):
    """Selects the build the functions below call: "serial" (the default) or "openmp" (the same
    source compiled with -fopenmp, bitwise the same results; used only to time the oracle on all
    host cores, with OMP_NUM_THREADS threads)."""
    global _variant
    assert name in ("serial", "openmp")
    _variant = name


def _load():
    lib = _libs.get(_variant)
    if lib is None:
        lib = ctypes.CDLL(_build(openmp=(_variant == "openmp")))
        lib.oracle_geqr2.argtypes = [_i64, _i64, _dp, _i64, _dp]
        lib.oracle_org2r.argtypes = [_i64, _i64, _dp, _i64, _dp, _dp, _i64]
        lib.oracle_apply_qt.argtypes = [_i64, _i64, _dp, _i64, _dp, _i64, _dp, _i64]
        lib.oracle_apply_q.argtypes = [_i64, _i64, _dp, _i64, _dp, _i64, _dp, _i64]
        lib.oracle_signs.argtypes = [_i64, _dp, _i64, _dp]
        lib.oracle_qr.argtypes = [_i64, _i64, _dp, _i64, _dp, _dp, _dp, _dp, _i64, _dp, _i64]
        lib.oracle_backward_error.argtypes = [_i64, _i64, _dp, _i64, _dp, _i64, _dp, _i64]
        lib.oracle_backward_error.restype = ctypes.c_double
        lib.oracle_orthogonality.argtypes = [_i64, _i64, _dp, _i64]
        lib.oracle_orthogonality.restype = ctypes.c_double
        _libs[_variant] = lib
    return lib


def _p(a):
    return a.ctypes.data_as(_dp)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def geqr2(A):
    """Householder QR in place on a copy: returns (VR, tau), VR holding R above and v below."""
    A = _c64(A).copy()
    m, n = A.shape
    assert m >= n >= 1
    tau = np.zeros(n)
    _load().oracle_geqr2(m, n, _p(A), n, _p(tau))
    return A, tau


def qr(A, want_q=True):
    """Sign-normalised thin QR of A (m x n, m >= n).

    Returns a dict with R (n x n, diag >= 0), Q (m x n, or None), D (signs), V (reflectors,
    m x n, R_raw in the upper triangle) and tau.
    """
    A = _c64(A)
    m, n = A.shape
    assert m >= n >= 1
    V = np.zeros((m, n))
    tau = np.zeros(n)
    D = np.zeros(n)
    R = np.zeros((n, n))
    Q = np.zeros((m, n)) if want_q else None
    _load().oracle_qr(m, n, _p(A), n, _p(V), _p(tau), _p(D), _p(R), n,
                      _p(Q) if want_q else None, n)
    return {"R": R, "Q": Q, "D": D, "V": V, "tau": tau}


def org2r(V, tau):
    """Thin Q = H_0 ... H_{n-1} [I; 0] (unnormalised signs)."""
    V = _c64(V)
    m, n = V.shape
    Q = np.zeros((m, n))
    _load().oracle_org2r(m, n, _p(V), n, _p(_c64(tau)), _p(Q), n)
    return Q


def apply_qt(V, tau, B):
    """Returns Q^T B for the full m x m Q = H_0 ... H_{n-1} (unnormalised signs)."""
    V = _c64(V)
    m, n = V.shape
    B = _c64(B).copy()
    squeeze = B.ndim == 1
    if squeeze:
        B = B[:, None].copy()
    _load().oracle_apply_qt(m, n, _p(V), n, _p(_c64(tau)), B.shape[1], _p(B), B.shape[1])
    return B[:, 0] if squeeze else B


def apply_q(V, tau, B):
    """Returns Q B for the full m x m Q = H_0 ... H_{n-1} (unnormalised signs)."""
    V = _c64(V)
    m, n = V.shape
    B = _c64(B).copy()
    squeeze = B.ndim == 1
    if squeeze:
        B = B[:, None].copy()
    _load().oracle_apply_q(m, n, _p(V), n, _p(_c64(tau)), B.shape[1], _p(B), B.shape[1])
    return B[:, 0] if squeeze else B


def thin_qt(A, B):
    """Top n rows of Q_norm^T B, with Q_norm the sign-normalised factor of A: D (Q^T B)_{0:n}."""
    f = qr(A, want_q=False)
    n = A.shape[1]
    top = apply_qt(f["V"], f["tau"], B)[:n]
    return (f["D"][:, None] * top) if top.ndim == 2 else f["D"] * top


def backward_error(A, Q, R):
    """||A - Q R||_F / ||A||_F (R upper triangular)."""
    A, Q, R = _c64(A), _c64(Q), _c64(R)
    m, n = A.shape
    return _load().oracle_backward_error(m, n, _p(A), n, _p(Q), n, _p(R), n)


def orthogonality(Q):
    """||I - Q^T Q||_F."""
    Q = _c64(Q)
    m, n = Q.shape
    return _load().oracle_orthogonality(m, n, _p(Q), n)
