"""ctypes binding of the plain-C oracle routines (test infrastructure only)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from .build_oracle import build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        i64 = C.c_int64
        _lib.or_gen_eig.argtypes = [i64, P, P, P, P]
        _lib.or_gen_eig_lowest.argtypes = [i64, P, P, i64, P, P]
        _lib.or_tridiag_eig.argtypes = [i64, P, P, P, P]
        _lib.or_ldlt_bk.argtypes = [i64, P, P, P, P]
        _lib.or_band_ldlt.argtypes = [i64, i64, P, P, P]
        _lib.or_csr_mm.argtypes = [i64, P, P, P, i64, P, P]
        _lib.or_csr_mm.restype = None
        _lib.or_num_threads.restype = C.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def num_threads() -> int:
    return int(lib().or_num_threads())


def gen_eig(A: np.ndarray, B: np.ndarray, vectors: bool = True):
    """All eigenpairs of A x = lambda B x (Eq. 1); X^T B X = I.  Returns (lam, X|None)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    n = A.shape[0]
    lam = np.empty(n)
    X = np.empty((n, n)) if vectors else None
    rc = lib().or_gen_eig(n, _p(A), _p(B), _p(lam), _p(X))
    if rc == 1:
        raise np.linalg.LinAlgError("B is not positive definite")
    if rc:
        raise RuntimeError(f"or_gen_eig failed ({rc})")
    return lam, X


def gen_eig_lowest(A: np.ndarray, B: np.ndarray, m: int):
    """The lowest m eigenpairs of A x = lambda B x (Eq. 1) by the same reduction as
    gen_eig, with the tridiagonal matrix's eigenvectors from inverse iteration and the
    Householder back-transform (no full set of vectors is formed).  Returns (theta, X):
    theta the eigenvalues of the reduced matrix, X (n x m) with x^T B x = 1."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    n = A.shape[0]
    lam = np.empty(m)
    X = np.empty((n, m))
    rc = lib().or_gen_eig_lowest(n, _p(A), _p(B), m, _p(lam), _p(X))
    if rc == 1:
        raise np.linalg.LinAlgError("B is not positive definite")
    if rc:
        raise RuntimeError(f"or_gen_eig_lowest failed ({rc})")
    return lam, X


def tridiag_eig(d: np.ndarray, off: np.ndarray, vectors: bool = True):
    d = np.ascontiguousarray(d, dtype=np.float64)
    off = np.ascontiguousarray(off, dtype=np.float64)
    m = d.size
    th = np.empty(m)
    Z = np.empty((m, m)) if vectors else None
    rc = lib().or_tridiag_eig(m, _p(d), _p(off), _p(th), _p(Z))
    if rc:
        raise RuntimeError("tridiagonal QL did not converge")
    return th, Z


def ldlt_bk(M: np.ndarray):
    """Dense Bunch-Kaufman LDL^T; returns (inertia (neg, zero, pos), piv_kind, dvals)."""
    W = np.array(M, dtype=np.float64, order="C", copy=True)
    n = W.shape[0]
    inert = np.zeros(3, dtype=np.int64)
    kind = np.zeros(n, dtype=np.int32)
    dv = np.zeros(2 * n)
    lib().or_ldlt_bk(n, _p(W), _p(inert), _p(kind), _p(dv))
    return tuple(int(x) for x in inert), kind, dv


def band_ldlt(band: np.ndarray):
    """Unpivoted band LDL^T; band is (n, bw+1) with band[j, t] = M[j+t, j].

    Returns (inertia, min |d_j| / max |M_jj|, rc)."""
    W = np.array(band, dtype=np.float64, order="C", copy=True)
    n, ld = W.shape
    inert = np.zeros(3, dtype=np.int64)
    rmin = np.zeros(1)
    rc = lib().or_band_ldlt(n, ld - 1, _p(W), _p(inert), _p(rmin))
    return tuple(int(x) for x in inert), float(rmin[0]), int(rc)


def csr_mm(rowptr, colind, vals, X):
    """Y = M X for CSR M and row-major X (n x k)."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    n = rowptr.size - 1
    Y = np.empty((n, X.shape[1]))
    lib().or_csr_mm(n, _p(rowptr), _p(colind), _p(vals), X.shape[1], _p(X), _p(Y))
    return Y
