"""Exact spectral quantities from the dense oracle (test infrastructure only).

* inertia / eigenvalue counts: Sylvester's law, Section 2.2 -- the number of negative
  pivots of LDL^T(A - sigma B) equals #{lambda_i < sigma}.
* slice membership: the slice (lo, hi] holds the eigenpairs with lo < lambda <= hi,
  and its count is nu(hi) - nu(lo) (Section 2.2 validation counts).
* residuals: R_j = A X_j - B X_j Lambda_j, column 2-norms (after Alg. 2), normalised by
  ||A||_1 ||x||_2.
* lowest eigenvalues of a pencil (Eq. 1) as Rayleigh quotients x^T A x / x^T B x of the
  reduced solver's eigenvectors on the original sparse A and B: the quotient's error is
  second order in the eigenvector's, while forming L^-1 A L^-T (B = L L^T) leaves a
  first-order error of about u ||A|| ||x||_2^2 in the reduced eigenvalue -- large for
  eigenvectors with ||x||_B = 1 but ||x||_2 >> 1 when B is ill-conditioned.
"""
from __future__ import annotations

import numpy as np

from . import dense


def count_below(lam: np.ndarray, sigma: float) -> int:
    """nu(sigma) = #{lambda_i < sigma}."""
    return int(np.sum(np.asarray(lam) < sigma))


def slice_members(lam: np.ndarray, lo: float, hi: float) -> np.ndarray:
    """Indices i with lo < lambda_i <= hi."""
    lam = np.asarray(lam)
    return np.nonzero((lam > lo) & (lam <= hi))[0]


def csr_norm1(rowptr, colind, vals, n) -> float:
    """||M||_1 = max column abs-sum (= ||M||_inf for symmetric M)."""
    s = np.zeros(n)
    np.add.at(s, colind, np.abs(vals))
    return float(s.max()) if n else 0.0


def residual_norms(pencil, lam, X):
    """||A x_i - lambda_i B x_i||_2 / (||A||_1 ||x_i||_2) for each column of X (N x k)."""
    X = np.asarray(X, dtype=np.float64)
    AX = dense.csr_mm(pencil.rowptr, pencil.colind, pencil.a, X)
    BX = dense.csr_mm(pencil.rowptr, pencil.colind, pencil.b, X)
    R = AX - BX * np.asarray(lam)[None, :]
    na = csr_norm1(pencil.rowptr, pencil.colind, pencil.a, pencil.n)
    return np.linalg.norm(R, axis=0) / (na * np.linalg.norm(X, axis=0))


def b_orthonormality_error(pencil, X) -> float:
    """max |X^T B X - I|."""
    BX = dense.csr_mm(pencil.rowptr, pencil.colind, pencil.b, X)
    G = np.asarray(X).T @ BX
    return float(np.abs(G - np.eye(G.shape[0])).max())


def rayleigh_quotients(pencil, X):
    """x^T A x / x^T B x for each column x of X, with the products on the stored CSR."""
    X = np.asarray(X, dtype=np.float64)
    AX = dense.csr_mm(pencil.rowptr, pencil.colind, pencil.a, X)
    BX = dense.csr_mm(pencil.rowptr, pencil.colind, pencil.b, X)
    return np.einsum("ij,ij->j", X, AX) / np.einsum("ij,ij->j", X, BX)


def lowest_eigenpairs(pencil, m: int):
    """The m lowest eigenvalues of the pencil and their B-normalised eigenvectors: the
    reduced solver's eigenvectors (dense.gen_eig_lowest), each eigenvalue taken as the
    Rayleigh quotient of its vector on the original pencil.  Returned in ascending
    order of the quotient."""
    _, X = dense.gen_eig_lowest(pencil.dense("a"), pencil.dense("b"), m)
    lam = rayleigh_quotients(pencil, X)
    order = np.argsort(lam, kind="stable")
    return lam[order], X[:, order]


def dense_pencil_eig(pencil, vectors=True):
    """All eigenpairs of the pencil from the dense oracle solver."""
    return dense.gen_eig(pencil.dense("a"), pencil.dense("b"), vectors=vectors)


def band_of(pencil, sigma: float):
    """Lower band of A - sigma B in natural order: band[j, t] = M[j+t, j]."""
    rows = pencil.rows()
    cols = pencil.colind.astype(np.int64)
    low = rows >= cols
    bw = int((rows[low] - cols[low]).max()) if low.any() else 0
    band = np.zeros((pencil.n, bw + 1))
    band[cols[low], rows[low] - cols[low]] = pencil.a[low] - sigma * pencil.b[low]
    return band


def band_inertia(pencil, sigma: float):
    """(neg, zero, pos) of A - sigma B by unpivoted band LDL^T, with the pivot ratio."""
    inert, rmin, rc = dense.band_ldlt(band_of(pencil, sigma))
    return inert, rmin, rc
