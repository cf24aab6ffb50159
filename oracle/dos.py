"""Lanczos density-of-states estimate and closed-form DOS/CDOS (Section 3.1).

Test infrastructure only.  Follows the paper's steps in order:

1. B-orthonormal Lanczos on B^-1 A (the second form of Section 3.1, the one whose
   N(0,1) start vector the paper describes), start vector passed in, k steps, full
   re-orthogonalisation (the paper does not say; we take full re-orthogonalisation).
2. Ritz pairs (theta_j, g_j) of the Lanczos tridiagonal, zeta_j = e_1^T g_j (Eq. 4).
3. Gaussian widths nu_j: d_j = max of the neighbour gaps (one gap at the ends), floored
   at 1e-3 (theta_max - theta_min)/k, nu_j = d_j / 3 (our reading of "nearly vanishes").
4. phi(omega) = N/sqrt(2 pi) sum zeta_j^2/nu_j exp(-kappa_j^2),
   kappa_j = (omega - theta_j)/(nu_j sqrt 2) (Eq. 4);
   Phi(omega) = N/2 sum zeta_j^2 [erf(kappa_j) + 1] (Eq. 5);
   several start vectors are averaged.
5. psi_i(omega) = theta_i/2 erf(kappa_i) - nu_i/sqrt(2 pi) exp(-kappa_i^2) and the
   expectation shift sigma = N/(Phi(u) - Phi(l)) sum zeta_i^2 (psi_i(u) - psi_i(l))
   (Eqs. 7-8).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
from scipy.special import erf

from . import dense


def lanczos_ritz(A: np.ndarray, B: np.ndarray, x0: np.ndarray, k: int):
    """k-step B-orthonormal Lanczos on B^-1 A from start vector x0 (Section 3.1).

    x_1 = x0 / ||x0||_B; w = B^-1 A x_j - alpha_j x_j - beta_{j-1} x_{j-1} with
    alpha_j = x_j^T A x_j; full re-orthogonalisation in the B inner product; beta_j =
    ||w||_B.  Returns (theta, zeta2, alpha, beta); zeta_j = e_1^T g_j for the Ritz
    vectors g_j of the tridiagonal (Eq. 4).  This is Lanczos on L^-1 A L^-T started
    from L^T x0 for any B = L L^T."""
    n = A.shape[0]
    Lb = np.linalg.cholesky(B)
    def binv(v):
        return sla.solve_triangular(Lb, sla.solve_triangular(Lb, v, lower=True), lower=True, trans="T")
    k = min(k, n)
    X = np.zeros((n, k))
    alpha = np.zeros(k)
    beta = np.zeros(k)
    x = np.asarray(x0, dtype=np.float64)
    x = x / math.sqrt(x @ (B @ x))
    x_prev = np.zeros(n)
    b_prev = 0.0
    m = k
    for j in range(k):
        X[:, j] = x
        u = A @ x
        alpha[j] = x @ u
        w = binv(u) - alpha[j] * x - b_prev * x_prev
        for _ in range(2):                       # full re-orthogonalisation (B inner product)
            w = w - X[:, : j + 1] @ (X[:, : j + 1].T @ (B @ w))
        beta[j] = math.sqrt(max(w @ (B @ w), 0.0))
        if j + 1 < k and beta[j] <= 1e-13 * max(1.0, abs(alpha[j])):
            m = j + 1
            break
        x_prev, x, b_prev = x, w / beta[j], beta[j]
    theta, Z = dense.tridiag_eig(alpha[:m], beta[: m - 1], vectors=True)
    zeta2 = Z[0, :] ** 2
    return theta, zeta2, alpha[:m], beta[: m - 1]


def lanczos_ritz_cholesky_frame(A: np.ndarray, B: np.ndarray, y0: np.ndarray, k: int):
    """Lanczos on L^-1 A L^-T (B = L L^T, the Cholesky factor) started at y0: the same
    run as B-orthonormal Lanczos on B^-1 A from x0 = L^-T y0 (Section 3.1, first form)."""
    L = np.linalg.cholesky(B)
    x0 = sla.solve_triangular(L, np.asarray(y0, dtype=np.float64), lower=True, trans="T")
    return lanczos_ritz(A, B, x0, k)


def gaussian_widths(theta: np.ndarray) -> np.ndarray:
    """nu_j = d_j / 3, d_j = max neighbour gap (single gap at the ends), floored."""
    theta = np.asarray(theta, dtype=np.float64)
    m = theta.size
    if m == 1:
        return np.array([1.0])
    gaps = np.diff(theta)
    d = np.empty(m)
    d[0] = gaps[0]
    d[-1] = gaps[-1]
    for j in range(1, m - 1):
        d[j] = max(gaps[j - 1], gaps[j])
    floor = 1e-3 * (theta[-1] - theta[0]) / m
    d = np.maximum(d, floor)
    return d / 3.0


def dos_phi(omega, n, runs):
    """phi(omega) averaged over runs = [(theta, zeta2, nu), ...] (Eq. 4)."""
    omega = np.atleast_1d(np.asarray(omega, dtype=np.float64))
    tot = np.zeros_like(omega)
    for theta, zeta2, nu in runs:
        kap = (omega[:, None] - theta[None, :]) / (nu[None, :] * math.sqrt(2.0))
        tot += n / math.sqrt(2.0 * math.pi) * np.sum(zeta2[None, :] / nu[None, :] * np.exp(-kap * kap), axis=1)
    return tot / len(runs)


def cdos_Phi(omega, n, runs):
    """Phi(omega) averaged over runs (Eq. 5)."""
    omega = np.atleast_1d(np.asarray(omega, dtype=np.float64))
    tot = np.zeros_like(omega)
    for theta, zeta2, nu in runs:
        kap = (omega[:, None] - theta[None, :]) / (nu[None, :] * math.sqrt(2.0))
        tot += n / 2.0 * np.sum(zeta2[None, :] * (erf(kap) + 1.0), axis=1)
    return tot / len(runs)


def psi(omega, theta, nu):
    """psi_i(omega) for every Ritz value (Eq. 8); returns shape (len(omega), k)."""
    omega = np.atleast_1d(np.asarray(omega, dtype=np.float64))
    kap = (omega[:, None] - theta[None, :]) / (nu[None, :] * math.sqrt(2.0))
    return theta[None, :] / 2.0 * erf(kap) - nu[None, :] / math.sqrt(2.0 * math.pi) * np.exp(-kap * kap)


def expectation_shift(l, u, n, runs):
    """sigma = (integral_l^u omega phi) / (Phi(u) - Phi(l)) (Eq. 7), runs averaged."""
    num = 0.0
    for theta, zeta2, nu in runs:
        ps = psi(np.array([l, u]), theta, nu)
        num += n * float(np.sum(zeta2 * (ps[1] - ps[0])))
    num /= len(runs)
    den = float(cdos_Phi(u, n, runs)[0] - cdos_Phi(l, n, runs)[0])
    return num / den
