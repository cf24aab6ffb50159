"""Pins for the DOS / CDOS oracle (Section 3.1, Eqs. 4-8)."""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import dense, dos, partition
from workloads.pencils import gaussian_pencil, laplacian_1d, normal_block


def _runs(p, k, nv, seed):
    A, B = p.dense("a"), p.dense("b")
    X0 = normal_block(p.n, nv, seed)
    out = []
    for v in range(nv):
        th, z2, _, _ = dos.lanczos_ritz(A, B, X0[:, v], k)
        out.append((th, z2, dos.gaussian_widths(th)))
    return out


def test_zeta_sum_and_cdos_limits():
    p = gaussian_pencil((3, 3, 3), seed=5)
    runs = _runs(p, 30, 2, 1)
    for th, z2, nu in runs:
        assert abs(z2.sum() - 1.0) < 1e-12            # sum zeta^2 = |e_1|^2
    assert abs(dos.cdos_Phi(1e6, p.n, runs)[0] - p.n) < 1e-9 * p.n    # Phi(+inf) = N
    assert abs(dos.cdos_Phi(-1e6, p.n, runs)[0]) < 1e-9


def test_full_lanczos_reproduces_spectrum_and_weights():
    p = gaussian_pencil((2, 2, 3), seed=9)
    A, B = p.dense("a"), p.dense("b")
    x0 = normal_block(p.n, 1, 4)[:, 0]
    th, z2, _, _ = dos.lanczos_ritz(A, B, x0, p.n)
    lam, X = dense.gen_eig(A, B)
    assert np.allclose(th, lam, atol=1e-9 * np.abs(lam).max())
    # zeta_j^2 = (x_j^T B x_1)^2 for the B-orthonormal eigenvectors x_j and the
    # B-normalised start vector x_1
    x1 = x0 / np.sqrt(x0 @ B @ x0)
    w = (X.T @ B @ x1) ** 2
    assert np.allclose(z2, w, atol=1e-9)


def test_phi_integrates_to_Phi_and_expectation_shift():
    p = gaussian_pencil((3, 3, 2), seed=2)
    runs = _runs(p, 25, 3, 2)
    lo, hi = runs[0][0][3], runs[0][0][15]
    integ, _ = quad(lambda w: dos.dos_phi(w, p.n, runs)[0], lo, hi, limit=400, epsabs=1e-10)
    dPhi = dos.cdos_Phi(hi, p.n, runs)[0] - dos.cdos_Phi(lo, p.n, runs)[0]
    assert abs(integ - dPhi) < 1e-7 * max(1, dPhi)
    num, _ = quad(lambda w: w * dos.dos_phi(w, p.n, runs)[0], lo, hi, limit=400, epsabs=1e-10)
    assert abs(dos.expectation_shift(lo, hi, p.n, runs) - num / integ) < 1e-7 * (1 + abs(num / integ))


def test_average_cdos_approaches_exact_count():
    p = laplacian_1d(120)
    lam = np.sort(2 - 2 * np.cos(np.arange(1, 121) * np.pi / 121))
    runs = _runs(p, 40, 64, 7)
    for w in (0.5, 1.0, 2.0, 3.0):
        est = dos.cdos_Phi(w, p.n, runs)[0]
        exact = (lam < w).sum()
        assert abs(est - exact) < 0.15 * p.n / math.sqrt(8)    # statistical: ~1/sqrt(n_v)


def test_widths_rule():
    th = np.array([0.0, 1.0, 1.5, 4.0])
    nu = dos.gaussian_widths(th)
    assert np.allclose(nu, np.array([1.0, 1.0, 2.5, 2.5]) / 3)
    th = np.array([0.0, 0.0, 1.0])
    assert dos.gaussian_widths(th)[0] == pytest.approx(1e-3 * 1.0 / 3 / 3)


def test_uniform_spectrum_gives_equispaced_shifts():
    # Ritz values on a uniform grid with equal weights (a flat DOS): the CDOS roots
    # are equally spaced, as the printed shifts of Section 5 are.
    m = 400
    th = np.linspace(-1.0, 1.0, m)
    runs = [(th, np.full(m, 1.0 / m), dos.gaussian_widths(th))]
    iv = partition.cdos_root_intervals(-0.5, 0.5, 10, 1000, runs)
    widths = np.array([u - l for l, u in iv])
    assert np.allclose(widths, 0.1, rtol=2e-3)
    shifts = [dos.expectation_shift(l, u, 1000, runs) for l, u in iv]
    assert np.allclose(shifts, [0.5 * (l + u) for l, u in iv], atol=1e-3)


def test_cholesky_frame_start_is_unbiased_on_gaussian_pencil():
    # with an N(0,1) start in the Cholesky frame the averaged CDOS tracks the exact count
    # even though B is ill-conditioned (an i.i.d. start in the original basis does not)
    from workloads.pencils import config_pencil
    p = config_pencil(1)
    A, B = p.dense("a"), p.dense("b")
    lam, _ = dense.gen_eig(A, B, vectors=False)
    Y = normal_block(p.n, 16, 8)
    runs = []
    for c in range(16):
        th, z2, _, _ = dos.lanczos_ritz_cholesky_frame(A, B, Y[:, c], 60)
        runs.append((th, z2, dos.gaussian_widths(th)))
    for i in (20, 86, 300):
        w = 0.5 * (lam[i] + lam[i + 1])
        assert abs(dos.cdos_Phi(w, p.n, runs)[0] - (i + 1)) <= 0.1 * (i + 1) + 4
