"""Pins for the band-energy gradient: closed form on the 1D Laplacian and central
finite differences on a small Gaussian pencil (Hellmann-Feynman)."""
import numpy as np

from oracle import dense, grad
from workloads.pencils import gaussian_pencil, laplacian_1d


def test_laplacian_diagonal_gradient_closed_form():
    n, ne = 30, 7
    p = laplacian_1d(n)
    lam, X = dense.gen_eig(p.dense("a"), p.dense("b"))
    ga, gb = grad.band_energy_grad(p, lam[:ne], X[:, :ne])
    rows = p.rows()
    diag = rows == p.colind
    j = np.arange(1, n + 1)
    ex = sum(2.0 / (n + 1) * np.sin(j * k * np.pi / (n + 1)) ** 2 for k in range(1, ne + 1))
    assert np.allclose(ga[diag], ex, atol=1e-12)
    assert np.allclose(gb[diag], -sum(lam[k - 1] * 2.0 / (n + 1) * np.sin(j * k * np.pi / (n + 1)) ** 2
                                       for k in range(1, ne + 1)), atol=1e-12)


def test_finite_differences_gaussian():
    p = gaussian_pencil((2, 2, 2), seed=13)
    ne = 9
    A0, B0 = p.dense("a"), p.dense("b")
    lam, X = dense.gen_eig(A0, B0)
    ga, gb = grad.band_energy_grad(p, lam[:ne], X[:, :ne])
    rows, cols = p.rows(), p.colind
    rng = np.random.default_rng(5)
    h = 1e-6
    for e in rng.choice(p.nnz, 12, replace=False):
        r, c = rows[e], cols[e]
        E = np.zeros((p.n, p.n))
        E[r, c] = 1.0
        E[c, r] = 1.0
        mult = 1.0 if r == c else 2.0
        for which, g in (("a", ga), ("b", gb)):
            Ap = A0 + h * E if which == "a" else A0
            Am = A0 - h * E if which == "a" else A0
            Bp = B0 + h * E if which == "b" else B0
            Bm = B0 - h * E if which == "b" else B0
            Ep = dense.gen_eig(Ap, Bp, vectors=False)[0][:ne].sum()
            Em = dense.gen_eig(Am, Bm, vectors=False)[0][:ne].sum()
            fd = (Ep - Em) / (2 * h)
            assert abs(fd - mult * g[e]) < 1e-6 * max(1.0, abs(fd))
