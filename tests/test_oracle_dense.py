"""Pins for the dense oracle: closed forms, an outside library (LAPACK via scipy),
brute force on tiny inputs, and Sylvester's law (Section 2.2)."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import dense, spectral
from workloads.pencils import config_pencil, gaussian_pencil, laplacian_1d, random_sparse_pencil


@pytest.mark.parametrize("n", [1, 2, 7, 50, 201])
@pytest.mark.parametrize("mass", [False, True])
def test_laplacian_closed_form(n, mass):
    p = laplacian_1d(n, mass)
    lam, X = dense.gen_eig(p.dense("a"), p.dense("b"))
    th = np.arange(1, n + 1) * np.pi / (n + 1)
    ex = 2 - 2 * np.cos(th)
    if mass:
        ex = ex / ((4 + 2 * np.cos(th)) / 6)
    ex = np.sort(ex)
    assert np.allclose(lam, ex, rtol=0, atol=1e-12 * max(1, ex.max()))
    # eigenvectors are sin(j k pi/(n+1)) up to sign and B-normalisation
    j = np.arange(1, n + 1)
    order = np.argsort(2 - 2 * np.cos(th))
    for col, k in enumerate(order + 1):
        s = np.sin(j * k * np.pi / (n + 1))
        x = X[:, col]
        cosang = abs(s @ x) / (np.linalg.norm(s) * np.linalg.norm(x))
        assert cosang > 1 - 1e-10
    B = p.dense("b")
    assert np.abs(X.T @ B @ X - np.eye(n)).max() < 1e-12


@pytest.mark.parametrize("seed", range(6))
def test_tiny_vs_lapack(seed):
    n = 3 + seed
    p = random_sparse_pencil(n, 0.5, seed)
    lam, X = dense.gen_eig(p.dense("a"), p.dense("b"))
    w = sla.eigh(p.dense("a"), p.dense("b"), eigvals_only=True)
    assert np.allclose(lam, w, rtol=1e-12, atol=1e-12)


def test_gaussian_small_vs_lapack_and_residual():
    p = gaussian_pencil((3, 3, 3), seed=7)
    A, B = p.dense("a"), p.dense("b")
    lam, X = dense.gen_eig(A, B)
    w = sla.eigh(A, B, eigvals_only=True)
    assert np.abs(lam - w).max() <= 1e-10 * np.abs(w).max()
    r = spectral.residual_norms(p, lam, X)
    assert r.max() < 1e-13
    assert spectral.b_orthonormality_error(p, X) < 1e-10


def test_config1_pencil_spd_and_vs_lapack():
    p = config_pencil(1)
    assert p.n == 864
    B = p.dense("b")
    assert np.allclose(B, B.T) and np.allclose(p.dense("a"), p.dense("a").T)
    assert np.linalg.eigvalsh(B).min() > 0      # drop rule keeps S positive definite
    lam, X = dense.gen_eig(p.dense("a"), B)
    w = sla.eigh(p.dense("a"), B, eigvals_only=True)
    assert np.abs(lam - w).max() <= 1e-10 * np.abs(w).max()
    assert spectral.residual_norms(p, lam, X).max() < 1e-12


def test_not_spd_reported():
    A = np.eye(3)
    B = np.diag([1.0, -1.0, 1.0])
    with pytest.raises(np.linalg.LinAlgError):
        dense.gen_eig(A, B)


def test_tridiag_closed_form():
    m = 40
    th, Z = dense.tridiag_eig(2 * np.ones(m), -np.ones(m - 1))
    ex = np.sort(2 - 2 * np.cos(np.arange(1, m + 1) * np.pi / (m + 1)))
    assert np.allclose(th, ex, atol=1e-13)
    assert np.allclose(Z.T @ Z, np.eye(m), atol=1e-12)


def test_bk_two_by_two_pivots():
    # needs a 2x2 pivot at the first step; inertia (1, 0, 1)
    inert, kind, dv = dense.ldlt_bk(np.array([[0.0, 1.0], [1.0, 0.0]]))
    assert inert == (1, 0, 1) and kind[0] == 2
    inert, _, _ = dense.ldlt_bk(np.array([[1e-20, 1.0, 0], [1.0, 1e-20, 0], [0, 0, -3.0]]))
    assert inert == (2, 0, 1)
    inert, _, _ = dense.ldlt_bk(np.zeros((3, 3)))
    assert inert == (0, 3, 0)


@pytest.mark.parametrize("seed", range(8))
def test_bk_inertia_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    n = 1 + seed * 3
    M = rng.standard_normal((n, n))
    M = M + M.T
    if seed % 2:
        M[0, 0] = 0.0
    inert, _, _ = dense.ldlt_bk(M)
    ev = np.linalg.eigvalsh(M)
    assert inert == (int((ev < 0).sum()), 0, int((ev > 0).sum()))


def test_sylvester_inertia_equals_eigencount_config1():
    p = config_pencil(1)
    lam, _ = dense.gen_eig(p.dense("a"), p.dense("b"), vectors=False)
    A, B = p.dense("a"), p.dense("b")
    sigmas = list(0.5 * (lam[[0, 10, 85, 86, 400]] + lam[[1, 11, 86, 87, 401]])) + [-10.0, 100.0]
    for s in sigmas:
        inert, _, _ = dense.ldlt_bk(A - s * B)
        assert inert[0] == spectral.count_below(lam, s)
        assert inert[1] == 0 and inert[0] + inert[2] == p.n


def test_band_ldlt_matches_bk():
    p = gaussian_pencil((4, 4, 4), seed=11)
    lam, _ = dense.gen_eig(p.dense("a"), p.dense("b"), vectors=False)
    for s in [lam[0] - 1, 0.5 * (lam[20] + lam[21]), 0.5 * (lam[100] + lam[101]), lam[-1] + 1]:
        inert_b, rmin, rc = spectral.band_inertia(p, s)
        inert_d, _, _ = dense.ldlt_bk(p.dense("a") - s * p.dense("b"))
        assert rc == 0 and rmin > 1e-12
        assert inert_b == inert_d == (spectral.count_below(lam, s), 0, p.n - spectral.count_below(lam, s))


def test_csr_mm_matches_dense():
    p = gaussian_pencil((3, 2, 2), seed=3)
    X = np.random.default_rng(0).standard_normal((p.n, 5))
    assert np.allclose(dense.csr_mm(p.rowptr, p.colind, p.a, X), p.dense("a") @ X, atol=1e-13)


# ---- lowest eigenpairs: inverse iteration + back-transform + Rayleigh quotient (Eq. 1)
@pytest.mark.parametrize("mass", [False, True])
def test_lowest_eigenpairs_laplacian_closed_form(mass):
    n = 80
    p = laplacian_1d(n, mass=mass)
    lam, X = spectral.lowest_eigenpairs(p, 20)
    k = np.arange(1, 21)
    th = k * np.pi / (n + 1)
    ref = 2 - 2 * np.cos(th)
    if mass:
        ref = ref / ((4 + 2 * np.cos(th)) / 6)
    assert np.abs(lam - ref).max() <= 1e-13
    # eigenvectors are the sines, B-normalised (up to sign)
    j = np.arange(1, n + 1)
    B = p.dense("b")
    for c in range(20):
        s = np.sin(j * (c + 1) * np.pi / (n + 1))
        s /= np.sqrt(s @ B @ s)
        assert min(np.abs(X[:, c] - s).max(), np.abs(X[:, c] + s).max()) <= 1e-10


def test_lowest_eigenpairs_gaussian_vs_lapack():
    p = gaussian_pencil((3, 3, 3), seed=5)
    A, B = p.dense("a"), p.dense("b")
    lam, X = spectral.lowest_eigenpairs(p, 40)
    w = sla.eigh(A, B, eigvals_only=True)[:40]
    assert np.abs(lam - w).max() <= 1e-12 * max(1.0, np.abs(w).max())
    assert np.abs(X.T @ B @ X - np.eye(40)).max() <= 1e-10
    assert spectral.residual_norms(p, lam, X).max() <= 1e-12


def _ill_conditioned_pencil(n, seed, bmin):
    """B = Q diag(b) Q^T with b log-spaced in [bmin, 1], A = Q diag(lambda b) Q^T plus a
    small symmetric perturbation, lambda ~ U(-50, 10): the low eigenvectors are
    B-normalised with ||x||_2 up to about bmin^-1/2, as on the low tail of the Gaussian
    pencils."""
    from workloads.pencils import Pencil
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    b = np.logspace(np.log10(bmin), 0, n)
    a = rng.uniform(-50, 10, n) * b
    B = (Q * b) @ Q.T
    B = 0.5 * (B + B.T)
    E = 1e-3 * rng.standard_normal((n, n))
    A = (Q * a) @ Q.T + E + E.T
    A = 0.5 * (A + A.T)
    rows, cols = np.nonzero(np.ones((n, n)))
    rowptr = np.arange(0, n * n + 1, n, dtype=np.int64)
    return Pencil(n, rowptr, cols.astype(np.int32), A[rows, cols].copy(), B[rows, cols].copy())


@pytest.mark.parametrize("seed", [1, 2])
def test_lowest_eigenpairs_extended_precision_on_ill_conditioned_b(seed):
    """Against eigenvalues computed in 40-digit arithmetic (Cholesky reduction and a
    symmetric eigensolver in mpmath) on a pencil whose low eigenvectors have ||x||_2 of a
    few hundred at ||x||_B = 1."""
    mp = pytest.importorskip("mpmath")
    n, m = 32, 8
    p = _ill_conditioned_pencil(n, seed, 1e-6)
    mp.mp.dps = 40
    A = mp.matrix(p.dense("a").tolist())
    B = mp.matrix(p.dense("b").tolist())
    Li = mp.inverse(mp.cholesky(B))
    C = Li * A * Li.T
    C = (C + C.T) / 2
    ref = np.array(sorted(float(v) for v in mp.eigsy(C, eigvals_only=True)))[:m]
    lam, X = spectral.lowest_eigenpairs(p, m)
    assert np.abs(X).max() > 100.0
    rel = np.abs(lam - ref) / np.maximum(np.abs(ref), 1.0)
    assert rel.max() <= 1e-10, rel
