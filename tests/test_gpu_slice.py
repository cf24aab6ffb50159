"""GPU parity of the in-slice solver (Alg. 2) against the dense oracle: slice
membership bit-exact, eigenvalues to 1e-10 relative, residuals <= 1e-10, X^T B X = I."""
import numpy as np
import pytest
import torch

from oracle import dense, spectral
from tests.gpu_util import setup
from workloads.pencils import config_pencil, laplacian_1d, normal_block

pytestmark = pytest.mark.gpu


def _check_probe(p, lam, lo, hi, pr, tol=1e-10):
    # converged Ritz values in the window are exactly the slice's eigenvalues
    inside = (pr.theta > lo) & (pr.theta <= hi) & (pr.resid <= tol)
    members = spectral.slice_members(lam, lo, hi)
    assert inside.sum() == members.size == pr.n_found
    th = pr.theta[inside]
    ref = lam[members]
    assert np.all(np.abs(th - ref) <= 1e-10 * np.maximum(np.abs(ref), 1.0))
    assert pr.resid[inside].max() <= tol
    X = pr.X.cpu().numpy()[:, inside]
    r = spectral.residual_norms(p, th, X)
    assert r.max() <= tol                                  # recomputed by the oracle SpMV
    assert spectral.b_orthonormality_error(p, X) <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_laplacian_slice(gpu_lib, precision):
    n = 400
    p = laplacian_1d(n, mass=True)
    th = np.arange(1, n + 1) * np.pi / (n + 1)
    lam = np.sort((2 - 2 * np.cos(th)) / ((4 + 2 * np.cos(th)) / 6))
    ctx, sym, a, b = setup(gpu_lib, p, nd_leaf=16)
    s = 0.5 * (lam[100] + lam[101])
    lo, hi = 0.5 * (lam[94] + lam[95]), 0.5 * (lam[106] + lam[107])
    f = sym.factor(a, b, [s], precision)
    V0 = torch.tensor(normal_block(n, 32, 1), device="cuda")
    pr = f.slice_solve(0, lo, hi, V0, max_iter=300, n_expect=12)
    assert pr.converged
    _check_probe(p, lam, lo, hi, pr)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_config1_probe(gpu_lib, precision):
    p = config_pencil(1)
    lam, _ = dense.gen_eig(p.dense("a"), p.dense("b"), vectors=False)
    ctx, sym, a, b = setup(gpu_lib, p)
    s = 0.5 * (lam[40] + lam[41])
    lo, hi = 0.5 * (lam[30] + lam[31]), 0.5 * (lam[50] + lam[51])
    f = sym.factor(a, b, [s], precision)
    V0 = torch.tensor(normal_block(p.n, 48, 11), device="cuda")
    pr = f.slice_solve(0, lo, hi, V0, max_iter=300, n_expect=20)
    assert pr.converged and pr.n_found == 20
    _check_probe(p, lam, lo, hi, pr)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_config1_block_lanczos_probe(gpu_lib, precision):
    p = config_pencil(1)
    lam, _ = dense.gen_eig(p.dense("a"), p.dense("b"), vectors=False)
    ctx, sym, a, b = setup(gpu_lib, p)
    s = 0.5 * (lam[60] + lam[61])
    lo, hi = 0.5 * (lam[45] + lam[46]), 0.5 * (lam[75] + lam[76])
    f = sym.factor(a, b, [s], precision)
    # Krylov extraction converges slowly at the edge of a wide window, so the first run
    # is followed by restarts from its Ritz vectors until the window validates
    V0 = torch.tensor(normal_block(p.n, 32, 5), device="cuda")
    pr = f.slice_solve(0, lo, hi, V0, driver="lanczos", max_iter=6, k_out=64, allow_noconv=True)
    assert pr.X.shape == (p.n, 64)
    for _ in range(40):
        if pr.n_found >= 30:
            break
        pr = f.slice_solve(0, lo, hi, pr.X, driver="lanczos", max_iter=2, k_out=64, allow_noconv=True)
    assert pr.n_found == 30
    _check_probe(p, lam, lo, hi, pr)


def test_laplacian_block_lanczos_restart(gpu_lib):
    # a first short Krylov run, then a restart from its Ritz vectors (two blocks)
    n = 600
    p = laplacian_1d(n)
    lam = np.sort(2 - 2 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1)))
    ctx, sym, a, b = setup(gpu_lib, p, nd_leaf=32)
    s = 0.5 * (lam[300] + lam[301])
    lo, hi = 0.5 * (lam[290] + lam[291]), 0.5 * (lam[310] + lam[311])
    f = sym.factor(a, b, [s], "mixed")
    V0 = torch.tensor(normal_block(n, 16, 6), device="cuda")
    pr = f.slice_solve(0, lo, hi, V0, driver="lanczos", max_iter=4, k_out=40, allow_noconv=True)
    for _ in range(40):
        if pr.n_found >= 20:
            break
        pr = f.slice_solve(0, lo, hi, pr.X, driver="lanczos", max_iter=2, k_out=40, allow_noconv=True)
    assert pr.n_found == 20
    _check_probe(p, lam, lo, hi, pr)


def _gauss16_golden():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "gauss16_eigs.txt")
    return np.array([float(l) for l in open(path) if not l.startswith("#")])


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_gauss16_probe_matches_dense_golden(gpu_lib, precision):
    # full-size pencil of the benchmark (N = 16,384): a 60-eigenvalue window around a
    # shift in the middle of the wanted region, against the dense-oracle eigenvalues
    from workloads.pencils import config_pencil
    lam = _gauss16_golden()
    p = config_pencil(2)
    ctx, sym, a, b = setup(gpu_lib, p)
    i = 1000
    s = 0.5 * (lam[i] + lam[i + 1])
    lo, hi = 0.5 * (lam[i - 31] + lam[i - 30]), 0.5 * (lam[i + 29] + lam[i + 30])
    f = sym.factor(a, b, [s], precision)
    assert f.inertia(0)[0] == i + 1
    V0 = torch.tensor(normal_block(p.n, 136, 9), device="cuda")
    pr = f.slice_solve(0, lo, hi, V0, n_expect=60, max_iter=80)
    inside = (pr.theta > lo) & (pr.theta <= hi) & (pr.resid <= 1e-10)
    ref = lam[(lam > lo) & (lam <= hi)]
    assert inside.sum() == ref.size == 60
    assert np.all(np.abs(pr.theta[inside] - ref) <= 1e-10 * np.maximum(np.abs(ref), 1.0))
    X = pr.X.cpu().numpy()[:, inside]
    assert spectral.residual_norms(p, pr.theta[inside], X).max() <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_config1_dense_pencil_path(gpu_lib, precision):
    # dense-pencil path: one front holding the whole N = 864 matrix (no dissection);
    # inertia and a probe against the dense oracle
    p = config_pencil(1)
    lam, _ = dense.gen_eig(p.dense("a"), p.dense("b"), vectors=False)
    ctx = gpu_lib.Context(0)
    sym = ctx.analyze(p.rowptr, p.colind, dense=True)
    assert sym.info["n_supernodes"] == 1 and sym.info["max_front"] == p.n
    a = torch.tensor(p.a, device="cuda")
    b = torch.tensor(p.b, device="cuda")
    sig = [0.5 * (lam[i] + lam[i + 1]) for i in (5, 40, 85, 431)]
    f = sym.factor(a, b, sig, precision)
    for j, i in enumerate((5, 40, 85, 431)):
        assert f.inertia(j)[0] == i + 1
    lo, hi = 0.5 * (lam[30] + lam[31]), 0.5 * (lam[50] + lam[51])
    pr = f.slice_solve(1, lo, hi, torch.tensor(normal_block(p.n, 48, 11), device="cuda"), max_iter=300,
                       n_expect=20)
    assert pr.converged and pr.n_found == 20
    _check_probe(p, lam, lo, hi, pr)
