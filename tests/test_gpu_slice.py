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
