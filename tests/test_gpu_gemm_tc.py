"""The probes' FP64 products on the tensor cores (ss_set_gemm_mode "tensor"): the dense
Gram and tall products (Cholesky-QR and Rayleigh-Ritz, Alg. 2 steps 4-5) through
ss_dense_gram / ss_dense_gemm, and the sparse products A X, B X (Alg. 2 steps 3-5)
through ss_spmm, against numpy / scipy FP64 products.

Bound.  Every operand row is split exactly into digits of one scale fixed by its largest
entry, the leading digit products are summed exactly and the sum rounded once, so the
error of an entry is a few units of 2^-53 of K max|a_row| max|b_row| (K the reduction
length); numpy's own error is within K u (|A|^T |B|).  The tests allow
8 * 2^-53 K max|a_row| max|b_row| + 2 K u (|A|^T |B|) per entry -- a dropped digit
product, a wrong exponent, a misplaced tile or a lost piece is off by far more."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _tol(A, B):
    """A, B: K x m1, K x m2 (the reduction runs down the rows)."""
    K = A.shape[0]
    amax, bmax = np.abs(A).max(axis=0), np.abs(B).max(axis=0)
    return 8 * U * K * np.outer(amax, bmax) + 2 * K * U * (np.abs(A).T @ np.abs(B))


def _operand(rng, n, k, spread=20):
    """Normal entries with row and column scales 2^U(-spread, spread), a zero column and
    a zero row."""
    X = rng.standard_normal((n, k))
    X *= np.exp2(rng.integers(-spread, spread + 1, size=(n, 1)))
    X *= np.exp2(rng.integers(-spread // 2, spread // 2 + 1, size=(1, k)))
    X[:, k // 3] = 0.0
    X[n // 2, :] = 0.0
    return X


def _dev(x):
    return torch.tensor(x, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("n,k1,k2", [(5000, 100, 72), (2048, 48, 48), (16384, 160, 160), (4099, 257, 65)])
def test_gram_matches_fp64(gpu_lib, n, k1, k2):
    rng = np.random.default_rng(n + k1 + k2)
    X, Y = _operand(rng, n, k1), _operand(rng, n, k2)
    ctx = gpu_lib.Context(0)
    ctx.set_gemm_mode("tensor")
    ctx.profile(["gemm_tc", "gram"])
    G = ctx.dense_gram(_dev(X), _dev(Y)).cpu().numpy()
    assert ctx.profile_query("gemm_tc")[0] > 0 and ctx.profile_query("gram")[0] == 0
    ref = X.T @ Y
    assert np.all(np.abs(G - ref) <= _tol(X, Y))
    ctx.set_gemm_mode("simt")
    Gs = ctx.dense_gram(_dev(X), _dev(Y)).cpu().numpy()
    assert np.all(np.abs(Gs - ref) <= _tol(X, Y))


def test_gram_strided_operands_and_wide_range(gpu_lib):
    """Row strides above the width (views into wider blocks) and entries spanning 2^+-300
    along the reduction: the operand-row exponent and the strided reads."""
    rng = np.random.default_rng(7)
    n, k = 3000, 96
    W = rng.standard_normal((n, 2 * k + 5)) * np.exp2(rng.integers(-300, 300, size=(n, 1)))
    X, Y = W[:, :k], W[:, k + 5:]
    Xd = _dev(W)[:, :k]
    Yd = _dev(W)[:, k + 5:]
    ctx = gpu_lib.Context(0)
    ctx.set_gemm_mode("tensor")
    G = ctx.dense_gram(Xd, Yd).cpu().numpy()
    assert np.all(np.abs(G - X.T @ Y) <= _tol(X, Y))


@pytest.mark.parametrize("transq", [False, True])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-0.5, 1.5)])
def test_tall_product_matches_fp64(gpu_lib, transq, alpha, beta):
    rng = np.random.default_rng(11 + int(transq))
    n, k1, k2 = 6001, 130, 70
    X = _operand(rng, n, k1, spread=8)
    Qe = rng.standard_normal((k1, k2)) * np.exp2(rng.integers(-6, 7, size=(1, k2)))   # effective k1 x k2
    Q = np.ascontiguousarray(Qe.T) if transq else Qe
    Y0 = rng.standard_normal((n, k2))
    ctx = gpu_lib.Context(0)
    ctx.set_gemm_mode("tensor")
    Yd = _dev(Y0) if beta != 0.0 else torch.full((n, k2), float("nan"), dtype=torch.float64, device="cuda")
    ctx.profile(["gemm_tc", "gemm"])
    ctx.dense_gemm(_dev(X), _dev(Q), Yd, alpha=alpha, beta=beta, transq=transq)
    assert ctx.profile_query("gemm_tc")[0] > 0 and ctx.profile_query("gemm")[0] == 0
    Yt = Yd.cpu().numpy()
    ref = alpha * (X @ Qe) + (beta * Y0 if beta != 0.0 else 0.0)
    tol = abs(alpha) * _tol(X.T, Qe) + 4 * U * abs(beta) * np.abs(Y0)
    assert np.all(np.isfinite(Yt))                  # beta = 0 never read the NaNs
    assert np.all(np.abs(Yt - ref) <= tol)


def test_small_products_stay_on_cuda_cores(gpu_lib):
    """Below 2,048 rows or a small dimension of 48 the CUDA-core kernels run."""
    rng = np.random.default_rng(3)
    X, Y = rng.standard_normal((2047, 64)), rng.standard_normal((2047, 64))
    ctx = gpu_lib.Context(0)
    ctx.set_gemm_mode("tensor")
    ctx.profile(["gemm_tc", "gram"])
    G = ctx.dense_gram(_dev(X), _dev(Y)).cpu().numpy()
    assert ctx.profile_query("gemm_tc")[0] == 0 and ctx.profile_query("gram")[0] == 1
    assert np.all(np.abs(G - X.T @ Y) <= _tol(X, Y))
    X2 = rng.standard_normal((8192, 40))
    G2 = ctx.dense_gram(_dev(X2), _dev(X2)).cpu().numpy()
    assert ctx.profile_query("gemm_tc")[0] == 0
    assert np.all(np.abs(G2 - X2.T @ X2) <= _tol(X2, X2))


def test_empty_and_bad_arguments(gpu_lib):
    ctx = gpu_lib.Context(0)
    ctx.set_gemm_mode("tensor")
    X = torch.zeros(0, 64, dtype=torch.float64, device="cuda")
    G = ctx.dense_gram(X, X)
    assert torch.count_nonzero(G) == 0
    with pytest.raises(Exception):
        ctx.set_gemm_mode("int8")
    Xg = torch.zeros(4096, 64, dtype=torch.float64, device="cuda")
    Q = torch.zeros(32, 64, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        ctx.dense_gemm(Xg, Q, torch.zeros(4096, 64, dtype=torch.float64, device="cuda"))


# ---------------------------------------------------------------- sparse products
def _sparse_ref(p, vals, X):
    import scipy.sparse as sp
    M = sp.csr_matrix((vals, np.asarray(p.colind), np.asarray(p.rowptr)), shape=(p.n, p.n))
    Mabs = sp.csr_matrix((np.abs(vals), np.asarray(p.colind), np.asarray(p.rowptr)), shape=(p.n, p.n))
    nnz_row = np.diff(np.asarray(p.rowptr)).astype(np.float64)
    rmax = np.maximum.reduceat(np.abs(vals), np.asarray(p.rowptr)[:-1])
    xmax = np.abs(X).max(axis=0)
    tol = 8 * U * np.outer(nnz_row * rmax, xmax) + 2 * nnz_row[:, None] * U * (Mabs @ np.abs(X))
    return M @ X, tol


@pytest.mark.parametrize("k", [64, 100, 304])
def test_spmm_matches_fp64(gpu_lib, k):
    """Y = diag(alpha) A X + diag(beta) B X on the N = 16,384 Gaussian pencil, columns of X
    scaled by 2^+-40, against scipy's FP64 products."""
    from tests.gpu_util import setup
    from workloads.pencils import config_pencil
    p = config_pencil(2)
    ctx, sym, a, b = setup(gpu_lib, p)
    rng = np.random.default_rng(k)
    X = rng.standard_normal((p.n, k)) * np.exp2(rng.integers(-40, 41, size=(1, k)))
    X[:, 3] = 0.0
    al = rng.uniform(-2, 2, k)
    be = rng.uniform(-2, 2, k)
    ctx.set_gemm_mode("tensor")
    ctx.profile(["spmm_tc", "spmm"])
    Y = sym.spmm(a, b, _dev(X), al, be).cpu().numpy()
    assert ctx.profile_query("spmm_tc")[0] > 0 and ctx.profile_query("spmm")[0] == 0
    AX, ta = _sparse_ref(p, np.asarray(p.a), X)
    BX, tb = _sparse_ref(p, np.asarray(p.b), X)
    ref = al * AX + be * BX
    tol = np.abs(al) * ta + np.abs(be) * tb + 4 * U * (np.abs(al * AX) + np.abs(be * BX))
    assert np.all(np.abs(Y - ref) <= tol)
    YA = sym.spmm(a, b, _dev(X)).cpu().numpy()          # A alone
    assert np.all(np.abs(YA - AX) <= ta)


def test_spmm_zero_rows_and_small_k(gpu_lib):
    """A banded pattern whose values vanish on a whole 128-row tile and on scattered rows
    (rows of exponent zero give zero rows of Y), and k below 48 on the CUDA cores."""
    n, bw = 3001, 70
    rows, cols = [], []
    for i in range(n):
        for j in range(max(0, i - bw), min(n, i + bw + 1)):
            rows.append(i)
            cols.append(j)
    rows, cols = np.array(rows), np.array(cols)
    rowptr = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))]).astype(np.int64)
    rng = np.random.default_rng(5)
    vals = rng.standard_normal(rows.size)
    vals = 0.5 * (vals + vals[np.lexsort((rows, cols))])       # symmetric values
    dead = ((rows >= 256) & (rows < 384)) | (rows % 97 == 5)
    vals[dead] = 0.0
    ctx = gpu_lib.Context(0)
    sym = ctx.analyze(rowptr, cols.astype(np.int32))
    vd = torch.tensor(vals, device="cuda")
    X = rng.standard_normal((n, 80))
    ctx.set_gemm_mode("tensor")
    Y = sym.spmm(vd, vd, _dev(X)).cpu().numpy()
    p = type("P", (), {"n": n, "rowptr": rowptr, "colind": cols})()
    ref, tol = _sparse_ref(p, vals, X)
    assert np.all(Y[256:384] == 0.0) and np.all(Y[5::97] == 0.0)
    assert np.all(np.abs(Y - ref) <= tol)
    ctx.profile(["spmm_tc", "spmm"])
    Y2 = sym.spmm(vd, vd, _dev(X[:, :40])).cpu().numpy()
    assert ctx.profile_query("spmm_tc")[0] == 0 and ctx.profile_query("spmm")[0] == 1
    assert np.all(np.abs(Y2 - ref[:, :40]) <= tol[:, :40])
