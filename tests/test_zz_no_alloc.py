"""The allocation-free solve (ss_solve_noalloc) against the ordinary FP64 solve.

ss_solve_noalloc serves callers that cannot allocate device memory: it works in a
file-scope device array instead.  This file runs last (pytest collects files in
alphabetical order) so that a failure here cannot hide any other test; it also passes
on its own in a fresh process.  Two calls in a row check that the array's leftover
contents from the first call do not leak into the second.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from tests.gpu_util import setup
from workloads.pencils import config_pencil, normal_block

pytestmark = pytest.mark.gpu


def _noalloc(f, j, R):
    X = torch.empty_like(R)
    rc = f.ctx.lib.ss_solve_noalloc(f.h, j, C.c_void_p(R.data_ptr()), R.shape[1], C.c_void_p(X.data_ptr()))
    f.ctx.check(rc, "ss_solve_noalloc")
    return X


def test_noalloc_solve_matches_ss_solve_twice(gpu_lib):
    p = config_pencil(1)
    ctx, sym, a, b = setup(gpu_lib, p)
    f = sym.factor(a, b, [-0.3, 0.2], "fp64")
    for j, (k, seed) in enumerate([(24, 1), (7, 2)]):
        R = torch.tensor(normal_block(p.n, k, seed), device="cuda")
        ref = f.solve(j, R, refine=0)
        for _ in range(2):                      # two calls in a row share the scratch array
            X = _noalloc(f, j, R)
            torch.cuda.synchronize()
            # same kernels, but the solve sweeps scatter with atomics (summation order may
            # differ), amplified by the conditioning of A - sigma B
            assert ((X - ref).norm() / ref.norm()).item() <= 1e-9
            res = sym.spmm(a, b, X, 1.0, -f.sigma[j]) - R
            assert (res.norm() / R.norm()).item() <= 1e-8


def test_noalloc_in_place(gpu_lib):
    """R and X may be the same buffer: the right-hand sides are copied into the scratch
    array before anything is written to X."""
    p = config_pencil(1)
    ctx, sym, a, b = setup(gpu_lib, p)
    f = sym.factor(a, b, [0.2], "fp64")
    R = torch.tensor(normal_block(p.n, 12, 5), device="cuda")
    ref = f.solve(0, R, refine=0)
    RX = R.clone()
    rc = f.ctx.lib.ss_solve_noalloc(f.h, 0, C.c_void_p(RX.data_ptr()), RX.shape[1], C.c_void_p(RX.data_ptr()))
    f.ctx.check(rc, "ss_solve_noalloc")
    torch.cuda.synchronize()
    assert ((RX - ref).norm() / ref.norm()).item() <= 1e-9


def test_noalloc_rejects_oversized(gpu_lib):
    p = config_pencil(1)
    ctx, sym, a, b = setup(gpu_lib, p)
    f = sym.factor(a, b, [0.2], "fp64")
    # N k alone beyond the array
    too_many = 4_194_304 // p.n + 1
    R = torch.zeros((p.n, too_many), dtype=torch.float64, device="cuda")
    with pytest.raises(gpu_lib.SisliceError) as ei:
        _noalloc(f, 0, R)
    assert "exceeds" in str(ei.value)
    # N k fits, but the backward sweep's gather buffer (64 k per panel of the widest
    # solve level) does not
    fits = 4_194_304 // p.n
    R = torch.zeros((p.n, fits), dtype=torch.float64, device="cuda")
    with pytest.raises(gpu_lib.SisliceError) as ei:
        _noalloc(f, 0, R)
    assert "exceeds" in str(ei.value)
    # the context stays usable after a rejected call
    R = torch.tensor(normal_block(p.n, 4, 9), device="cuda")
    X = _noalloc(f, 0, R)
    torch.cuda.synchronize()
    ref = f.solve(0, R, refine=0)
    assert ((X - ref).norm() / ref.norm()).item() <= 1e-9
