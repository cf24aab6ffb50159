"""CPU tests of the C-ABI library: it loads, exports every declared symbol, and its
host-side symbolic analysis is consistent (no GPU calls)."""
import os
import re

import numpy as np
import pytest

from paper_1908_06043_gb300 import _lib as L
from paper_1908_06043_gb300 import api, build
from workloads.pencils import config_pencil, gaussian_pencil, laplacian_1d, random_sparse_pencil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "sislice.h")).read()
    return sorted(set(re.findall(r"^\s*(?:ss_status|const char \*)\s*(ss_\w+)\s*\(", txt, re.M)))


def test_exports_every_declared_symbol():
    lib = L.load()
    names = declared_symbols()
    assert len(names) >= 16
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) <= set(L.EXPORTS)


def test_host_only_context_refuses_device_calls():
    ctx = api.Context(-1)
    p = laplacian_1d(10)
    sym = ctx.analyze(p.rowptr, p.colind)
    import ctypes as C
    h = C.c_void_p()
    sig = np.zeros(1)
    rc = ctx.lib.ss_factor(sym.h, C.c_void_p(1), C.c_void_p(1), sig.ctypes.data_as(C.c_void_p), 1, 0, C.byref(h))
    assert rc == L.SS_ERR_ARG


@pytest.mark.parametrize("name", ["lap1", "lap2", "lap777", "gauss_small", "config1", "random", "gauss_thin"])
def test_symbolic_analysis_consistent(name):
    p = {"lap1": lambda: laplacian_1d(1), "lap2": lambda: laplacian_1d(2), "lap777": lambda: laplacian_1d(777),
         "gauss_small": lambda: gaussian_pencil((3, 4, 5), seed=2), "config1": lambda: config_pencil(1),
         "random": lambda: random_sparse_pencil(300, 0.01, 4),
         "gauss_thin": lambda: gaussian_pencil((40, 2, 2), seed=5)}[name]()
    ctx = api.Context(-1)
    sym = ctx.analyze(p.rowptr, p.colind)
    sym.validate()
    perm = sym.perm()
    assert np.array_equal(np.sort(perm), np.arange(p.n))
    inf = sym.info
    assert inf["n"] == p.n and inf["nnz"] == p.nnz
    assert inf["factor_entries"] >= (p.nnz + p.n) // 2
    assert inf["max_front"] <= p.n


def test_disconnected_components():
    a = laplacian_1d(50)
    # two disjoint copies of the same chain
    rowptr = np.concatenate([a.rowptr, a.rowptr[1:] + a.rowptr[-1]])
    colind = np.concatenate([a.colind, a.colind + 50]).astype(np.int32)
    ctx = api.Context(-1)
    sym = ctx.analyze(rowptr, colind, nd_leaf=8)
    sym.validate()
    assert sym.info["n"] == 100


def test_nested_dissection_reduces_fill_on_a_lattice():
    p = gaussian_pencil((12, 12, 12), seed=1)
    ctx = api.Context(-1)
    sym = ctx.analyze(p.rowptr, p.colind)
    sym.validate()
    # a dense LDL^T costs n^3/3 flops; the dissection ordering needs far fewer
    assert sym.info["factor_flops"] < 0.3 * p.n ** 3 / 3


@pytest.mark.parametrize("bad", ["unsorted", "asym", "nodiag", "range"])
def test_pattern_errors(bad):
    p = laplacian_1d(6)
    rowptr, colind = p.rowptr.copy(), p.colind.copy()
    if bad == "unsorted":
        colind[[0, 1]] = colind[[1, 0]]
    elif bad == "asym":
        colind[1] = 2                           # (0,2) without (2,0)
    elif bad == "nodiag":
        colind[0] = 1
        colind[1] = 1
        colind = colind
    elif bad == "range":
        colind[-1] = 99
    ctx = api.Context(-1)
    with pytest.raises(api.SisliceError) as ei:
        ctx.analyze(rowptr, colind)
    assert ei.value.status == L.SS_ERR_ARG
