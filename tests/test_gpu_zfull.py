"""End-to-end parity at the benchmark size (N = 16,384, n_e = 1,640, 16 shifts, mixed
precision, the launch configuration bench.py times): every delivered eigenvalue against the
dense-oracle golden eigenvalues, the count below lambda_max against the golden count, and
every residual recomputed by the oracle's SpMV.  Collected after the other GPU tests (it
takes about a minute)."""
import os

import numpy as np
import pytest
import torch

from oracle import spectral
from tests.gpu_util import setup
from workloads.pencils import config_pencil, normal_block

pytestmark = pytest.mark.gpu


def test_gauss16_all_slices_match_dense_golden(gpu_lib):
    from paper_1908_06043_gb300.driver import DosModel, SliceSolver
    path = os.path.join(os.path.dirname(__file__), "golden", "gauss16_eigs.txt")
    lam = np.array([float(l) for l in open(path) if not l.startswith("#")])
    p = config_pencil(2)
    ctx, sym, a, b = setup(gpu_lib, p)
    start = torch.tensor(normal_block(p.n, 4, 1000), device="cuda")
    model = DosModel(p.n, sym.dos_estimate(a, b, 100, start))
    solver = SliceSolver(sym, a, b, precision="mixed")
    lam_min, lam_max, shifts, splits, ks = solver.place_shifts(model, 1640, 16)
    res = solver.run(shifts, lam_min, lam_max, model, seed=0, splits=splits, ks=ks)
    assert res.timings["converged"]
    n_below = spectral.count_below(lam, lam_max)
    assert n_below < lam.size                       # the golden list reaches past lambda_max
    assert res.timings["n_below_max"] == n_below
    assert res.eigenvalues.size == n_below
    ref = lam[:n_below]
    assert np.all(np.abs(res.eigenvalues - ref) <= 1e-10 * np.maximum(np.abs(ref), 1.0))
    X = res.eigenvectors.cpu().numpy()
    assert spectral.residual_norms(p, res.eigenvalues, X).max() <= 1e-10
