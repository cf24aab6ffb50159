"""End-to-end parity at the benchmark size (N = 16,384, n_e = 1,640, 16 shifts, mixed
precision): every delivered eigenvalue against the golden eigenvalues of the dense
oracle (tests/golden/gauss16_eigs.txt: Rayleigh quotients of the oracle's eigenvectors),
the count below lambda_max against the golden count, and every residual recomputed by the
oracle's SpMV -- once through the batched driver (SliceSolver.run) and once slice by slice
in the launch configuration bench.py times (plan_slices + solve_slice).  Collected after
the other GPU tests (each takes about a minute)."""
import os

import numpy as np
import pytest
import torch

from oracle import spectral
from tests.gpu_util import setup
from workloads.pencils import config_pencil, normal_block

pytestmark = pytest.mark.gpu


def _golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "gauss16_eigs.txt")
    return np.array([float(l) for l in open(path) if not l.startswith("#")])


def _model(sym, a, b, n):
    from paper_1908_06043_gb300.driver import DosModel
    start = torch.tensor(normal_block(n, 4, 1000), device="cuda")
    return DosModel(n, sym.dos_estimate(a, b, 100, start))


def test_gauss16_all_slices_match_dense_golden(gpu_lib):
    from paper_1908_06043_gb300.driver import SliceSolver
    lam = _golden()
    p = config_pencil(2)
    ctx, sym, a, b = setup(gpu_lib, p)
    model = _model(sym, a, b, p.n)
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


@pytest.mark.parametrize("precision,gemm", [("mixed", "simt"), ("fp64", "simt"), ("mixed", "tensor")])
def test_gauss16_slice_solves_match_dense_golden(gpu_lib, precision, gemm):
    """The benchmark's step on a spread of windows (the sparse low tail, the body, the
    top): exact window counts from inertia against the golden, eigenvalues to 1e-10;
    the probes' dense products on the CUDA cores or on the tensor cores."""
    from paper_1908_06043_gb300.driver import SliceSolver, plan_slices, solve_slice
    lam = _golden()
    p = config_pencil(2)
    ctx, sym, a, b = setup(gpu_lib, p)
    ctx.set_gemm_mode(gemm)
    solver = SliceSolver(sym, a, b, precision=precision)
    plan = plan_slices(solver, _model(sym, a, b, p.n), 1640, 16)
    assert plan.counts[-1] < lam.size
    assert plan.counts == [spectral.count_below(lam, x) for x in plan.bounds]
    for j in (0, 1, 8, 15):
        o = solve_slice(solver, plan, j, seed=j)
        lo, hi = plan.window(j)
        ref = lam[spectral.slice_members(lam, lo, hi)]
        assert o.ok and o.theta.size == ref.size == o.n_exact
        assert o.n_neg_sigma == spectral.count_below(lam, plan.shifts[j])
        assert np.all(np.abs(o.theta - ref) <= 1e-10 * np.maximum(np.abs(ref), 1.0))
        assert spectral.residual_norms(p, o.theta, o.X.cpu().numpy()).max() <= 1e-10
