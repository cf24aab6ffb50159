"""GPU parity of the whole slicing driver against the dense oracle: DOS shift placement,
batched factorisation, probes and validation for the lowest n_e eigenpairs of one pencil,
and the SCF-like pencil sequence with k-means probe migration (Section 3.2)."""
import numpy as np
import pytest
import torch

from oracle import dense, partition, spectral
from tests.gpu_util import setup
from workloads.pencils import config_pencil, normal_block, scf_pencil, scf_sequence_perturbation

pytestmark = pytest.mark.gpu


def _check_lowest(p, res, n_e, tol=1e-10):
    lam, _ = dense.gen_eig(p.dense("a"), p.dense("b"), vectors=False)
    assert spectral.count_below(lam, res.lam_max) == n_e
    assert spectral.count_below(lam, res.lam_min) == 0
    assert res.eigenvalues.size == n_e
    ref = lam[:n_e]
    assert np.all(np.abs(res.eigenvalues - ref) <= 1e-10 * np.maximum(np.abs(ref), 1.0))
    X = res.eigenvectors.cpu().numpy()
    r = spectral.residual_norms(p, res.eigenvalues, X)
    assert r.max() <= tol
    # pairs from different probes are B-orthogonal up to their residuals over their gap:
    # (lambda_j - lambda_i) x_i^T B x_j = x_j^T r_i - x_i^T r_j
    G = X.T @ p.dense("b") @ X
    assert np.abs(np.diag(G) - 1.0).max() <= 1e-9
    na = np.abs(p.dense("a")).sum(axis=0).max()
    rn = r * na * np.linalg.norm(X, axis=0)                    # ||r_i||_2
    xn = np.linalg.norm(X, axis=0)
    gap = np.abs(res.eigenvalues[:, None] - res.eigenvalues[None, :])
    bound = (xn[None, :] * rn[:, None] + xn[:, None] * rn[None, :]) / np.where(gap > 0, gap, np.inf)
    off = np.abs(G - np.diag(np.diag(G)))
    assert np.all(off <= bound + 1e-10)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_config1_lowest_eigenpairs(gpu_lib, precision):
    from paper_1908_06043_gb300.driver import DosModel, SliceSolver
    p = config_pencil(1)
    ctx, sym, a, b = setup(gpu_lib, p)
    start = torch.tensor(normal_block(p.n, 4, 1000), device="cuda")
    model = DosModel(p.n, sym.dos_estimate(a, b, 100, start))
    solver = SliceSolver(sym, a, b, precision=precision)
    lam_min, lam_max, shifts, splits, ks = solver.place_shifts(model, 86, 4)
    res = solver.run(shifts, lam_min, lam_max, model, splits=splits, ks=ks)
    assert res.timings["converged"]
    # the region holds n_e = 86 eigenvalues up to the DOS margin
    _check_lowest(p, res, res.timings["n_below_max"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_scf_sequence_with_probe_migration(gpu_lib, precision):
    # A_i = A_0 + 0.1 2^-i R, R seeded U(-1, 1) on A's pattern; the shifts of step i > 0
    # come from k-means of step i-1's validated eigenvalues and must equal the oracle's
    # migration of the same data; every step must reproduce the dense eigenvalues
    from paper_1908_06043_gb300.driver import solve_sequence
    p0 = config_pencil(1)
    r = scf_sequence_perturbation(p0, seed=33)
    pencils = [scf_pencil(p0, r, i) for i in range(3)]
    ctx, sym, _, b = setup(gpu_lib, pencils[0])
    a_list = [torch.tensor(q.a, device="cuda") for q in pencils]
    uniforms = np.random.default_rng(7).random(4)
    res = solve_sequence(sym, a_list, b, 86, 4, precision=precision, uniforms=uniforms,
                         start=torch.tensor(normal_block(p0.n, 4, 1000), device="cuda"))
    for i, (q, rs) in enumerate(zip(pencils, res)):
        assert rs.timings["converged"], (i, rs.slices, rs.shifts, rs.timings["iterations"],
                                         rs.timings["basis_growth"], rs.timings["migration"])
        _check_lowest(q, rs, 86)
        if i == 0:
            continue
        prev = res[i - 1]
        after_dos = prev.timings["migration"] is None
        init = partition.kmeans_pp_init(prev.eigenvalues, 4, uniforms) if after_dos else np.asarray(prev.shifts)
        ref = partition.migrate(prev.eigenvalues, prev.owners, prev.shifts, init,
                                balance=rs.timings["migration"]["balance"])
        got = rs.timings["migration"]["shifts"]
        assert len(got) == len(ref)
        assert np.allclose(got, [s for s, _ in ref], rtol=1e-12, atol=1e-12)
        assert rs.timings["migration"]["sizes"] == [len(m) for _, m in ref]


def test_config1_dos_cluster_placement(gpu_lib):
    # Alg. 3 placement (clusters of the DOS, expectation shifts) through the whole driver
    from paper_1908_06043_gb300.driver import DosModel, SliceSolver
    p = config_pencil(1)
    ctx, sym, a, b = setup(gpu_lib, p)
    start = torch.tensor(normal_block(p.n, 4, 1000), device="cuda")
    model = DosModel(p.n, sym.dos_estimate(a, b, 100, start))
    solver = SliceSolver(sym, a, b, precision="fp64")
    lam_min, lam_max, shifts, splits, ks = solver.place_shifts(model, 86, 4, mode="cluster")
    assert len(shifts) == 4 and all(lam_min < s_ < lam_max for s_ in shifts)
    res = solver.run(shifts, lam_min, lam_max, model, splits=splits, ks=ks)
    assert res.timings["converged"]
    _check_lowest(p, res, res.timings["n_below_max"])


def test_missing_eigenvalues_recovered_by_probe_insertion(gpu_lib):
    # host-side fault injection (Section 3.3): all four shifts misplaced at the top of the
    # region and too few rounds for the low slices; validation reports missing
    # eigenvalues and the inserted probes recover them
    from paper_1908_06043_gb300.driver import DosModel, SliceSolver
    p = config_pencil(1)
    lam, _ = dense.gen_eig(p.dense("a"), p.dense("b"), vectors=False)
    ctx, sym, a, b = setup(gpu_lib, p)
    start = torch.tensor(normal_block(p.n, 4, 1000), device="cuda")
    model = DosModel(p.n, sym.dos_estimate(a, b, 100, start))
    solver = SliceSolver(sym, a, b, precision="fp64")
    lam_min = float(lam[0]) - 1.0
    lam_max = 0.5 * float(lam[85] + lam[86])
    shifts = list(0.5 * (lam[[80, 82, 83]] + lam[[81, 83, 84]])) + [0.5 * float(lam[84] + lam[85])]
    res = solver.run_with_recovery(shifts, lam_min, lam_max, model, max_inserts=4, max_rounds=8)
    assert res.timings["inserted"] and len(res.shifts) > 4     # the first attempt missed some
    assert res.timings["converged"], (res.slices, res.timings["inserted"])
    _check_lowest(p, res, 86)


def test_eta_monitor_trace_form(gpu_lib):
    # Eq. 9: Tr(X^T A X) of the library's SpMM against the dense form, and for
    # B-orthonormal eigenvectors equal to the sum of their eigenvalues
    from paper_1908_06043_gb300.driver import trace_form
    p = config_pencil(1)
    lam, X = dense.gen_eig(p.dense("a"), p.dense("b"))
    ctx, sym, a, b = setup(gpu_lib, p)
    Xd = torch.tensor(np.ascontiguousarray(X[:, :86]), device="cuda")
    eta = trace_form(sym, a, Xd)
    assert abs(eta - float(np.trace(X[:, :86].T @ p.dense("a") @ X[:, :86]))) <= 1e-10 * abs(eta)
    assert abs(eta - float(lam[:86].sum())) <= 1e-9 * max(1.0, abs(eta))


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_tc"])
def test_config1_slice_at_a_time(gpu_lib, precision):
    """plan_slices + solve_slice (the benchmark's unit of work): every window's eigenpairs
    against the dense oracle -- membership exact, eigenvalues to 1e-10, residuals by the
    oracle's SpMV, the window's validation flag."""
    from paper_1908_06043_gb300.driver import DosModel, SliceSolver, plan_slices, solve_slice
    p = config_pencil(1)
    ctx, sym, a, b = setup(gpu_lib, p)
    lam, _ = dense.gen_eig(p.dense("a"), p.dense("b"), vectors=False)
    start = torch.tensor(normal_block(p.n, 4, 1000), device="cuda")
    model = DosModel(p.n, sym.dos_estimate(a, b, 100, start))
    solver = SliceSolver(sym, a, b, precision=precision)
    plan = plan_slices(solver, model, 86, 4)
    assert plan.counts == [spectral.count_below(lam, x) for x in plan.bounds]
    assert plan.counts[0] == 0
    for j in range(4):
        o = solve_slice(solver, plan, j, seed=j)
        lo, hi = plan.window(j)
        ref = lam[spectral.slice_members(lam, lo, hi)]
        assert o.ok and o.n_exact == ref.size == o.theta.size
        assert o.n_neg_sigma == spectral.count_below(lam, plan.shifts[j])
        assert np.all(np.abs(o.theta - ref) <= 1e-10 * np.maximum(np.abs(ref), 1.0))
        r = spectral.residual_norms(p, o.theta, o.X.cpu().numpy())
        assert r.max() <= 1e-10
