"""Band-energy gradient (Hellmann-Feynman, SDDMM backward) through torch.autograd:
against the dense oracle's gradient on the N = 864 pencil, against central finite
differences (h = 1e-6) of E on seeded stored entries of A and B of the N = 16,384 pencil,
and the non-differentiability report when lambda_(n_e+1) - lambda_(n_e) < 1e-8."""
import numpy as np
import pytest
import torch

from oracle import dense, grad
from tests.gpu_util import setup
from workloads.pencils import Pencil, config_pencil, laplacian_1d, normal_block

pytestmark = pytest.mark.gpu


def _plan(gpu_lib, p, n_e, n_s, sym, a, b):
    from paper_1908_06043_gb300.driver import DosModel, SliceSolver, plan_slices
    start = torch.tensor(normal_block(p.n, 4, 1000), device="cuda")
    model = DosModel(p.n, sym.dos_estimate(a, b, 100, start))
    solver = SliceSolver(sym, a, b, precision="fp64")
    return solver, plan_slices(solver, model, n_e, n_s)


def _energy_fn(sym, plan, seed=0):
    from paper_1908_06043_gb300.driver import SliceSolver, energy_differentiable, solve_plan

    def fn(a_vals, b_vals):
        sv = SliceSolver(sym, a_vals, b_vals, precision="fp64")
        lam, X, _ = solve_plan(sv, plan, seed=seed)
        return torch.tensor(lam, device="cuda"), X, energy_differentiable(sv, lam)
    return fn


def test_config1_autograd_gradient_matches_dense_oracle(gpu_lib):
    p = config_pencil(1)
    ctx, sym, a, b = setup(gpu_lib, p)
    solver, plan = _plan(gpu_lib, p, 86, 4, sym, a, b)
    n_e = plan.counts[-1]
    ap = a.clone().requires_grad_(True)
    bp = b.clone().requires_grad_(True)
    E = gpu_lib.BandEnergy.apply(ap, bp, sym, _energy_fn(sym, plan))
    E.backward()
    lam_o, X_o = dense.gen_eig(p.dense("a"), p.dense("b"))
    assert abs(E.item() - lam_o[:n_e].sum()) <= 1e-10 * np.abs(lam_o[:n_e]).sum()
    ga_o, gb_o = grad.band_energy_grad(p, lam_o[:n_e], X_o[:, :n_e])
    # the gradient is the projector onto the n_e eigenvectors: its error is the
    # eigenvectors' residual over the gap to lambda_(n_e+1)
    assert np.abs(ap.grad.cpu().numpy() - ga_o).max() <= 1e-7 * np.abs(ga_o).max()
    assert np.abs(bp.grad.cpu().numpy() - gb_o).max() <= 1e-7 * np.abs(gb_o).max()


def test_gauss16_gradient_central_finite_differences(gpu_lib):
    """64 seeded stored entries (p < q, each tying (p, q) and (q, p)), 32 of A and 32 of B:
    the sum of their gradients against one central difference of E along all of them
    together, and one entry of each matrix on its own."""
    from paper_1908_06043_gb300.driver import SliceSolver, solve_plan
    p = config_pencil(2)
    ctx, sym, a, b = setup(gpu_lib, p)
    solver, plan = _plan(gpu_lib, p, 1640, 16, sym, a, b)
    lam0, X0, outs = solve_plan(solver, plan, seed=1)
    ga, gb = sym.band_energy_grad(X0, torch.tensor(lam0, device="cuda"))
    ga, gb = ga.cpu().numpy(), gb.cpu().numpy()
    rows = p.rows()
    upper = np.flatnonzero(rows < p.colind)
    rng = np.random.default_rng(5)
    pick = rng.choice(upper, 64, replace=False)
    mirror = {}
    for e in pick:
        r, c = rows[e], p.colind[e]
        lo, hi = p.rowptr[c], p.rowptr[c + 1]
        mirror[e] = lo + int(np.searchsorted(p.colind[lo:hi], r))
    warm = [o.X for o in outs]
    h = 1e-6

    def energy(da, db):
        sv = SliceSolver(sym, a + da, b + db, precision="fp64")
        counts = sv.count_below(plan.bounds)
        assert counts == plan.counts             # the perturbation moves no eigenvalue across a bound
        lam, _, _ = solve_plan(sv, plan, seed=7, warm=warm, first_iters=12)
        return float(np.sum(lam))

    def direction(entries, signs):
        d = np.zeros(p.nnz)
        for e, sg in zip(entries, signs):
            d[e] += sg
            d[mirror[e]] += sg
        return torch.tensor(d, device="cuda")

    def check(entries, signs, on_a):
        d = direction(entries, signs)
        g = ga if on_a else gb
        exact = sum(sg * (g[e] + g[mirror[e]]) for e, sg in zip(entries, signs))
        z = torch.zeros_like(d)
        ep = energy(h * d, z) if on_a else energy(z, h * d)
        em = energy(-h * d, z) if on_a else energy(z, -h * d)
        fd = (ep - em) / (2 * h)
        # E is computed to about 1e-15 of sum |lambda| (double-double Rayleigh quotients),
        # so the difference carries ~ 1e-15 sum|lambda| / h; the truncation is O(h^2)
        tol = 2e-15 * np.abs(lam0).sum() / h + 1e-6 * abs(exact) + 1e-7
        assert abs(fd - exact) <= tol, (fd, exact, tol)

    signs = rng.choice([-1.0, 1.0], 64)
    check(pick[:32], signs[:32], True)
    check(pick[32:], signs[32:], False)
    check([pick[0]], [1.0], True)
    check([pick[32]], [1.0], False)


def test_band_energy_not_differentiable_at_a_degenerate_boundary(gpu_lib):
    """Two uncoupled copies of a 1D Laplacian (B = I): every eigenvalue is double, so the
    sum of the lowest 5 is not differentiable and the backward pass returns NaN, while the
    sum of the lowest 6 is."""
    from paper_1908_06043_gb300.driver import SliceSolver, energy_differentiable, solve_plan, plan_slices
    from paper_1908_06043_gb300.driver import SlicePlan
    q = laplacian_1d(40)
    n = 2 * q.n
    rowptr = np.concatenate([q.rowptr, q.rowptr[1:] + q.nnz]).astype(np.int64)
    colind = np.concatenate([q.colind, q.colind + q.n]).astype(np.int32)
    p = Pencil(n, rowptr, colind, np.concatenate([q.a, q.a]), np.concatenate([q.b, q.b]))
    ctx, sym, a, b = setup(gpu_lib, p)
    lam1 = 2 - 2 * np.cos(np.arange(1, 5) * np.pi / 41)
    for n_e, diff in ((5, False), (6, True)):
        solver = SliceSolver(sym, a, b, precision="fp64")
        bounds = [-0.5, 0.5 * (lam1[(n_e - 1) // 2] + lam1[(n_e - 1) // 2 + 1]) if n_e % 2 == 0 else lam1[n_e // 2] + 1e-12]
        counts = solver.count_below(bounds)
        plan = SlicePlan([0.5 * (bounds[0] + bounds[1])], bounds, counts, [32], bounds[0], bounds[1])
        lam, X, _ = solve_plan(solver, plan)
        assert lam.size == counts[1]
        if not diff:
            # lambda_5 = lambda_6: the 5 lowest are taken by the bound just above lambda_5's pair
            lam = lam[:5]
            X = X[:, :5].contiguous()
        assert energy_differentiable(solver, lam) == diff
        ap = a.clone().requires_grad_(True)
        bp = b.clone().requires_grad_(True)
        E = gpu_lib.BandEnergy.apply(ap, bp, sym, lambda av, bv: (torch.tensor(lam, device="cuda"), X,
                                                                     energy_differentiable(solver, lam)))
        E.backward()
        assert bool(torch.isnan(ap.grad).all()) == (not diff)
