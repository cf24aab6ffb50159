"""Helpers shared by the GPU tests (device copies of the seeded pencils)."""
import numpy as np
import torch


def to_dev(p):
    a = torch.tensor(p.a, dtype=torch.float64, device="cuda")
    b = torch.tensor(p.b, dtype=torch.float64, device="cuda")
    return a, b


def setup(api, p, nd_leaf=0):
    ctx = api.Context(0)
    sym = ctx.analyze(p.rowptr, p.colind, nd_leaf=nd_leaf)
    a, b = to_dev(p)
    return ctx, sym, a, b


def mid_gap_shifts(lam, idx):
    """Shifts halfway between eigenvalues idx and idx+1 (well away from the spectrum)."""
    lam = np.asarray(lam)
    return [0.5 * (lam[i] + lam[i + 1]) for i in idx]
