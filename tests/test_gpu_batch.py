"""GPU parity of the batched factorisation of many pencils (Alg. 2 step 2 over a batch of
independent pencils of uneven size, Section 2.2 inertia per pencil): the pencils stacked
into one block-diagonal pattern, each factored at its own shifts in the same launches, and
each pencil's inertia compared bit-exactly with the oracle's eigenvalue count below its
shift."""
import numpy as np
import pytest
import torch

from oracle import dense, spectral
from tests.gpu_util import mid_gap_shifts, setup
from workloads.pencils import (EXPONENTS_2, EXPONENTS_4, gaussian_pencil, laplacian_1d, stack_pencils,
                               uneven_batch_specs, batch_pencils)

pytestmark = pytest.mark.gpu


def _small_batch():
    return [gaussian_pencil((4, 5, 6), EXPONENTS_2, seed=11), laplacian_1d(300, mass=True),
            gaussian_pencil((6, 6, 6), EXPONENTS_4, seed=12), gaussian_pencil((3, 7, 5), EXPONENTS_4, seed=13)]


def test_stacked_pencils_inertia_per_pencil(gpu_lib):
    ps = _small_batch()
    st, seg, offs = stack_pencils(ps)
    lams = [dense.gen_eig(q.dense("a"), q.dense("b"), vectors=False)[0] for q in ps]
    ctx, sym, a, b = setup(gpu_lib, st)
    # three call slots: each pencil at its own mid-gap shift (different eigenvalue indices,
    # so every pencil's count differs between slots), and one slot below every spectrum
    picks = [[3, q.n // 2, q.n - 5] for q in ps]
    sig = np.array([[mid_gap_shifts(lams[p], [picks[p][j]])[0] for p in range(len(ps))] for j in range(3)]
                   + [[lams[p][0] - 1.0 for p in range(len(ps))]])
    f = sym.factor_segments(a, b, seg, sig)
    assert not f.singular
    for j in range(sig.shape[0]):
        neg, zero, pos, tiny = f.inertia_segments(j)
        for p, q in enumerate(ps):
            want = spectral.count_below(lams[p], sig[j, p])
            assert (neg[p], zero[p], pos[p]) == (want, 0, q.n - want), (j, p)
            assert tiny[p] == 0
        # the stack's own counts are the sums over its pencils
        tneg, tzero, tpos, _ = f.inertia(j)
        assert (tneg, tzero, tpos) == (int(neg.sum()), int(zero.sum()), int(pos.sum()))


def test_stacked_equals_one_pencil_at_a_time(gpu_lib):
    # the first pencils of the seeded uneven batch (smallest dims kept small for the test):
    # the stacked factor's per-pencil counts equal each pencil factored on its own
    specs = [((min(d[0], 9), min(d[1], 9), min(d[2], 9)), e, s_) for d, e, s_ in uneven_batch_specs(5)]
    ps = batch_pencils(specs)
    st, seg, _ = stack_pencils(ps)
    ctx, sym, a, b = setup(gpu_lib, st)
    rng = np.random.default_rng(3)
    sig = rng.uniform(-0.5, 1.5, size=(2, len(ps)))
    f = sym.factor_segments(a, b, seg, sig)
    for p, q in enumerate(ps):
        _, sym1, a1, b1 = setup(gpu_lib, q)
        f1 = sym1.factor(a1, b1, sig[:, p], "inertia", allow_singular=True)
        for j in range(2):
            neg, zero, pos, _ = f.inertia_segments(j)
            assert (neg[p], zero[p], pos[p]) == f1.inertia(j)[:3], (p, j)


def test_stack_rejects_a_coupling_entry(gpu_lib):
    ps = [laplacian_1d(20), laplacian_1d(30)]
    st, seg, _ = stack_pencils(ps)
    ctx, sym, a, b = setup(gpu_lib, st)
    bad = seg.copy()
    bad[19] = 1                       # row 19 couples to row 18 of pencil 0
    with pytest.raises(gpu_lib.SisliceError):
        sym.factor_segments(a, b, bad, np.zeros((1, 2)))
    with pytest.raises(gpu_lib.SisliceError):
        sym.factor_segments(a, b, seg, np.array([[0.0, np.nan]]))
