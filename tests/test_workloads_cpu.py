"""The seeded pencil generator: the drop rule keeps the four-exponent pencils positive
definite, and for the eight-exponent basis (whose overlap the drop alone leaves
indefinite) the diagonal compensation adds exactly the overlap mass each row loses and
restores positive definiteness (Eq. 1 needs B SPD)."""
import numpy as np
import scipy.linalg as sla

from workloads.pencils import EXPONENTS_4, exponents_8, gaussian_pencil


def test_four_exponent_overlap_stays_positive_definite():
    p = gaussian_pencil((6, 6, 6), EXPONENTS_4, seed=1)
    assert sla.eigvalsh(p.dense("b"))[0] > 1e-4


def test_drop_compensation_eight_exponents():
    dims = (5, 5, 5)
    plain = gaussian_pencil(dims, exponents_8(), seed=3)
    comp = gaussian_pencil(dims, exponents_8(), seed=3, compensate_drop=True)
    exact = gaussian_pencil(dims, exponents_8(), seed=3, drop=1e-16)   # all pairs above 1e-16
    Sk, Sc, Se = plain.dense("b"), comp.dense("b"), exact.dense("b")
    assert np.array_equal(plain.colind, comp.colind) and np.array_equal(plain.a, comp.a)
    mass = np.abs(Se - Sk).sum(axis=1)
    assert np.abs(np.diag(Sc) - np.diag(Sk) - mass).max() <= 1e-13
    assert np.array_equal(Sc - np.diag(np.diag(Sc)), Sk - np.diag(np.diag(Sk)))
    # the compensated overlap dominates the exact one
    assert sla.eigvalsh(Sc - Se)[0] >= -1e-12
    assert sla.eigvalsh(Sc)[0] > 0.0
    # without it the drop breaks definiteness once the lattice is large enough
    big = gaussian_pencil((8, 8, 8), exponents_8(), seed=3)
    assert sla.eigvalsh(big.dense("b"))[0] < 0.0
    big_c = gaussian_pencil((8, 8, 8), exponents_8(), seed=3, compensate_drop=True)
    assert sla.eigvalsh(big_c.dense("b"))[0] > 1e-5


def test_uneven_batch_specs_ranges_and_seeding():
    from workloads.pencils import EXPONENTS_2, EXPONENTS_4, uneven_batch_specs
    specs = uneven_batch_specs(256)
    assert specs == uneven_batch_specs(256)                 # seeded
    dims = np.array([d for d, _, _ in specs])
    assert dims.min() == 8 and dims.max() == 18
    kinds = {e for _, e, _ in specs}
    assert kinds == {EXPONENTS_2, EXPONENTS_4}
    n = np.array([np.prod(d) * len(e) for d, e, _ in specs])
    assert 1000 <= n.min() and n.max() <= 4 * 18 ** 3


def test_stack_pencils_is_block_diagonal_and_analyses_per_pencil():
    from paper_1908_06043_gb300 import api
    from workloads.pencils import EXPONENTS_2, gaussian_pencil, laplacian_1d, stack_pencils
    ps = [gaussian_pencil((3, 4, 5), EXPONENTS_2, seed=5), laplacian_1d(50, mass=True), gaussian_pencil((4, 4, 4), seed=6)]
    st, seg, offs = stack_pencils(ps)
    assert st.n == sum(q.n for q in ps) and st.nnz == sum(q.nnz for q in ps)
    rows = st.rows()
    assert np.array_equal(seg[rows], seg[st.colind])        # no entry couples two pencils
    for i, q in enumerate(ps):
        blk = slice(offs[i], offs[i + 1])
        assert np.array_equal(st.dense("a")[blk, blk], q.dense("a"))
        assert np.array_equal(st.dense("b")[blk, blk], q.dense("b"))
    # the dissection keeps each pencil in its own subtrees: the stack's factor flops are
    # the sum of the pencils' own
    ctx = api.Context(-1)
    whole = ctx.analyze(st.rowptr, st.colind)
    whole.validate()
    parts = sum(ctx.analyze(q.rowptr, q.colind).info["factor_flops"] for q in ps)
    assert abs(whole.info["factor_flops"] - parts) <= 1e-9 * parts


def test_stacked_spectrum_is_the_union_of_the_pencils_spectra():
    # the oracle's eigenvalues of the stack are the pencils' eigenvalues merged, so each
    # pencil's count below its own shift is the stack's count restricted to its rows
    from oracle import dense
    from workloads.pencils import EXPONENTS_2, gaussian_pencil, laplacian_1d, stack_pencils
    ps = [gaussian_pencil((3, 3, 4), EXPONENTS_2, seed=8), laplacian_1d(40, mass=True)]
    st, _, _ = stack_pencils(ps)
    lam_st = dense.gen_eig(st.dense("a"), st.dense("b"), vectors=False)[0]
    parts = np.sort(np.concatenate([dense.gen_eig(q.dense("a"), q.dense("b"), vectors=False)[0] for q in ps]))
    assert np.allclose(lam_st, parts, rtol=1e-12, atol=1e-12 * np.abs(parts).max())
