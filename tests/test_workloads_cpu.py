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
