"""Band-energy gradient sampled on the stored pattern (test infrastructure only).

E = sum_{i <= n_e} lambda_i.  For B-orthonormal eigenvectors, Hellmann-Feynman gives
d lambda_i / d A_pq = x_pi x_qi and d lambda_i / d B_pq = -lambda_i x_pi x_qi when the
single stored entry (p, q) is perturbed.  Returned per stored CSR entry; the gradient
with respect to a symmetric parameter tying (p, q) and (q, p) is the sum of the two
mirror entries.
"""
from __future__ import annotations

import numpy as np


def band_energy_grad(pencil, lam, X):
    rows = pencil.rows()
    cols = pencil.colind.astype(np.int64)
    X = np.asarray(X, dtype=np.float64)
    ga = np.einsum("ei,ei->e", X[rows], X[cols])
    gb = -np.einsum("ei,ei,i->e", X[rows], X[cols], np.asarray(lam))
    return ga, gb
