"""Write stored expected values for the N = 16,384 Gaussian pencil (16^3 lattice,
4 s-functions per atom, seed 2) using only the CPU oracle.

Outputs (text, one value per line after a '#' header):
* gauss16_eigs.txt     lowest 2,048 eigenvalues of (A, B), Eq. 1: the Rayleigh quotients
                       on the sparse pencil of the eigenvectors of the dense oracle
                       (Cholesky-reduced tridiagonal QL, inverse iteration, back-
                       transform; oracle.spectral.lowest_eigenpairs).  The reduced
                       eigenvalues alone carry an error of about u ||A|| ||x||_2^2, up to
                       2e-8 on the low tail of this pencil, whose eigenvectors have
                       ||x||_2 up to 270 at ||x||_B = 1.
* gauss16_inertia.txt  sigma, n_neg, n_zero, n_pos of A - sigma B from the band
                       LDL^T oracle (Sylvester's law, Section 2.2), for a few shifts.

Run: python tests/golden/make_goldens.py [--eigs-only]   (about an hour on 8 cores)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import spectral  # noqa: E402
from workloads.pencils import config_pencil  # noqa: E402

N_KEEP = 2048
SIGMAS = (-2.0, -0.5, 0.0, 0.25, 0.5, 1.0)


def main():
    p = config_pencil(2)
    t = time.time()
    if "--eigs-only" not in sys.argv:
        write_inertia(p, t)
    lam, _ = spectral.lowest_eigenpairs(p, N_KEEP)
    print("dense eig", time.time() - t, flush=True)
    with open(os.path.join(HERE, "gauss16_eigs.txt"), "w") as f:
        f.write("# lowest 2048 eigenvalues, 16^3 Gaussian pencil (4 fn/atom, seed 2): Rayleigh quotients of "
                "the dense oracle's eigenvectors\n")
        for v in lam:
            f.write(f"{float(v)!r}\n")


def write_inertia(p, t):
    with open(os.path.join(HERE, "gauss16_inertia.txt"), "w") as f:
        f.write("# A - sigma B inertia, 16^3 Gaussian pencil (4 fn/atom, seed 2), band LDL^T oracle\n")
        f.write("# sigma n_neg n_zero n_pos min_pivot_ratio\n")
        for s in SIGMAS:
            inert, rmin, rc = spectral.band_inertia(p, s)
            assert rc == 0
            f.write(f"{s!r} {inert[0]} {inert[1]} {inert[2]} {rmin:.3e}\n")
            f.flush()
            print("band", s, inert, rmin, time.time() - t, flush=True)


if __name__ == "__main__":
    main()
