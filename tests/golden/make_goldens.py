"""Write stored expected values for the N = 16,384 Gaussian pencil (16^3 lattice,
4 s-functions per atom, seed 2) using only the CPU oracle.

Outputs (text, one value per line after a '#' header):
* gauss16_eigs.txt     lowest 2,048 eigenvalues of (A, B) from the dense oracle
                       (Cholesky-reduced tridiagonal QL), Eq. 1.
* gauss16_inertia.txt  sigma, n_neg, n_zero, n_pos of A - sigma B from the band
                       LDL^T oracle (Sylvester's law, Section 2.2), for a few shifts.

Run: python tests/golden/make_goldens.py   (about 10-20 minutes on 8 cores)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import dense, spectral  # noqa: E402
from workloads.pencils import config_pencil  # noqa: E402

N_KEEP = 2048
SIGMAS = (-2.0, -0.5, 0.0, 0.25, 0.5, 1.0)


def main():
    p = config_pencil(2)
    t = time.time()
    with open(os.path.join(HERE, "gauss16_inertia.txt"), "w") as f:
        f.write("# A - sigma B inertia, 16^3 Gaussian pencil (4 fn/atom, seed 2), band LDL^T oracle\n")
        f.write("# sigma n_neg n_zero n_pos min_pivot_ratio\n")
        for s in SIGMAS:
            inert, rmin, rc = spectral.band_inertia(p, s)
            assert rc == 0
            f.write(f"{s!r} {inert[0]} {inert[1]} {inert[2]} {rmin:.3e}\n")
            f.flush()
            print("band", s, inert, rmin, time.time() - t, flush=True)
    lam, _ = dense.gen_eig(p.dense("a"), p.dense("b"), vectors=False)
    print("dense eig", time.time() - t, flush=True)
    with open(os.path.join(HERE, "gauss16_eigs.txt"), "w") as f:
        f.write("# lowest 2048 eigenvalues, 16^3 Gaussian pencil (4 fn/atom, seed 2), dense oracle\n")
        for v in lam[:N_KEEP]:
            f.write(f"{float(v)!r}\n")


if __name__ == "__main__":
    main()
