"""CPU oracle for the SISLICE slice-solve hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct FP64 implementations of what the GPU path computes,
each citing the paper passage it follows.  Only ``tests/``, ``__graft_entry__.smoke``
and ``bench.py``'s CPU-baseline / reference leg may import anything from here; the
library in ``paper_1908_06043_gb300`` never does, and the oracle never imports the
library.  The only code both sides share is the seeded input generator module
``workloads`` (inputs only, none of the method's arithmetic).

Modules
-------
dense      ctypes binding of ``oracle.c``: dense generalised eigensolver, dense
           Bunch-Kaufman inertia, band LDL^T inertia, CSR products, tridiagonal eig.
spectral   slice membership, inertia counts, residuals, B-orthonormality (Eq. 1,
           Section 2.2 validation counts, residual definition after Alg. 2).
dos        Lanczos DOS estimate and closed-form CDOS / shift formulas (Eqs. 4-8).
partition  CDOS-root intervals, expectation shifts, exactly-n_s safeguards, slice
           validation (Section 2.2) and k-means++ / Lloyd shift migration (Sec. 3.2).
grad       band-energy gradient sampled on the pattern (Hellmann-Feynman).

Parity status: every function here is pinned by ``tests/test_oracle_*.py`` against
closed forms, invariants, an outside library (scipy/numpy LAPACK) or brute force.
"""
