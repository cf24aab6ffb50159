"""GB300-native shift-invert spectrum slicing (SISLICE, arXiv 1908.06043) hot path.

The CUDA library (``_build/libsislice.so``, C ABI in ``include/sislice.h``) holds the
path: symbolic analysis, multifrontal LDL^T with inertia, panel solves, the in-slice
subspace iteration, the Lanczos DOS sweeps and the band-energy gradient.  ``api``
marshals arguments to it; ``driver`` holds the host-side slicing logic (shift
placement from the DOS, slice validation, k-means shift migration).
"""
from .build import build  # noqa: F401
