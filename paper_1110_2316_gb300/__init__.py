"""GB300 (sm_103a) library for the hot path of the nonconforming h-p
least-squares spectral element method (A. Husain, 2010): the matrix-free
normal operator of the functional of eq. (4.2), the separable block
preconditioner of eq. (5.19)-(5.20) and PCG with FP64 iterative refinement.

The compute path is the CUDA library ``libhpse.so`` (C ABI in include/hpse.h);
``api`` is its Python binding.  Importing this package does not load the
library; ``api.Mesh`` does, and fails loudly if it has not been built.
"""

from .build import build  # noqa: F401
