"""FP64 CPU oracle for the TT-UTV sweep -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, deliberately unoptimised restatement of the
paper's method ("Effective algorithms for tensor-train decomposition via the
UTV framework", arXiv 2501.07904) in numpy FP64.  It exists to check the CUDA
path.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the library itself never does, and it shares no
code with the CUDA path (only the seeded input generators in ``synth`` are
common to both).

Modules
-------
linalg  Householder QR (optionally column-pivoted) and one-sided Jacobi SVD.
philox  Philox4x32-10 counter-based generator and the Rademacher sketch matrix.
tt      TT format (Eq. TT), TT-ULV (Alg. 1/2), TT-URV (Alg. 3 and its
        prescribed-accuracy analogue), TT-ULV right-to-left (the appendix's
        Alg. 4, both middle blocks), TT-SVD, the range step with optional
        power iterations, masked evaluation and gradients.
rgrad   Riemannian gradient completion (Sec. 4.2.2): tangent-space
        projection at a fixed-rank TT, the exact line-search step, the
        fixed-rank TT-UTV / TT-SVD retraction and spectral initialisation.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, LAPACK, brute force or the paper's Table (tab: Beps);
``philox`` is pinned bit for bit against PyTorch's independently written
Philox4x32-10 engine (ATen/core/PhiloxRNGEngine.h, compiled on the host by
``tests/test_oracle_philox_pin.py``) and by statistical properties.
"""
from . import linalg, philox, rgrad, tt  # noqa: F401
