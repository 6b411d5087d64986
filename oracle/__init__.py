"""Plain, slow, FP64 CPU oracle for s-step GMRES with two-stage block
orthogonalization (Yamazaki, Higgins, Boman, Szyld, arXiv 2402.15033).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may use it.  It shares no code with the CUDA library; the only
common dependency is the seeded input generator module ``synth``.

Every routine follows the paper's definitions step by step in numpy FP64
(library primitives such as a matrix product, a triangular solve or a sparse
matrix-vector product serve as single steps; there is no blocking, fusion or
reordering).  The paper's pseudocode figures are not in its source, so the
algorithms are restated from its prose, captions and equations; each function
names the passage it follows.

Modules
-------
``blockortho``  CholQR, CholQR2, BCGS, BCGS2 with CholQR2, BCGS-PIP, BCGS-PIP2,
                the two stages of the two-stage scheme, Householder QR (checker).
``krylov``      MPK, Givens least squares, Hessenberg recovery, standard
                GMRES with CGS2, s-step GMRES with the three block schemes.
``checks``      orthogonality error, condition number, exact dot products.
``precond``     multicolor Gauss-Seidel (greedy coloring, forward sweep).
"""
from . import blockortho, krylov, checks, precond  # noqa: F401
