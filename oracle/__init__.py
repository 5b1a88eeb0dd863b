"""FP64 CPU oracle for the filtered Lanczos procedure (arXiv 2409.15053).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import, call or execute
anything in this package. The product path (the CUDA library and its Python
binding) never imports it and shares no code with it.

It is a plain, slow, obviously correct restatement of the paper in numpy /
scipy FP64, following the paper's steps in its order and notation:

- ``chebyshev``: the spectral map (eq. transf), the closed-form Chebyshev
  coefficients of the ideal filter (Section 2.2), the truncated filter p_m,
  the degree rule (eq. optimaldegree) and Clenshaw's algorithm for p_m(A)V
  (end of Section 2.2).
- ``lanczos``: spectrum-bound estimation by a few Lanczos steps (Section 2.2,
  after eq. transf), and the block filtered Lanczos procedure with full
  reorthogonalization, Rayleigh-Ritz, Rayleigh quotients and the convergence
  test (Sections 2.3 and 3.2.2).
- ``dense``: the result by definition for small matrices (all eigenpairs of
  A inside [alpha, beta]) and a Sylvester-inertia eigenvalue count.
- ``reorth``: the inner products and updates of the full reorthogonalization
  (Section 3.2.2) and the Ritz-vector combinations (Section 2.3) evaluated
  exactly in integer arithmetic on the FP64 inputs as given, rounded once.

Library primitives used as single steps: scipy sparse matrix products,
numpy matrix products, ``numpy.linalg.qr`` (Householder QR) and
``numpy.linalg.eigh`` (dense symmetric eigensolve).

Every function is pinned by ``tests/test_oracle_*.py`` against values the
paper prints (Table 2 filter degrees), closed forms (Chebyshev identities,
Laplacian spectra), brute force on tiny inputs and library routines.
"""

from . import chebyshev, dense, lanczos, reorth  # noqa: F401
