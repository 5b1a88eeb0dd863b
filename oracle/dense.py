"""The result by definition, for matrices small enough to solve densely. Test infrastructure only.

The problem (program summary and Section 2.2 of arXiv 2409.15053): all
eigenpairs (lambda_j, x_j) of the symmetric matrix A with lambda_j in
[alpha, beta], counted with multiplicity.
"""

from __future__ import annotations

import numpy as np


def eigenpairs_in_interval(A_dense: np.ndarray, alpha: float, beta: float):
    """All eigenpairs of A with alpha <= lambda <= beta, ascending, by a dense FP64 eigensolve."""
    w, V = np.linalg.eigh(np.asarray(A_dense, dtype=np.float64))
    sel = (w >= alpha) & (w <= beta)
    return w[sel], V[:, sel]


def bandwidth(A) -> int:
    """Largest |i - j| over the stored entries of a scipy sparse matrix."""
    coo = A.tocoo()
    if coo.nnz == 0:
        return 0
    return int(np.max(np.abs(coo.row - coo.col)))


def count_below(A, sigma: float) -> int:
    """Number of eigenvalues of symmetric A below sigma, by Sylvester's law of inertia.

    Factor A - sigma I = L D L^T (band Gaussian elimination without pivoting,
    which keeps the band) and count the negative pivots of D. Valid when sigma
    is not an eigenvalue; the endpoints used in the tests sit in spectral gaps.
    """
    import scipy.sparse as sp

    A = sp.csr_matrix(A)
    n = A.shape[0]
    b = bandwidth(A)
    # Dense working window: row/col i of the trailing matrix held in W[0, :],
    # W is (b+1) x (b+1) over rows/cols i..i+b.
    Ad = A.tolil()
    W = np.zeros((b + 1, b + 1))
    for p in range(min(b + 1, n)):
        for q in range(min(b + 1, n)):
            W[p, q] = Ad[p, q]
    W[np.arange(b + 1), np.arange(b + 1)] -= sigma
    negatives = 0
    rows = A.tocsr()
    for i in range(n):
        d = W[0, 0]
        if d == 0.0:
            raise ZeroDivisionError("zero pivot: sigma is an eigenvalue of a leading block")
        if d < 0.0:
            negatives += 1
        l = W[1:, 0] / d
        W[1:, 1:] -= d * np.outer(l, l)
        # Shift the window by one and bring in row/col i+b+1 of A - sigma I.
        W[:-1, :-1] = W[1:, 1:]
        W[-1, :] = 0.0
        W[:, -1] = 0.0
        j = i + b + 1
        if j < n:
            start, end = rows.indptr[j], rows.indptr[j + 1]
            for cidx, v in zip(rows.indices[start:end], rows.data[start:end]):
                off = cidx - (i + 1)
                if 0 <= off <= b:
                    W[b, off] = v
                    W[off, b] = v
            W[b, b] -= sigma
    return negatives


def count_in_interval(A, alpha: float, beta: float) -> int:
    """Eigenvalue count in [alpha, beta] by two inertia counts (endpoints in gaps)."""
    return count_below(A, beta) - count_below(A, alpha)
