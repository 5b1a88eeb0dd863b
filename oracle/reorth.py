"""Inner products of the full reorthogonalization (Section 3.2.2), evaluated exactly. Test infrastructure only.

Full reorthogonalization projects a block W on the Krylov basis Q: C = Q^T W,
then W - Q C (classical Gram-Schmidt, applied twice). The oracle here is that
definition evaluated with no rounding at all: every FP64 value is an integer
multiple of a power of two, so products and sums are formed exactly with
Python integers and rounded once, to the nearest FP64, at the end.

The fixed-point representation the tensor-core path works on is reproduced
as the input rounding:
- basis values are rounded to the grid of 2^-62 (round half to even);
- a block W (or a coefficient matrix H) is rounded per column to 62
  fractional bits of its scale 2^E, E the smallest integer with
  max |column| < 2^E.
The products of these rounded values are then exact; the functions return
them rounded to FP64. Callers that want the exact product of unrounded FP64
values pass values already on those grids.

Pins: tests/test_oracle_reorth.py (brute force with fractions, integer inputs
where FP64 arithmetic is exact, the FP64 error bound, idempotence of the
rounding).
"""

from __future__ import annotations

from fractions import Fraction

import numpy as np

GRID_BITS = 62


def column_scale_exponent(col: np.ndarray) -> int:
    """E with max |col| < 2^E (0 for a zero column)."""
    m = float(np.max(np.abs(col))) if col.size else 0.0
    if m == 0.0:
        return 0
    return int(np.frexp(m)[1])


def to_fixed(x: np.ndarray, exponent: int) -> list:
    """round(x * 2^(62 - exponent)) as Python integers (round half to even), flattened."""
    scaled = np.asarray(x, dtype=np.float64) * np.ldexp(1.0, GRID_BITS - exponent)  # exact scaling
    return [int(v) for v in np.rint(scaled).ravel()]


def grid_round(x: np.ndarray, exponent: int = 0) -> np.ndarray:
    """x rounded to the grid of 2^(exponent - 62), as FP64 (exact for |x| < 2^exponent)."""
    ints = to_fixed(x, exponent)
    return np.array([np.ldexp(float(v), exponent - GRID_BITS) for v in ints]).reshape(np.shape(x))


def _to_double(numerator: int, exponent: int) -> float:
    """numerator * 2^exponent rounded to the nearest FP64."""
    return float(Fraction(numerator) * Fraction(2) ** exponent)


def exact_projection(Q: np.ndarray, W: np.ndarray) -> np.ndarray:
    """C = Q^T W on the rounded values (Q on the 2^-62 grid, W per column), exactly, then rounded to FP64."""
    K, r = Q.shape[1], W.shape[1]
    q = [to_fixed(Q[:, k], 0) for k in range(K)]
    C = np.zeros((K, r))
    for j in range(r):
        E = column_scale_exponent(W[:, j])
        w = to_fixed(W[:, j], E)
        for k in range(K):
            C[k, j] = _to_double(sum(a * b for a, b in zip(q[k], w)), E - 2 * GRID_BITS)
    return C


def exact_update(Q: np.ndarray, H: np.ndarray, W: np.ndarray) -> np.ndarray:
    """W - Q H with Q on the 2^-62 grid and H rounded per column, exactly, then rounded to FP64.

    W itself enters unrounded (the update subtracts from the FP64 block)."""
    n, K = Q.shape
    r = H.shape[1]
    q = [to_fixed(Q[i, :], 0) for i in range(n)]
    out = np.zeros((n, r))
    for j in range(r):
        F = column_scale_exponent(H[:, j])
        h = to_fixed(H[:, j], F)
        for i in range(n):
            prod = Fraction(sum(a * b for a, b in zip(q[i], h))) * Fraction(2) ** (F - 2 * GRID_BITS)
            out[i, j] = float(Fraction(float(W[i, j])) - prod)
    return out
