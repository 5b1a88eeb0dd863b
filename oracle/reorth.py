"""Inner products and updates of the full reorthogonalization (Section 3.2.2), evaluated exactly. Test infrastructure only.

Full reorthogonalization projects a block W on the Krylov basis Q, C = Q^T W,
and removes that component, W - Q C (classical Gram-Schmidt, applied twice);
the Ritz vectors of Section 2.3 are the combinations X = Q Y. The oracle here
is each of those definitions evaluated on the FP64 inputs exactly as given,
with no rounding anywhere but one final rounding to the nearest FP64 per
output value: every finite FP64 number is an integer times a power of two, so
products and sums are formed exactly in Python integers.

Nothing here knows how any fast path represents its numbers; a fast path's
error is judged against these exact values.

Pins: tests/test_oracle_reorth.py (error-free products summed by math.fsum,
brute force in rationals, inputs on which FP64 arithmetic is itself exact, a
cancellation with a known exact result, the FP64 error bound).
"""

from __future__ import annotations

import math

import numpy as np


def _split(x: float) -> tuple[int, int]:
    """(m, e) with x = m * 2^e exactly, m an integer (|m| < 2^53)."""
    if x == 0.0:
        return 0, 0
    f, e = math.frexp(x)  # x = f 2^e, 0.5 <= |f| < 1, f has at most 53 significant bits
    return int(f * 2.0**53), e - 53


def _column(v: np.ndarray) -> tuple[list, int]:
    """Integers M_i and one exponent E with v_i = M_i 2^E exactly."""
    parts = [_split(float(x)) for x in np.asarray(v, dtype=np.float64).ravel()]
    E = min((e for m, e in parts if m != 0), default=0)
    return [m << (e - E) if m != 0 else 0 for m, e in parts], E


def _round(N: int, E: int) -> float:
    """N 2^E rounded once to the nearest FP64 (ties to even)."""
    if N == 0:
        return 0.0
    if E >= 0:
        return float(N << E)
    return N / (1 << -E)  # Python's int / int is correctly rounded


def exact_dot(a: np.ndarray, b: np.ndarray) -> float:
    """sum_i a_i b_i of two FP64 vectors, exactly, rounded once."""
    A, Ea = _column(a)
    B, Eb = _column(b)
    return _round(sum(x * y for x, y in zip(A, B)), Ea + Eb)


def exact_projection(Q: np.ndarray, W: np.ndarray) -> np.ndarray:
    """C = Q^T W (Q n x K, W n x r), each entry exact, rounded once."""
    K, r = Q.shape[1], W.shape[1]
    q = [_column(Q[:, k]) for k in range(K)]
    w = [_column(W[:, j]) for j in range(r)]
    C = np.zeros((K, r))
    for k in range(K):
        for j in range(r):
            C[k, j] = _round(sum(x * y for x, y in zip(q[k][0], w[j][0])), q[k][1] + w[j][1])
    return C


def exact_update(Q: np.ndarray, H: np.ndarray, W: np.ndarray) -> np.ndarray:
    """W - Q H (Q n x K, H K x r, W n x r), each entry exact, rounded once."""
    n, K = Q.shape
    r = H.shape[1]
    h = [_column(H[:, j]) for j in range(r)]
    out = np.zeros((n, r))
    for i in range(n):
        qi, Eq = _column(Q[i, :])
        for j in range(r):
            P = sum(x * y for x, y in zip(qi, h[j][0]))
            Ep = Eq + h[j][1]
            mw, ew = _split(float(W[i, j]))
            E = min(Ep, ew) if mw != 0 else Ep
            out[i, j] = _round((mw << (ew - E)) - (P << (Ep - E)), E)
    return out


def exact_combination(Q: np.ndarray, H: np.ndarray) -> np.ndarray:
    """X = Q H (the Ritz vectors' combination of basis columns), each entry exact, rounded once."""
    return exact_update(Q, -np.asarray(H, dtype=np.float64), np.zeros((Q.shape[0], H.shape[1])))
