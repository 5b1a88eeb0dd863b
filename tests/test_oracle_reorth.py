"""Pins of oracle/reorth.py, the exact inner products and updates of the full
reorthogonalization (Section 3.2.2) on unrounded FP64 inputs.

Each pin computes the same exact value another way or checks it against what
arithmetic fixes: error-free products (Dekker's splitting) summed by
math.fsum (Shewchuk's exactly rounded sum), brute force in rationals, inputs
on which FP64 arithmetic is itself exact, a cancellation whose exact result
is known in closed form, and the classical FP64 error bound."""

import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import reorth


def two_product(a: float, b: float) -> tuple[float, float]:
    """p + e = a * b exactly (Dekker, Veltkamp splitting; no overflow or underflow)."""
    p = a * b

    def split(x):
        c = 134217729.0 * x  # 2^27 + 1
        hi = c - (c - x)
        return hi, x - hi

    ah, al = split(a)
    bh, bl = split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def fsum_dot(a, b, extra=()):
    """Exactly rounded sum of extra + sum_i a_i b_i, by error-free products and math.fsum."""
    terms = list(extra)
    for x, y in zip(a, b):
        p, e = two_product(float(x), float(y))
        terms += [p, e]
    return math.fsum(terms)


def scaled_normal(rng, shape, lo=-30, hi=4):
    """Normal entries times random powers of two: wide exponents, no under/overflow."""
    return rng.standard_normal(shape) * np.ldexp(1.0, rng.integers(lo, hi, size=shape))


def test_projection_equals_error_free_products_summed_by_fsum():
    rng = np.random.default_rng(1)
    Q = scaled_normal(rng, (400, 5))
    W = scaled_normal(rng, (400, 3))
    C = reorth.exact_projection(Q, W)
    for k in range(5):
        for j in range(3):
            assert C[k, j] == fsum_dot(Q[:, k], W[:, j])


def test_update_equals_error_free_products_summed_by_fsum():
    rng = np.random.default_rng(2)
    Q = scaled_normal(rng, (7, 30))
    H = scaled_normal(rng, (30, 4))
    W = scaled_normal(rng, (7, 4))
    out = reorth.exact_update(Q, H, W)
    for i in range(7):
        for j in range(4):
            assert out[i, j] == fsum_dot(Q[i, :], -H[:, j], extra=[W[i, j]])
    X = reorth.exact_combination(Q, H)
    for i in range(7):
        for j in range(4):
            assert X[i, j] == fsum_dot(Q[i, :], H[:, j])


def test_projection_matches_brute_force_in_rationals():
    rng = np.random.default_rng(3)
    Q = rng.standard_normal((9, 3)) * 0.3
    W = rng.standard_normal((9, 2)) * np.array([5.0, 1e-7])
    C = reorth.exact_projection(Q, W)
    for k in range(3):
        for j in range(2):
            exact = sum(Fraction(float(Q[i, k])) * Fraction(float(W[i, j])) for i in range(9))
            assert C[k, j] == float(exact)


def test_projection_equals_fp64_where_fp64_is_exact():
    # integers scaled by powers of two: every product and partial sum is exact in FP64
    rng = np.random.default_rng(4)
    Q = rng.integers(-1000, 1000, size=(300, 5)) / 1024.0
    W = rng.integers(-50, 50, size=(300, 3)).astype(float) * 4.0
    assert np.array_equal(reorth.exact_projection(Q, W), Q.T @ W)
    H = rng.integers(-64, 64, size=(5, 3)) / 8.0
    assert np.array_equal(reorth.exact_update(Q, H, W), W - Q @ H)


def test_cancellation_with_a_known_exact_result():
    # 1 + 1e-20 - 1 in FP64 is 0; the exact value is the FP64 number 1e-20 itself
    q = np.array([[1.0], [1e-20], [-1.0]])
    w = np.array([[1.0], [1.0], [1.0]])
    assert (q.T @ w)[0, 0] == 0.0
    assert reorth.exact_projection(q, w)[0, 0] == 1e-20
    # W - Q H where the exact difference is 2^-80 below an O(1) value
    Q = np.array([[1.0, 2.0**-80]])
    H = np.array([[1.0], [-1.0]])
    W = np.array([[1.0]])
    assert reorth.exact_update(Q, H, W)[0, 0] == 2.0**-80


def test_projection_within_the_fp64_error_bound():
    rng = np.random.default_rng(5)
    n = 2000
    Q = rng.standard_normal((n, 6)) / np.sqrt(n)
    W = rng.standard_normal((n, 2))
    exact = reorth.exact_projection(Q, W)
    bound = n * 2.0**-53 * (np.abs(Q).T @ np.abs(W)) + 2.0**-1074
    assert np.all(np.abs(exact - Q.T @ W) <= bound)
    # plausible slips (a transposed operand, a dropped term) break it
    assert not np.allclose(exact[:, 0], (Q.T @ W)[:, 1])
    assert not np.all(np.abs(exact - Q[1:].T @ W[1:]) <= bound)


@pytest.mark.parametrize("n", [3, 9, 256])
def test_projection_of_an_orthonormal_basis_on_itself(n):
    rng = np.random.default_rng(n)
    Q, _ = np.linalg.qr(rng.standard_normal((n, 3)))
    G = reorth.exact_projection(Q, Q)
    assert np.max(np.abs(G - np.eye(3))) < 1e-15
    assert np.array_equal(G, G.T)  # the exact Gram matrix is symmetric after rounding
