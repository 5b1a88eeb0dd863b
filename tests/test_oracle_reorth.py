"""Pins of oracle/reorth.py, the exact inner products of the full
reorthogonalization (Section 3.2.2): brute force with fractions, inputs on
which FP64 arithmetic is itself exact, the FP64 error bound, and the input
rounding's fixed points."""

from fractions import Fraction

import numpy as np
import pytest

from oracle import reorth


def frac_round(x: float, exponent: int) -> Fraction:
    """x rounded to the grid 2^(exponent - 62), half to even, in rationals."""
    scale = Fraction(2) ** (62 - exponent)
    return Fraction(round(Fraction(x) * scale)) / scale


def test_projection_matches_brute_force_in_rationals():
    rng = np.random.default_rng(1)
    Q = rng.standard_normal((7, 3)) * 0.3
    W = rng.standard_normal((7, 2)) * np.array([5.0, 1e-7])
    C = reorth.exact_projection(Q, W)
    for j in range(2):
        m = max(abs(Fraction(float(x))) for x in W[:, j])
        E = 0
        while Fraction(2) ** E <= m:
            E += 1
        while Fraction(2) ** (E - 1) > m:
            E -= 1
        for k in range(3):
            exact = sum(frac_round(Q[i, k], 0) * frac_round(W[i, j], E) for i in range(7))
            assert C[k, j] == float(exact)


def test_projection_equals_fp64_where_fp64_is_exact():
    # integers scaled by powers of two: every product and partial sum is exact in FP64
    rng = np.random.default_rng(2)
    Q = rng.integers(-1000, 1000, size=(300, 5)) / 1024.0
    W = rng.integers(-50, 50, size=(300, 3)).astype(float) * 4.0
    assert np.array_equal(reorth.exact_projection(Q, W), Q.T @ W)


def test_projection_within_the_fp64_error_bound():
    rng = np.random.default_rng(3)
    n = 2000
    Q = reorth.grid_round(rng.standard_normal((n, 6)) / np.sqrt(n))
    W = rng.standard_normal((n, 2))
    W = np.column_stack([reorth.grid_round(W[:, j], reorth.column_scale_exponent(W[:, j])) for j in range(2)])
    exact = reorth.exact_projection(Q, W)
    bound = n * 2.0**-53 * (np.abs(Q).T @ np.abs(W)) + 2.0**-1074
    assert np.all(np.abs(exact - Q.T @ W) <= bound)
    # a plausible slip (a transposed operand, a dropped column scale) breaks it
    assert not np.allclose(exact[:, 0], (Q.T @ W)[:, 1])


def test_grid_rounding_fixed_points():
    rng = np.random.default_rng(4)
    x = rng.uniform(2.0**-10, 1.0, size=500) * rng.choice([-1, 1], size=500)
    assert np.array_equal(reorth.grid_round(x), x)  # 53 bits above 2^-10 fit the 2^-62 grid
    y = rng.standard_normal(500) * 1e-9
    g = reorth.grid_round(y)
    assert np.array_equal(reorth.grid_round(g), g)
    assert np.max(np.abs(g - y)) <= 2.0**-63
    assert reorth.column_scale_exponent(np.array([0.75, -0.1])) == 0
    assert reorth.column_scale_exponent(np.array([1.0])) == 1
    assert reorth.column_scale_exponent(np.zeros(3)) == 0


def test_update_matches_brute_force_in_rationals():
    rng = np.random.default_rng(5)
    Q = rng.standard_normal((6, 4)) * 0.4
    H = rng.standard_normal((4, 2)) * np.array([3.0, 1e-5])
    W = rng.standard_normal((6, 2))
    out = reorth.exact_update(Q, H, W)
    for j in range(2):
        F = reorth.column_scale_exponent(H[:, j])
        for i in range(6):
            prod = sum(frac_round(Q[i, k], 0) * frac_round(H[k, j], F) for k in range(4))
            assert out[i, j] == float(Fraction(float(W[i, j])) - prod)


@pytest.mark.parametrize("n", [1, 9, 256])
def test_projection_of_an_orthonormal_basis_on_itself(n):
    # Q^T Q = I up to the basis's own rounding: the diagonal is 1 within n 2^-62
    rng = np.random.default_rng(n)
    Q, _ = np.linalg.qr(rng.standard_normal((max(n, 3), 3)))
    Q = reorth.grid_round(Q)
    G = reorth.exact_projection(Q, Q)
    assert np.max(np.abs(G - np.eye(3))) < 1e-15
