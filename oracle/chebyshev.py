"""Chebyshev filter polynomials (Section 2.2 of arXiv 2409.15053). Test infrastructure only.

Notation follows the paper: the spectrum of A lies in [lambda_min, lambda_max],
A is mapped to [-1, 1] by eq. (transf), phi is the indicator of the mapped
interval [alpha, beta], b_i are its Chebyshev coefficients and p_m is the
degree-m truncation of the Chebyshev series of phi.
"""

from __future__ import annotations

import numpy as np

# The tolerance of eq. (optimaldegree). The paper only says it is chosen
# experimentally; 0.3123 is the reading under which the degree rule returns
# all five automatic degrees of Table 2 (49, 49, 61, 98, 308) from the
# Table 1 spectra and the Table 2 intervals.
DEGREE_EPS = 0.3123


def spectral_map(lmin: float, lmax: float):
    """Eq. (transf): A := (A - cI)/e with c = (lmin+lmax)/2, e = (lmax-lmin)/2."""
    c = 0.5 * (lmin + lmax)
    e = 0.5 * (lmax - lmin)
    return c, e


def map_interval(alpha: float, beta: float, lmin: float, lmax: float):
    """Apply eq. (transf) to the user's interval; returns (c, e, alpha', beta')."""
    c, e = spectral_map(lmin, lmax)
    return c, e, (alpha - c) / e, (beta - c) / e


def filter_coefficients(alpha: float, beta: float, m: int) -> np.ndarray:
    """b_0..b_m of the ideal filter phi on [alpha, beta] within [-1, 1] (Section 2.2).

    b_0 = (arccos(alpha) - arccos(beta)) / pi and, for i > 0,
    b_i = 2 (sin(i arccos(alpha)) - sin(i arccos(beta))) / (i pi).
    """
    ta = np.arccos(alpha)
    tb = np.arccos(beta)
    b = np.empty(m + 1)
    b[0] = (ta - tb) / np.pi
    for i in range(1, m + 1):
        b[i] = 2.0 * (np.sin(i * ta) - np.sin(i * tb)) / (i * np.pi)
    return b


def ideal_filter_norm_sq(alpha: float, beta: float) -> float:
    """||phi||^2 in the weighted Chebyshev 2-norm: the integral of 1/sqrt(1-z^2) over [alpha, beta]."""
    return float(np.arccos(alpha) - np.arccos(beta))


def truncation_error_sq(alpha: float, beta: float, m: int) -> float:
    """||p_m - phi||^2 in the weighted norm, by Parseval on the orthogonality relation.

    With ||T_0||^2 = pi and ||T_i||^2 = pi/2 (i > 0), the tail of the series is
    ||phi||^2 - pi b_0^2 - (pi/2) sum_{i=1..m} b_i^2.
    """
    b = filter_coefficients(alpha, beta, m)
    kept = np.pi * b[0] ** 2 + 0.5 * np.pi * float(np.sum(b[1:] ** 2))
    return ideal_filter_norm_sq(alpha, beta) - kept


def auto_degree(alpha: float, beta: float, eps: float = DEGREE_EPS, m_max: int = 100000) -> int:
    """Eq. (optimaldegree): the least m > 0 with ||p_m - phi|| < eps ||phi||."""
    norm_sq = ideal_filter_norm_sq(alpha, beta)
    ta = np.arccos(alpha)
    tb = np.arccos(beta)
    b0 = (ta - tb) / np.pi
    kept = np.pi * b0 ** 2
    for m in range(1, m_max + 1):
        bm = 2.0 * (np.sin(m * ta) - np.sin(m * tb)) / (m * np.pi)
        kept += 0.5 * np.pi * bm ** 2
        if norm_sq - kept < eps ** 2 * norm_sq:
            return m
    raise ValueError("degree rule did not terminate below m_max")


def clenshaw_scalar(b: np.ndarray, z) -> np.ndarray:
    """p_m(z) = sum_i b_i T_i(z) at points z by Clenshaw's algorithm."""
    z = np.asarray(z, dtype=np.float64)
    u1 = np.zeros_like(z)
    u2 = np.zeros_like(z)
    for k in range(len(b) - 1, 0, -1):
        u1, u2 = b[k] + 2.0 * z * u1 - u2, u1
    return b[0] + z * u1 - u2


def apply_mapped(A, c: float, e: float, Y: np.ndarray) -> np.ndarray:
    """(A - cI)/e times Y, eq. (transf) applied to a block."""
    return (A @ Y - c * Y) / e


def clenshaw_apply(A, c: float, e: float, b: np.ndarray, V: np.ndarray) -> np.ndarray:
    """p_m((A - cI)/e) V by the vectorized Clenshaw algorithm the paper uses (Section 2.2).

    U_{m+1} = U_{m+2} = 0; U_k = b_k V + 2 Ahat U_{k+1} - U_{k+2} for k = m..1;
    p_m(Ahat) V = b_0 V + Ahat U_1 - U_2.
    """
    V = np.asarray(V, dtype=np.float64)
    u1 = np.zeros_like(V)
    u2 = np.zeros_like(V)
    for k in range(len(b) - 1, 0, -1):
        u1, u2 = b[k] * V + 2.0 * apply_mapped(A, c, e, u1) - u2, u1
    return b[0] * V + apply_mapped(A, c, e, u1) - u2


def jackson_factors(m: int) -> np.ndarray:
    """Jackson damping factors g_0..g_m for a degree-m Chebyshev series.

    g_k = ((m - k + 1) cos(k pi/(m+1)) + sin(k pi/(m+1)) cot(pi/(m+1))) / (m + 1).
    The paper truncates without damping (Section 2.2); damping is an option of
    this library (FILTLAN-style smoothing of the Gibbs oscillations).
    """
    k = np.arange(m + 1, dtype=np.float64)
    a = np.pi / (m + 1)
    return ((m - k + 1) * np.cos(k * a) + np.sin(k * a) / np.tan(a)) / (m + 1)


def damped_filter_coefficients(alpha: float, beta: float, m: int) -> np.ndarray:
    """Jackson-damped coefficients g_k b_k of the ideal filter on [alpha, beta]."""
    return filter_coefficients(alpha, beta, m) * jackson_factors(m)


def lanczos_sigma_factors(m: int) -> np.ndarray:
    """Lanczos sigma factors sigma_0..sigma_m: sigma_k = sin(k pi/(m+1)) / (k pi/(m+1)), sigma_0 = 1.

    Another damping of the truncated series (not used by the paper): it
    averages the partial sum over one period of its highest term, which
    shrinks the Gibbs overshoot without removing it.
    """
    k = np.arange(m + 1, dtype=np.float64)
    x = k * np.pi / (m + 1)
    out = np.ones(m + 1)
    out[1:] = np.sin(x[1:]) / x[1:]
    return out


def sigma_damped_filter_coefficients(alpha: float, beta: float, m: int) -> np.ndarray:
    """Lanczos-sigma-damped coefficients sigma_k b_k of the ideal filter on [alpha, beta]."""
    return filter_coefficients(alpha, beta, m) * lanczos_sigma_factors(m)


def _cos_integral(k: int, t: float) -> float:
    """Antiderivative of cos(k t) at t."""
    return t if k == 0 else np.sin(k * t) / k


def _zcos_integral(k: int, t: float) -> float:
    """Antiderivative of cos(t) cos(k t) at t (the weighted integral of z T_k)."""
    if k == 1:
        return 0.5 * (t + 0.5 * np.sin(2.0 * t))
    return 0.5 * (np.sin((k - 1) * t) / (k - 1) + np.sin((k + 1) * t) / (k + 1))


def smoothed_step_coefficients(alpha: float, beta: float, delta: float, m: int) -> np.ndarray:
    """Least-squares polynomial filter of degree m for a smoothed step.

    The target is 1 on [alpha, beta], falls linearly to 0 over [alpha - delta,
    alpha] and [beta, beta + delta], and is 0 elsewhere on [-1, 1]. In the
    weighted Chebyshev 2-norm of the degree rule the best approximation of
    degree m is the truncated Chebyshev series, whose coefficients
    c_k = (2 - [k = 0]) / pi * integral_0^pi f(cos t) cos(k t) dt have closed
    forms piece by piece (t = arccos z): the flat part gives the indicator's
    coefficients, a ramp (z - z0) / (z1 - z0) gives integrals of cos t cos kt
    and cos kt. (A least-squares filter with a transition band, in the spirit of
    FILTLAN's; the paper itself uses the plain indicator.)
    """
    pieces = []  # (z_lo, z_hi, kind): kind 1 = constant 1, ('ramp', z0, z1)
    lo_flat, hi_flat = max(alpha, -1.0), min(beta, 1.0)
    if hi_flat > lo_flat:
        pieces.append((lo_flat, hi_flat, None))
    if delta > 0:
        zl0, zl1 = max(alpha - delta, -1.0), min(alpha, 1.0)
        if zl1 > zl0:
            pieces.append((zl0, zl1, (alpha - delta, alpha)))   # rises from 0 at alpha - delta to 1 at alpha
        zr0, zr1 = max(beta, -1.0), min(beta + delta, 1.0)
        if zr1 > zr0:
            pieces.append((zr0, zr1, (beta + delta, beta)))    # falls from 1 at beta to 0 at beta + delta
    c = np.zeros(m + 1)
    for k in range(m + 1):
        acc = 0.0
        for z_lo, z_hi, ramp in pieces:
            t_lo, t_hi = np.arccos(z_hi), np.arccos(z_lo)  # t increases as z decreases
            if ramp is None:
                acc += _cos_integral(k, t_hi) - _cos_integral(k, t_lo)
            else:
                z0, z1 = ramp  # f = (z - z0) / (z1 - z0)
                acc += ((_zcos_integral(k, t_hi) - _zcos_integral(k, t_lo))
                        - z0 * (_cos_integral(k, t_hi) - _cos_integral(k, t_lo))) / (z1 - z0)
        c[k] = (2.0 - (k == 0)) / np.pi * acc
    return c


def _dyadic(x: float) -> tuple[int, int]:
    """(m, e) with x = m 2^e exactly."""
    if x == 0.0:
        return 0, 0
    f, e = np.frexp(x)
    return int(f * 2.0**53), int(e) - 53


class _Dyadic:
    """A vector of exact dyadic rationals N_i 2^E with one shared exponent."""

    def __init__(self, N, E):
        self.N, self.E = N, E

    @staticmethod
    def of(x):
        parts = [_dyadic(float(v)) for v in x]
        E = min((e for m, e in parts if m), default=0)
        return _Dyadic([m << (e - E) if m else 0 for m, e in parts], E)

    def aligned(self, E):
        return [v << (self.E - E) for v in self.N]


def clenshaw_apply_exact(S2, b: np.ndarray, V: np.ndarray) -> np.ndarray:
    """p_m(Ahat) V for the matrix 2 Ahat given with FP64 entries, in exact arithmetic, rounded once.

    Clenshaw's recurrence of Section 2.2 with nothing rounded in between:
    U_{m+1} = U_{m+2} = 0; U_k = b_k V + (2 Ahat) U_{k+1} - U_{k+2}; p = b_0 V +
    (1/2)(2 Ahat) U_1 - U_2. Every FP64 number is an integer times a power of
    two, so each U_k is held as integers with a shared power of two. S2 is a
    scipy CSR matrix holding 2 Ahat; the result is p_m(Ahat) V rounded to FP64
    entry by entry (the reference for measuring a kernel's rounding error).
    Slow: for small matrices and degrees.
    """
    S2 = S2.tocsr()
    n = S2.shape[0]
    V = np.asarray(V, dtype=np.float64)
    vals = _Dyadic.of(S2.data)
    out = np.empty_like(V)
    bd = [_dyadic(float(x)) for x in b]
    for t in range(V.shape[1]):
        v = _Dyadic.of(V[:, t])

        def times_2ahat(u):
            E = vals.E + u.E
            N = [0] * n
            for i in range(n):
                acc = 0
                for j in range(S2.indptr[i], S2.indptr[i + 1]):
                    acc += vals.N[j] * u.N[S2.indices[j]]
                N[i] = acc
            return _Dyadic(N, E)

        def combine(terms):  # sum of (sign, vector) pairs, exactly
            E = min(x.E for _, x in terms)
            acc = [0] * n
            for sg, x in terms:
                for i, val in enumerate(x.aligned(E)):
                    acc[i] += sg * val
            return _Dyadic(acc, E)

        def scaled(k):  # b_k V
            mb, eb = bd[k]
            return _Dyadic([mb * x for x in v.N], v.E + eb)

        zero = _Dyadic([0] * n, 0)
        u1, u2 = zero, zero
        for k in range(len(b) - 1, 0, -1):
            u1, u2 = combine([(1, scaled(k)), (1, times_2ahat(u1)), (-1, u2)]), u1
        half = times_2ahat(u1)
        half.E -= 1
        p = combine([(1, scaled(0)), (1, half), (-1, u2)])
        for i in range(n):
            N, E = p.N[i], p.E
            out[i, t] = float(N << E) if E >= 0 else N / (1 << -E)
    return out


def damping_filter_coefficients(zc: float, d: int) -> np.ndarray:
    """Chebyshev coefficients in z of T_d(a z + b) / T_d(b - a), [zc, 1] -> [-1, 1] by z -> a z + b.

    The refinement of the mixed-precision form (not in the paper) damps the
    spectrum above zc: on [zc, 1] this is a Chebyshev polynomial of that
    interval, scaled to 1 at z = -1. Computed as numpy's Chebyshev series T_d
    with domain [zc, 1], re-expanded on [-1, 1]. A library primitive serves as
    the step.
    """
    T = np.polynomial.Chebyshev.basis(d, domain=[zc, 1.0])
    c = T.convert(domain=[-1.0, 1.0], kind=np.polynomial.Chebyshev).coef
    return c / T(-1.0)
