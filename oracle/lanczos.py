"""Spectrum bounds and the block filtered Lanczos procedure (Sections 2.2-2.3, 3.2.2). Test infrastructure only.

A plain FP64 restatement, step by step in the paper's order:

1. Bounds (Section 2.2 after eq. transf): lambda_min and lambda_max from a few
   Lanczos steps on A.
2. Map (eq. transf), filter coefficients (Section 2.2) and degree
   (eq. optimaldegree).
3. Block Lanczos on p(A) (eqs. krylov, lanczos): W = p(A) Q_j by Clenshaw,
   full reorthogonalization (Section 3.2.2), QR of W giving Q_{j+1} and the
   upper-triangular S_j.
4. Periodically (Section 3.2.2): Rayleigh-Ritz on T_k (eq. proj), Ritz vectors
   Q_k W_k, Rayleigh quotients (eq. rayleigh) and residuals; converged when
   all Ritz values in [alpha, beta] and a few of the nearest outside have small
   residuals.

Readings where the paper is silent (each listed in the design notes):
bounds use 60 Lanczos steps, padded by the Ritz residual bounds and clamped to
the Gershgorin interval; full reorthogonalization is classical Gram-Schmidt
applied twice; the check runs every 30 block steps; "a few of the nearest
outside" is max(r, 3) pairs; the Ritz pairs are ranked by their p(A) Ritz
value; the count in [alpha, beta] must also be unchanged since the previous
check; the residual is ||Ax - lambda x|| / ||A|| with ||A|| = max(|lmin|, |lmax|).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import chebyshev


def gershgorin_interval(A):
    """[min_i (a_ii - R_i), max_i (a_ii + R_i)] with R_i the off-diagonal absolute row sum."""
    d = A.diagonal()
    R = np.asarray(abs(A).sum(axis=1)).ravel() - np.abs(d)
    return float(np.min(d - R)), float(np.max(d + R))


def lanczos_bounds(A, v0: np.ndarray, steps: int = 60):
    """Estimate [lambda_min, lambda_max] with single-vector Lanczos on A.

    Full reorthogonalization (twice) keeps the basis orthonormal. The extreme
    Ritz values are padded by their residual bounds |beta_k s_k| and the result
    is clamped to the Gershgorin interval, which always contains the spectrum.
    Returns (lmin, lmax, info); info["ritz"] holds all Ritz values, ascending
    (by Cauchy interlacing the j-th smallest is >= the j-th smallest eigenvalue).
    """
    n = A.shape[0]
    k = min(int(steps), n)
    Q = np.zeros((n, k + 1))
    alphas, betas = [], []
    Q[:, 0] = v0 / np.linalg.norm(v0)
    for j in range(k):
        w = A @ Q[:, j]
        a = float(Q[:, j] @ w)
        w = w - a * Q[:, j]
        if j > 0:
            w = w - betas[-1] * Q[:, j - 1]
        for _ in range(2):
            w = w - Q[:, : j + 1] @ (Q[:, : j + 1].T @ w)
        b = float(np.linalg.norm(w))
        alphas.append(a)
        betas.append(b)
        if b <= 1e-14 * max(1.0, abs(a)):
            break
        Q[:, j + 1] = w / b
    kk = len(alphas)
    T = np.diag(alphas) + np.diag(betas[: kk - 1], 1) + np.diag(betas[: kk - 1], -1)
    theta, S = np.linalg.eigh(T)
    res = np.abs(betas[kk - 1] * S[kk - 1, :])
    lo = theta[0] - res[0]
    hi = theta[-1] + res[-1]
    g_lo, g_hi = gershgorin_interval(A)
    return max(lo, g_lo), min(hi, g_hi), {"steps": kk, "theta": (theta[0], theta[-1]), "res": (res[0], res[-1]),
                                          "ritz": theta}


@dataclass
class FLPResult:
    eigenvalues: np.ndarray
    eigenvectors: np.ndarray
    residuals: np.ndarray
    converged: bool
    iters: int
    degree: int
    block_size: int
    lmin: float
    lmax: float
    matvecs: int
    history: list = field(default_factory=list)


def block_tridiagonal(D: list, S: list) -> np.ndarray:
    """T_k of eq. (lanczos): D_i on the diagonal, S_i below and S_i^T above; symmetrized."""
    k = len(D)
    r = D[0].shape[0]
    T = np.zeros((k * r, k * r))
    for i in range(k):
        T[i * r:(i + 1) * r, i * r:(i + 1) * r] = D[i]
        if i + 1 < k:
            T[(i + 1) * r:(i + 2) * r, i * r:(i + 1) * r] = S[i]
            T[i * r:(i + 1) * r, (i + 1) * r:(i + 2) * r] = S[i].T
    return 0.5 * (T + T.T)


def filtered_lanczos(A, alpha: float, beta: float, start_block: np.ndarray, *,
                     bounds=None, bounds_start=None, bounds_steps: int = 60,
                     degree: int | None = None, eps: float = chebyshev.DEGREE_EPS,
                     tol: float = 1e-10, check_every: int = 30, max_blocks: int = 600,
                     guard: int | None = None) -> FLPResult:
    """All eigenpairs of symmetric A in [alpha, beta] by the filtered Lanczos procedure.

    ``start_block`` is the n x r starting block (its orthonormalization is the
    first step); ``bounds`` is an optional (lmin, lmax); otherwise they are
    estimated from ``bounds_start`` by :func:`lanczos_bounds`.
    """
    A = A.tocsr()
    n, r = start_block.shape
    if bounds is None:
        lmin, lmax, _ = lanczos_bounds(A, bounds_start, bounds_steps)
    else:
        lmin, lmax = bounds
    c, e, a_m, b_m = chebyshev.map_interval(alpha, beta, lmin, lmax)
    if b_m < -1.0 or a_m > 1.0 or a_m >= b_m:
        raise ValueError("interval misses the spectrum")
    a_m = max(a_m, -1.0)
    b_m = min(b_m, 1.0)
    m = degree if degree is not None else chebyshev.auto_degree(a_m, b_m, eps)
    coeffs = chebyshev.filter_coefficients(a_m, b_m, m)
    norm_a = max(abs(lmin), abs(lmax))
    g = guard if guard is not None else max(r, 3)

    Q1, _ = np.linalg.qr(start_block)
    blocks = [Q1]
    D, S = [], []
    prev_count = None
    history = []
    result = None
    for j in range(max_blocks):
        Qj = blocks[-1]
        W = chebyshev.clenshaw_apply(A, c, e, coeffs, Qj)
        Qall = np.hstack(blocks)
        C1 = Qall.T @ W
        W = W - Qall @ C1
        C2 = Qall.T @ W
        W = W - Qall @ C2
        D.append((C1 + C2)[-r:, :])
        Qn, Sj = np.linalg.qr(W)
        scale = max(np.max(np.abs(np.diag(Sj))), 1e-300)
        if np.min(np.abs(np.diag(Sj))) < 1e-12 * max(scale, np.linalg.norm(D[-1])):
            # Rank-deficient block: the new directions are arbitrary, so make
            # them orthogonal to the basis before continuing.
            for _ in range(2):
                Qn = Qn - Qall @ (Qall.T @ Qn)
            Qn, _ = np.linalg.qr(Qn)
        S.append(Sj)
        blocks.append(Qn)
        k = j + 1
        last = (k == max_blocks) or (k * r + r > n)
        if k % check_every != 0 and not last:
            continue
        T = block_tridiagonal(D, S[: k - 1])
        theta, Y = np.linalg.eigh(T)
        order = np.argsort(-theta)
        Qk = np.hstack(blocks[:k])
        inside, outside = [], 0
        all_small = True
        for idx in order:
            x = Qk @ Y[:, idx]
            x = x / np.linalg.norm(x)
            Ax = A @ x
            lam = float(x @ Ax)
            res = float(np.linalg.norm(Ax - lam * x)) / norm_a
            if res > tol:
                all_small = False
                break
            if alpha <= lam <= beta:
                inside.append((lam, x, res))
            else:
                outside += 1
                if outside >= g:
                    break
        count = len(inside)
        converged = all_small and outside >= g and prev_count is not None and count == prev_count
        history.append({"k": k, "count": count, "all_small": all_small})
        prev_count = count if all_small and outside >= g else None
        if converged or last:
            inside.sort(key=lambda t: t[0])
            result = FLPResult(
                eigenvalues=np.array([t[0] for t in inside]),
                eigenvectors=np.stack([t[1] for t in inside], axis=1) if inside else np.zeros((n, 0)),
                residuals=np.array([t[2] for t in inside]),
                converged=converged, iters=k, degree=m, block_size=r,
                lmin=lmin, lmax=lmax, matvecs=r * m * k, history=history)
            break
    return result
