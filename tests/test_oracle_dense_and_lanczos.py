"""Pins for oracle.dense and oracle.lanczos against closed forms, brute force and library routines.

- Dense eigenpairs and inertia counts against the closed-form spectra of the
  Dirichlet Laplacians (2D: 4 - 2cos(i pi/(nx+1)) - 2cos(j pi/(ny+1)); 3D the
  same with 6 and three cosines) and against numpy's dense eigensolver.
- Spectrum bounds enclose the closed-form extremes.
- The block filtered Lanczos procedure returns, with multiplicity, exactly the
  eigenvalues the closed forms or a dense eigensolve give in [alpha, beta].
"""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import dense, lanczos
from synth import (diagonal_csr, fd4_laplacian_3d, gaussian_wells_potential, laplacian_2d,
                   laplacian_3d_7pt, powerlaw_graph_laplacian, random_normal_block)


def lap2d_eigs(nx, ny):
    i = np.arange(1, nx + 1)[:, None]
    j = np.arange(1, ny + 1)[None, :]
    return np.sort((4 - 2 * np.cos(i * np.pi / (nx + 1)) - 2 * np.cos(j * np.pi / (ny + 1))).ravel())


def lap3d_eigs(nx, ny, nz):
    i = np.arange(1, nx + 1)[:, None, None]
    j = np.arange(1, ny + 1)[None, :, None]
    k = np.arange(1, nz + 1)[None, None, :]
    lam = 6 - 2 * np.cos(i * np.pi / (nx + 1)) - 2 * np.cos(j * np.pi / (ny + 1)) - 2 * np.cos(k * np.pi / (nz + 1))
    return np.sort(lam.ravel())


def gap_interval(eigs, lo_index, count):
    """[alpha, beta] at gap midpoints around eigs[lo_index : lo_index+count] (sorted)."""
    a = 0.5 * (eigs[lo_index - 1] + eigs[lo_index]) if lo_index > 0 else eigs[0] - 1.0
    b = 0.5 * (eigs[lo_index + count - 1] + eigs[lo_index + count])
    return a, b


# The config-1 window: 20 eigenvalues (10 doublets) of the 50x50 Laplacian.
CFG1_ALPHA, CFG1_BETA = 0.9198764447231507, 1.0094761615910202


def test_dense_eigenpairs_match_laplacian_closed_form():
    A = laplacian_2d(12, 15).to_dense()
    lam = lap2d_eigs(12, 15)
    w, V = dense.eigenpairs_in_interval(A, 1.0, 3.0)
    ref = lam[(lam >= 1.0) & (lam <= 3.0)]
    assert w.shape == ref.shape
    assert np.max(np.abs(w - ref)) < 1e-12
    assert np.max(np.abs(A @ V - V * w)) < 1e-12


@pytest.mark.parametrize("sigma", [0.3, 1.7, 4.1, 6.6])
def test_inertia_count_matches_2d_closed_form(sigma):
    A = laplacian_2d(30, 30).to_scipy()
    assert dense.count_below(A, sigma) == int(np.sum(lap2d_eigs(30, 30) < sigma))


def test_inertia_count_matches_3d_closed_form():
    A = laplacian_3d_7pt(8, 9, 10).to_scipy()
    lam = lap3d_eigs(8, 9, 10)
    for sigma in (0.9, 3.3, 6.01, 10.5):
        assert dense.count_below(A, sigma) == int(np.sum(lam < sigma))


def test_inertia_count_matches_dense_on_random_banded():
    rng = np.random.default_rng(4)
    n, bw = 120, 7
    M = np.zeros((n, n))
    for k in range(bw + 1):
        v = rng.standard_normal(n - k)
        M += np.diag(v, k)
        if k:
            M += np.diag(v, -k)
    w = np.linalg.eigvalsh(M)
    for sigma in (-2.0, 0.13, 1.9):
        assert dense.count_below(sp.csr_matrix(M), sigma) == int(np.sum(w < sigma))


def test_gershgorin_contains_spectrum():
    rng = np.random.default_rng(1)
    M = rng.standard_normal((60, 60))
    M = M + M.T
    lo, hi = lanczos.gershgorin_interval(sp.csr_matrix(M))
    w = np.linalg.eigvalsh(M)
    assert lo <= w[0] and w[-1] <= hi


def test_lanczos_bounds_enclose_extremes():
    A = laplacian_2d(40, 40).to_scipy()
    lam = lap2d_eigs(40, 40)
    lo, hi, info = lanczos.lanczos_bounds(A, random_normal_block(1600, 1, 3)[:, 0], 60)
    assert lo <= lam[0] and hi >= lam[-1]
    assert lo >= 0.0 and hi <= 8.0  # Gershgorin clamp
    d = np.linspace(-3.0, 5.0, 500)
    lo, hi, info = lanczos.lanczos_bounds(diagonal_csr(d).to_scipy(), random_normal_block(500, 1, 9)[:, 0], 60)
    assert lo <= -3.0 and hi >= 5.0 and hi - lo < 8.0 * 1.05


def test_block_tridiagonal_layout():
    D = [np.array([[1.0, 2.0], [2.0, 3.0]]), np.array([[4.0, 0.5], [0.5, 6.0]])]
    S = [np.array([[7.0, 8.0], [0.0, 9.0]])]
    T = lanczos.block_tridiagonal(D, S)
    assert np.allclose(T, T.T)
    assert T[2, 0] == 7.0 and T[2, 1] == 8.0 and T[3, 1] == 9.0 and T[3, 0] == 0.0
    assert T[0, 2] == 7.0 and T[1, 2] == 8.0


@pytest.mark.parametrize("r", [1, 2])
def test_flp_config1_window_matches_closed_form(r):
    A = laplacian_2d(50, 50).to_scipy()
    lam = lap2d_eigs(50, 50)
    ref = lam[(lam >= CFG1_ALPHA) & (lam <= CFG1_BETA)]
    assert ref.shape[0] == 20
    res = lanczos.filtered_lanczos(A, CFG1_ALPHA, CFG1_BETA, random_normal_block(2500, r, 7),
                                   bounds_start=random_normal_block(2500, 1, 8)[:, 0], degree=50, tol=1e-10)
    assert res.converged
    assert res.eigenvalues.shape == ref.shape
    assert np.max(np.abs(res.eigenvalues - ref)) < 1e-10 * np.max(np.abs(ref))
    assert np.max(res.residuals) <= 1e-10
    X = res.eigenvectors
    assert np.max(np.abs(X.T @ X - np.eye(X.shape[1]))) < 1e-12
    assert res.matvecs == r * 50 * res.iters


def _check_against_dense(Acsr, alpha, beta, r, seed, degree=None):
    A = Acsr.to_scipy()
    w = np.linalg.eigvalsh(Acsr.to_dense())
    ref = w[(w >= alpha) & (w <= beta)]
    res = lanczos.filtered_lanczos(A, alpha, beta, random_normal_block(Acsr.n, r, seed),
                                   bounds_start=random_normal_block(Acsr.n, 1, seed + 1)[:, 0],
                                   degree=degree, tol=1e-10)
    assert res.converged
    assert res.eigenvalues.shape == ref.shape
    scale = max(abs(w[0]), abs(w[-1]))
    assert np.max(np.abs(res.eigenvalues - ref)) < 1e-10 * scale
    return res


def test_flp_3d_laplacian_with_potential_matches_dense():
    rng = np.random.Generator(np.random.PCG64(5))
    A = laplacian_3d_7pt(12, 12, 12, 0.5 * rng.random(1728))
    w = np.linalg.eigvalsh(A.to_dense())
    a, b = gap_interval(w, 0, 40)
    _check_against_dense(A, a, b, 4, 21)


def test_flp_fd4_hamiltonian_matches_dense_auto_degree():
    N = 11
    A = fd4_laplacian_3d(N, gaussian_wells_potential(N, 8, seed=2))
    w = np.linalg.eigvalsh(A.to_dense())
    a, b = gap_interval(w, 3, 25)
    res = _check_against_dense(A, a, b, 4, 31)
    assert res.degree > 1


def test_flp_powerlaw_graph_matches_dense():
    A = powerlaw_graph_laplacian(2000, seed=7)
    w = np.linalg.eigvalsh(A.to_dense())
    a, b = gap_interval(w, 40, 15)
    _check_against_dense(A, a, b, 4, 41, degree=60)


def test_flp_count_matches_inertia_on_midsize_grid():
    rng = np.random.Generator(np.random.PCG64(9))
    A = laplacian_3d_7pt(16, 16, 16, 0.5 * rng.random(4096))
    S = A.to_scipy()
    # endpoints chosen between eigenvalues reported by an independent dense run
    w = np.linalg.eigvalsh(A.to_dense())
    a, b = gap_interval(w, 10, 30)
    cnt = dense.count_in_interval(S, a, b)
    assert cnt == 30
    res = lanczos.filtered_lanczos(S, a, b, random_normal_block(4096, 4, 3),
                                   bounds_start=random_normal_block(4096, 1, 4)[:, 0], tol=1e-10)
    assert res.converged and res.eigenvalues.shape[0] == cnt


def test_planted_transposed_coupling_block_is_caught(monkeypatch):
    # Eq. (lanczos) puts S_i below the diagonal and S_i^T above it. Swapping
    # them (a transposed operand) breaks the Rayleigh-Ritz step: the run no
    # longer converges to the closed-form window.
    A = laplacian_2d(50, 50).to_scipy()
    lam = lap2d_eigs(50, 50)
    ref = lam[(lam >= CFG1_ALPHA) & (lam <= CFG1_BETA)]

    def swapped(D, S):
        return lanczos_block_tridiagonal(D, [s.T for s in S])

    lanczos_block_tridiagonal = lanczos.block_tridiagonal
    monkeypatch.setattr(lanczos, "block_tridiagonal", swapped)
    res = lanczos.filtered_lanczos(A, CFG1_ALPHA, CFG1_BETA, random_normal_block(2500, 2, 7),
                                   bounds_start=random_normal_block(2500, 1, 8)[:, 0], degree=50,
                                   tol=1e-10, max_blocks=150)
    ok = (res.converged and res.eigenvalues.shape == ref.shape
          and np.max(np.abs(res.eigenvalues - ref)) < 1e-10)
    assert not ok
