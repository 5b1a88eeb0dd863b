"""The seeded generators: closed-form structure counts, symmetry, and
bit-stable output (the checksum recorded when the config-2 reference was
computed by the oracle must be reproduced on any host)."""

import json
import os

import numpy as np

from synth import (csr_checksum, fd4_laplacian_3d, laplacian_2d, laplacian_3d_7pt, powerlaw_graph_laplacian,
                   uneven_batch)
from synth.workloads import CONFIG2

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_stencil_nnz_closed_forms():
    assert laplacian_2d(50, 50).nnz == 5 * 2500 - 4 * 50
    assert laplacian_3d_7pt(10, 11, 12).nnz == 7 * 1320 - 2 * (11 * 12 + 10 * 12 + 10 * 11)
    N = 12
    assert fd4_laplacian_3d(N).nnz == N ** 3 + 3 * N * N * (2 * (N - 1) + 2 * (N - 2))


def test_generators_are_symmetric():
    for A in (laplacian_3d_7pt(7, 8, 9, np.linspace(0, 1, 504)), fd4_laplacian_3d(9),
              powerlaw_graph_laplacian(5000, seed=1)):
        S = A.to_scipy()
        assert abs(S - S.T).max() == 0.0


def test_graph_laplacian_annihilates_constants():
    A = powerlaw_graph_laplacian(20000, seed=4).to_scipy()
    assert np.max(np.abs(A @ np.ones(A.shape[0]))) < 1e-10


def test_uneven_batch_shapes():
    mats = uneven_batch(8, seed=3)
    assert len(mats) == 8
    for A, kind, dims in mats:
        assert A.n == int(np.prod(dims)) and kind in ("2d", "3d")


def test_config2_matrix_matches_the_oracle_reference():
    ref = json.load(open(os.path.join(GOLD, "config2_reference.json")))
    rng = np.random.Generator(np.random.PCG64(CONFIG2["seed"]))
    g = CONFIG2["grid"]
    A = laplacian_3d_7pt(g, g, g, CONFIG2["potential_scale"] * rng.random(g ** 3))
    assert csr_checksum(A) == ref["matrix_checksum"]
    assert CONFIG2["beta"] == ref["beta"] and CONFIG2["count"] == ref["count"] == len(ref["eigenvalues"])


def test_fd_weights_are_exact_on_polynomials():
    from synth.matrices import fd_second_derivative_weights
    assert np.allclose(fd_second_derivative_weights(1), [-2.0, 1.0])
    assert np.allclose(fd_second_derivative_weights(2), [-2.5, 4.0 / 3.0, -1.0 / 12.0])
    for N in (3, 6):
        c = fd_second_derivative_weights(N)
        k = np.arange(1, N + 1)
        # f = x^(2j) at x = 0: f'' = 2 for j = 1, 0 for 2 <= j <= N
        for j in range(1, N + 1):
            got = 2.0 * np.sum(c[1:] * k.astype(float) ** (2 * j))
            assert abs(got - (2.0 if j == 1 else 0.0)) < 1e-9


def test_parsec_like_hamiltonian_shape():
    from synth.matrices import parsec_like_hamiltonian
    A = parsec_like_hamiltonian(radius=12.0, heavy=10, light=8, seed=3)
    S = A.to_scipy()
    assert abs(S - S.T).max() == 0.0
    assert np.all(np.diff(A.rowptr) > 0)
    for i in range(0, A.n, 97):  # columns sorted within rows
        row = A.col[A.rowptr[i]:A.rowptr[i + 1]]
        assert np.all(np.diff(row) > 0)
    # n = lattice points in the ball of radius 12
    ax = np.arange(-12, 13)
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    assert A.n == int(np.sum(X * X + Y * Y + Z * Z <= 144))
    # the kinetic stencil alone gives 1 + 36 entries per interior row; the non-local blocks add more
    assert A.nnz / A.n > 30


def test_powerlaw_graph_zero_mode_is_simple_with_constant_eigenvector():
    # the ring keeps the graph connected: 0 is a simple eigenvalue of L = D - W
    # with eigenvector 1/sqrt(n); everything else is positive (L is PSD)
    from oracle import dense
    from synth import powerlaw_graph_laplacian
    n = 600
    L = powerlaw_graph_laplacian(n, seed=5).to_scipy().toarray()
    assert np.allclose(L, L.T)
    assert np.max(np.abs(L.sum(axis=1))) < 1e-12  # rows of a Laplacian sum to zero
    w, V = dense.eigenpairs_in_interval(L, -1.0, 1e-9)
    assert w.shape == (1,) and abs(w[0]) < 1e-10
    assert np.max(np.abs(np.abs(V[:, 0]) - 1.0 / np.sqrt(n))) < 1e-10
    w_all = np.linalg.eigvalsh(L)
    assert w_all[1] > 1e-6 and w_all[0] > -1e-10
