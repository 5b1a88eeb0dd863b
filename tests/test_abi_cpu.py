"""C-ABI checks that need no GPU: the library builds and loads, exports every
symbol include/flz.h declares, and its host-only logic (filter coefficients,
the degree rule, the projected-problem eigensolver, parameters and status
strings) agrees with the paper and with independent computations.
"""

import os
import re

import numpy as np
import pytest

import __graft_entry__
import paper_2409_15053_gb300 as flz
from oracle import chebyshev

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()


def header_symbols():
    text = open(os.path.join(ROOT, "include", "flz.h")).read()
    return sorted(set(re.findall(r"^(?:flz_status|const char\*)\s+(flz_\w+)\s*\(", text, flags=re.M)))


def test_header_and_binding_agree():
    assert sorted(flz.EXPORTED) == header_symbols()


def test_library_exports_every_declared_symbol():
    L = flz.lib()
    for name in header_symbols():
        assert hasattr(L, name), name


def test_status_strings_and_defaults():
    assert flz.flz_status_string(flz.FLZ_OK) == "FLZ_OK"
    assert flz.flz_status_string(flz.FLZ_ERR_EMPTY_INTERVAL) == "FLZ_ERR_EMPTY_INTERVAL"
    p = flz.flz_params_default()
    assert p.block_size == 3 and p.degree == 0 and abs(p.degree_eps - 0.3123) < 1e-15
    assert p.check_every == 30 and p.tol == 1e-10 and p.bounds_steps == 60


@pytest.mark.parametrize("a,b,m", [(-1.0, -0.5, 30), (0.1, 0.3, 80), (-0.9538, 0.2, 5), (-1.0, 1.0, 12)])
def test_coefficients_match_oracle(a, b, m):
    got = flz.flz_filter_coefficients(a, b, m)
    assert np.max(np.abs(got - chebyshev.filter_coefficients(a, b, m))) < 1e-14


@pytest.mark.parametrize("m", [0, 1, 9, 100])
def test_jackson_factors_match_oracle(m):
    assert np.max(np.abs(flz.flz_jackson_factors(m) - chebyshev.jackson_factors(m))) < 1e-14


@pytest.mark.parametrize("m", [0, 1, 9, 100])
def test_lanczos_sigma_factors_match_oracle(m):
    assert np.max(np.abs(flz.flz_lanczos_sigma_factors(m) - chebyshev.lanczos_sigma_factors(m))) < 1e-15


@pytest.mark.parametrize("a,b,d", [(0.1, 0.3, 0.05), (-1.0, -0.6, 0.1), (-0.2, 0.9, 0.2), (0.2, 0.4, 0.0)])
def test_smoothed_step_coefficients_match_oracle(a, b, d):
    got = flz.flz_smoothed_step_coefficients(a, b, d, 60)
    assert np.max(np.abs(got - chebyshev.smoothed_step_coefficients(a, b, d, 60))) < 1e-14


def test_degree_rule_reproduces_table2():
    import json
    rows = json.load(open(os.path.join(ROOT, "tests", "golden", "table2_auto_degree.json")))["rows"]
    for row in rows:
        c = 0.5 * (row["lmin"] + row["lmax"])
        e = 0.5 * (row["lmax"] - row["lmin"])
        assert flz.flz_filter_degree((row["alpha"] - c) / e, (row["beta"] - c) / e) == row["m_auto"]


def test_invalid_arguments_are_rejected_without_a_gpu():
    with pytest.raises(flz.FlzError) as e:
        flz.flz_filter_coefficients(0.5, 0.1, 10)
    assert e.value.status == flz.FLZ_ERR_INVALID_ARG
    assert "alpha < beta" in flz.flz_last_error()  # the thread's last failure message
    flz.flz_filter_coefficients(0.1, 0.5, 10)
    assert flz.flz_last_error() == ""  # cleared by the next successful call
    with pytest.raises(flz.FlzError) as e:
        flz.flz_filter_degree(-1.0, -0.99999999, 0.3123, 5)
    assert e.value.status == flz.FLZ_ERR_CAPACITY


def test_reorthogonalization_entry_points_reject_bad_arguments_without_a_gpu():
    # argument checks run before any device call
    assert flz.flz_params_default().ortho == flz.FLZ_ORTHO_AUTO
    fake = 16  # never dereferenced: every call below fails its checks first
    cases = [
        dict(n=100, nb=2, r=17, method=flz.FLZ_ORTHO_TENSOR),    # block wider than 16
        dict(n=100, nb=2, r=4, method=7),                        # unknown method
        dict(n=100, nb=2, r=4, method=flz.FLZ_ORTHO_AUTO),       # AUTO is a solver setting only
        dict(n=0, nb=2, r=4, method=flz.FLZ_ORTHO_TENSOR),       # empty basis
        dict(n=100, nb=0, r=4, method=flz.FLZ_ORTHO_CUDA_CORES),
    ]
    for c in cases:
        for fn in (flz.flz_basis_project, flz.flz_basis_orthogonalize):
            with pytest.raises(flz.FlzError) as e:
                fn(c["n"], c["nb"], c["r"], fake, fake, fake, c["method"])
            assert e.value.status == flz.FLZ_ERR_INVALID_ARG
    with pytest.raises(flz.FlzError) as e:
        flz.flz_basis_project(100, 2, 4, None, fake, fake, flz.FLZ_ORTHO_TENSOR)
    assert e.value.status == flz.FLZ_ERR_INVALID_ARG


@pytest.mark.parametrize("np_,a_bytes,b_bytes,strides", [
    (24, 4096, 1024, (128, 2048, 128, 256)),       # N not one of 16, 32, 64, 128
    (32, 4008, 1024, (128, 2048, 128, 256)),       # image not a multiple of 16 bytes
    (32, 40960, 1024, (128, 2048, 128, 256)),      # A image larger than its 36 KB region
    (32, 4096, 1024, (128, 2056, 128, 256)),       # stride not a multiple of 16
    (32, 4096, 1024, (2048, 4096, 128, 256)),      # A reach past 36 KB under one reading
    (128, 4096, 4096, (128, 2048, 128, 4096)),     # B reach past 20 KB
])
def test_mma_probe_rejects_out_of_range_layouts_without_a_gpu(np_, a_bytes, b_bytes, strides):
    a = np.zeros(a_bytes // 2 + (a_bytes % 2), dtype=np.uint16)
    b = np.zeros(b_bytes // 2, dtype=np.uint16)
    L = flz.lib()
    d = np.zeros((128, max(np_, 16)), dtype=np.float32)
    st = L.flz_tc_mma_probe(flz._ptr(a), a_bytes, flz._ptr(b), b_bytes, np_, 0, *strides, flz._ptr(d))
    assert st == flz.FLZ_ERR_INVALID_ARG, flz.flz_last_error()


def _random_band(K, b, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    T = np.zeros((K, K))
    for k in range(b + 1):
        v = rng.standard_normal(K - k) * scale
        T += np.diag(v, k)
        if k:
            T += np.diag(v, -k)
    return T


@pytest.mark.parametrize("K,b", [(1, 1), (7, 3), (60, 1), (200, 4), (480, 16)])
def test_band_eigenvalues_match_dense_eigensolver(K, b):
    T = _random_band(K, b, K + b)
    got = flz.flz_band_eigenvalues(T, b)
    ref = np.linalg.eigvalsh(T)
    assert np.max(np.abs(got - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_band_eigenvectors_are_orthonormal_eigenvectors():
    T = _random_band(300, 4, 9)
    theta = flz.flz_band_eigenvalues(T, 4)
    idx = np.arange(299, 259, -1)
    Y = flz.flz_band_eigenvectors(T, 4, theta, idx)
    assert np.max(np.abs(T @ Y - Y * theta[idx])) < 1e-11
    assert np.max(np.abs(Y.T @ Y - np.eye(Y.shape[1]))) < 1e-12


def test_band_eigenvectors_span_a_multiple_eigenvalue():
    # block-diagonal copies of one matrix: every eigenvalue has multiplicity 3,
    # as in block Lanczos on a matrix with repeated eigenvalues
    B = _random_band(40, 2, 4)
    T = np.kron(np.eye(3), B)
    theta = flz.flz_band_eigenvalues(T, 2)
    ref = np.linalg.eigvalsh(T)
    assert np.max(np.abs(theta - ref)) < 1e-12
    top = np.arange(119, 113, -1)  # two triple eigenvalues
    Y = flz.flz_band_eigenvectors(T, 2, theta, top)
    assert np.max(np.abs(Y.T @ Y - np.eye(6))) < 1e-10
    assert np.max(np.abs(T @ Y - Y * theta[top])) < 1e-10


def test_laplacian_tridiagonal_closed_form():
    # 1D Dirichlet Laplacian: eigenvalues 2 - 2 cos(k pi / (K + 1))
    K = 150
    T = 2 * np.eye(K) - np.eye(K, k=1) - np.eye(K, k=-1)
    got = flz.flz_band_eigenvalues(T, 1)
    ref = np.sort(2 - 2 * np.cos(np.arange(1, K + 1) * np.pi / (K + 1)))
    assert np.max(np.abs(got - ref)) < 1e-13


@pytest.mark.parametrize("n", [1, 3, 40, 200])
def test_dense_symmetric_eigensolver_matches_numpy(n):
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, n))
    M = M + M.T
    w, Z = flz.flz_sym_eig(M)
    assert np.max(np.abs(w - np.linalg.eigvalsh(M))) < 1e-12 * max(1.0, np.max(np.abs(w)))
    assert np.max(np.abs(M @ Z - Z * w)) < 1e-12 * max(1.0, np.max(np.abs(w)))
    assert np.max(np.abs(Z.T @ Z - np.eye(n))) < 1e-13


def test_dense_symmetric_eigensolver_on_laplacian_closed_form():
    K = 80
    T = 2 * np.eye(K) - np.eye(K, k=1) - np.eye(K, k=-1)
    w, Z = flz.flz_sym_eig(T)
    ref = np.sort(2 - 2 * np.cos(np.arange(1, K + 1) * np.pi / (K + 1)))
    assert np.max(np.abs(w - ref)) < 1e-13
    # eigenvector k is sin(k i pi/(K+1)) up to sign and norm
    i = np.arange(1, K + 1)
    for k in (1, 17, 80):
        u = np.sin(k * i * np.pi / (K + 1))
        u /= np.linalg.norm(u)
        assert abs(abs(u @ Z[:, k - 1]) - 1.0) < 1e-12


@pytest.mark.parametrize("zc,d", [(-0.9, 12), (-0.98, 40), (0.3, 7)])
def test_damping_coefficients_match_the_oracle(zc, d):
    from oracle import chebyshev
    got = flz.flz_damping_coefficients(zc, d)
    want = chebyshev.damping_filter_coefficients(zc, d)
    assert got.shape == want.shape and np.max(np.abs(got - want)) < 1e-12
    with pytest.raises(flz.FlzError):
        flz.flz_damping_coefficients(1.0, 3)
