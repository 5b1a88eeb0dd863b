"""The 64-bit fixed-point filter (FLZ_PREC_FX64): W = p_m((A - cI)/e) V with
the recurrence vectors, the running sum, the entries of 2 Ahat and the
coefficients as integers (Section 2.2's forward recurrence on the integer
pipes).

Checks:
- element by element against the oracle's Clenshaw evaluation, within
  1e-12 max|V| (and within the FP64 rounding bound of test_gpu_filter);
- against the exact value of the same polynomial (the oracle's Clenshaw in
  exact dyadic arithmetic): its rounding error is no larger than the FP64
  kernel's on the same inputs;
- a spectrum outside [-1, 1] is reported (INVALID_ARG), not wrapped around;
- where the format does not apply (block width 5, a row of 2 Ahat with
  absolute sum above 3.9) the filter runs in FP64 and says so in the stats;
- solves with the fixed-point filter match closed forms, dense eigensolves
  and, at full size, the oracle's config-2 eigenvalues.
"""

import numpy as np
import pytest
import scipy.sparse as sp

import __graft_entry__
import paper_2409_15053_gb300 as flz
from oracle import chebyshev
from synth import (fd4_laplacian_3d, gaussian_wells_potential, laplacian_2d, laplacian_3d_7pt,
                   powerlaw_graph_laplacian, random_normal_block)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
FX = flz.FLZ_PREC_FX64
TIGHT = 1e-12  # element-wise, relative to max |V|


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


class Mat:
    def __init__(self, csr):
        self.csr = csr
        self.h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)

    def __del__(self):
        try:
            flz.flz_matrix_destroy(self.h)
        except Exception:
            pass


def run_filter(M, c, e, coeffs, V, precision=FX):
    Vd = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    Wd = torch.full_like(Vd, float("nan"))
    flz.flz_filter_apply(M.h, c, e, coeffs, len(coeffs) - 1, V.shape[1], Vd, Wd, precision)
    torch.cuda.synchronize()
    return Wd.cpu().numpy()


def fp64_bound(csr, c, e, m, V):
    S = csr.to_scipy()
    rowsum = np.asarray(abs(S).sum(axis=1)).ravel() + abs(c)
    return 32.0 * (m + 1) ** 2 * U64 * (1.0 + rowsum.max() / e) * np.max(np.abs(V))


def gershgorin_map(csr):
    S = csr.to_scipy()
    d = S.diagonal()
    rad = np.asarray(abs(S).sum(axis=1)).ravel() - np.abs(d)
    lo, hi = float(np.min(d - rad)), float(np.max(d + rad))
    return 0.5 * (lo + hi), 0.5 * (hi - lo)


def scaled_matrix(csr, c, e):
    """2 Ahat = (2/e)(A - cI) with the library's FP64 operations (s (a - c) per stored entry, s = 2/e)."""
    S = csr.to_scipy().tocsr().astype(np.float64)
    S.sort_indices()
    s = 2.0 / e
    data = S.data.copy()
    for i in range(S.shape[0]):
        for j in range(S.indptr[i], S.indptr[i + 1]):
            data[j] = s * (data[j] - (c if S.indices[j] == i else 0.0))
    return sp.csr_matrix((data, S.indices, S.indptr), shape=S.shape)


CASES = [
    ("lap2d_37x41", lambda: laplacian_2d(37, 41)),
    ("lap3d_pot_13x9x11", lambda: laplacian_3d_7pt(13, 9, 11, 0.5 * np.linspace(0, 1, 1287))),
    ("fd4_wells_10", lambda: fd4_laplacian_3d(10, gaussian_wells_potential(10, 5, seed=3))),
    ("graph_3000", lambda: powerlaw_graph_laplacian(3000, seed=2)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[x[0] for x in CASES])
@pytest.mark.parametrize("r", [1, 2, 3, 4, 8, 16])
def test_fixed_point_filter_matches_oracle(name, make, r):
    csr = make()
    c, e = gershgorin_map(csr)
    M = Mat(csr)
    m = 37
    coeffs = chebyshev.filter_coefficients(-0.8, -0.35, m)
    V = random_normal_block(csr.n, r, 300 + r)
    got = run_filter(M, c, e, coeffs, V)
    ref = chebyshev.clenshaw_apply(csr.to_scipy(), c, e, coeffs, V)
    err = np.max(np.abs(got - ref))
    assert err <= TIGHT * np.max(np.abs(V)), err
    assert err <= fp64_bound(csr, c, e, m, V)


@pytest.mark.parametrize("m", [0, 1, 2, 3, 4, 5, 6, 7, 50, 101, 200])
@pytest.mark.parametrize("r", [3, 4])
def test_fixed_point_filter_degrees(m, r):
    # degrees of every residue mod 3: the running sum takes its terms three
    # at a time, and the last degree adds the one or two still pending
    csr = laplacian_3d_7pt(12, 12, 12, 0.5 * np.linspace(0, 1, 1728))
    M = Mat(csr)
    coeffs = chebyshev.filter_coefficients(-1.0, -0.9, m)
    V = random_normal_block(csr.n, r, 7)
    got = run_filter(M, 6.25, 6.25, coeffs, V)
    ref = chebyshev.clenshaw_apply(csr.to_scipy(), 6.25, 6.25, coeffs, V)
    assert np.max(np.abs(got - ref)) <= TIGHT * np.max(np.abs(V))


@pytest.mark.parametrize("k", [0, 1, 2, 9, 64])
def test_single_term_is_cosine_on_a_diagonal_matrix(k):
    n = 5000
    d = np.cos(np.linspace(0.0, np.pi, n))
    from synth import diagonal_csr
    M = Mat(diagonal_csr(d))
    b = np.zeros(k + 1)
    b[k] = 1.0
    V = random_normal_block(n, 4, 1)
    got = run_filter(M, 0.0, 1.0, b, V)
    want = np.cos(k * np.arccos(d))[:, None] * V
    assert np.max(np.abs(got - want)) <= 64 * (k + 1) ** 2 * U64 * np.max(np.abs(V))


@pytest.mark.parametrize("k", range(11))
def test_single_term_inside_the_series_is_counted_once(k):
    # degree 10 with only b_k nonzero, for every k: each term enters the
    # running sum exactly once, whichever degree step adds it
    n = 5000
    d = np.cos(np.linspace(0.0, np.pi, n))
    from synth import diagonal_csr
    M = Mat(diagonal_csr(d))
    b = np.zeros(11)
    b[k] = 1.0
    V = random_normal_block(n, 4, 2)
    got = run_filter(M, 0.0, 1.0, b, V)
    want = np.cos(k * np.arccos(d))[:, None] * V
    assert np.max(np.abs(got - want)) <= 64 * 11 ** 2 * U64 * np.max(np.abs(V))


@pytest.mark.parametrize("name,make,r", [("lap3d_pot_13x9x11", CASES[1][1], 2), ("fd4_wells_8",
                                         lambda: fd4_laplacian_3d(8, gaussian_wells_potential(8, 4, seed=5)), 4),
                                         ("graph_1500", lambda: powerlaw_graph_laplacian(1500, seed=4), 3)])
def test_rounding_error_no_larger_than_fp64(name, make, r):
    # Reference: the same polynomial of the FP64-stored 2 Ahat in exact arithmetic.
    csr = make()
    c, e = gershgorin_map(csr)
    M = Mat(csr)
    m = 40
    coeffs = chebyshev.filter_coefficients(-0.7, -0.2, m)
    V = random_normal_block(csr.n, r, 21)
    exact = chebyshev.clenshaw_apply_exact(scaled_matrix(csr, c, e), coeffs, V)
    err_fx = np.linalg.norm(run_filter(M, c, e, coeffs, V, FX) - exact)
    err_64 = np.linalg.norm(run_filter(M, c, e, coeffs, V, flz.FLZ_PREC_FP64) - exact)
    assert err_fx <= err_64, (err_fx, err_64)


def test_spectrum_outside_the_unit_interval_is_reported():
    # 2D Laplacian, spectrum in (0, 8); c = 4, e = 2.1 maps it to about [-1.9, 1.9] (rows of 2 Ahat
    # sum to 3.81 in absolute value, inside the format's bound of 3.9):
    # T_k grows, the kernel flags the first value above 1.25 instead of wrapping.
    csr = laplacian_2d(30, 30)
    M = Mat(csr)
    V = random_normal_block(csr.n, 4, 3)
    coeffs = chebyshev.filter_coefficients(-0.5, 0.5, 60)
    Vd = torch.from_numpy(V).cuda()
    Wd = torch.zeros_like(Vd)
    with pytest.raises(flz.FlzError) as ei:
        flz.flz_filter_apply(M.h, 4.0, 2.1, coeffs, 60, 4, Vd, Wd, FX)
    assert ei.value.status == flz.FLZ_ERR_INVALID_ARG
    # the flag is cleared: a well-mapped call on the same handle succeeds
    got = run_filter(M, 4.0, 4.0, coeffs, V)
    ref = chebyshev.clenshaw_apply(csr.to_scipy(), 4.0, 4.0, coeffs, V)
    assert np.max(np.abs(got - ref)) <= TIGHT * np.max(np.abs(V))


def test_rows_too_large_for_the_format_run_in_fp64():
    # all-ones 40 x 40 block plus a diagonal: eigenvalues near 0..1 and 40, and
    # rows of 2 Ahat with absolute sums near 4 (beyond the fixed-point bound)
    n = 40
    H = np.ones((n, n)) + np.diag(np.linspace(0.0, 1.0, n))
    from synth.matrices import CSR
    S = sp.csr_matrix(H)
    csr = CSR(n, S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))
    c, e = gershgorin_map(csr)
    M = Mat(csr)
    coeffs = chebyshev.filter_coefficients(-1.0, -0.5, 30)
    V = random_normal_block(n, 4, 2)
    got = run_filter(M, c, e, coeffs, V)
    ref = chebyshev.clenshaw_apply(S, c, e, coeffs, V)
    assert np.max(np.abs(got - ref)) <= fp64_bound(csr, c, e, 30, V)


def solve(csr, alpha, beta, **kw):
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
    p = flz.flz_params_default()
    for k, v in kw.items():
        setattr(p, k, v)
    s = flz.flz_solver_create(h, p)
    flz.flz_solver_set_interval(s, alpha, beta)
    st = flz.flz_solve(s)
    out = {"status": st, "vals": flz.flz_get_eigenvalues(s), "res": flz.flz_get_residuals(s),
           "vecs": flz.get_eigenvectors_host(s, csr.n), "stats": flz.flz_get_stats(s)}
    flz.flz_solver_destroy(s)
    flz.flz_matrix_destroy(h)
    return out


def test_solver_with_the_fixed_point_filter_matches_closed_form():
    A = laplacian_3d_7pt(24, 24, 24)
    out = solve(A, 0.0, 0.436, block_size=4, degree=60, check_every=10, precision=FX)
    assert out["status"] == flz.FLZ_OK
    assert out["stats"]["filter_precision"] == FX
    k = np.arange(1, 25)
    lam = np.sort((6 - 2 * (np.cos(k[:, None, None] * np.pi / 25) + np.cos(k[None, :, None] * np.pi / 25) +
                            np.cos(k[None, None, :] * np.pi / 25))).ravel())
    want = lam[(lam >= 0.0) & (lam <= 0.436)]
    assert out["vals"].shape == want.shape and np.max(np.abs(out["vals"] - want)) < 1e-12
    X = out["vecs"]
    R = A.to_scipy() @ X - X * out["vals"]
    assert np.max(np.linalg.norm(R, axis=0)) / 12.0 < 1e-10
    assert np.max(np.abs(X.T @ X - np.eye(X.shape[1]))) < 1e-10


@pytest.mark.parametrize("r,expect", [(3, FX), (5, flz.FLZ_PREC_FP64)])
def test_solver_reports_the_filter_arithmetic(r, expect):
    from oracle import dense
    rng = np.random.Generator(np.random.PCG64(15))
    csr = laplacian_3d_7pt(12, 12, 12, 0.5 * rng.random(12 ** 3))
    w = np.linalg.eigvalsh(csr.to_dense())
    a, b = 0.5 * (w[19] + w[20]) - 1.0, 0.5 * (w[19] + w[20])
    out = solve(csr, a, b, block_size=r, degree=50, check_every=10, precision=FX)
    assert out["status"] == flz.FLZ_OK
    assert out["stats"]["filter_precision"] == expect
    ref = w[(w >= a) & (w <= b)]
    assert out["vals"].shape == ref.shape and np.max(np.abs(out["vals"] - ref)) < 1e-10 * 12.5
    assert dense.count_in_interval(csr.to_scipy(), a, b) == ref.shape[0]


def test_fd4_hamiltonian_vs_dense_with_the_fixed_point_filter():
    csr = fd4_laplacian_3d(11, gaussian_wells_potential(11, 6, seed=9))
    w = np.linalg.eigvalsh(csr.to_dense())
    a, b = w[0] - 1.0, 0.5 * (w[24] + w[25])
    out = solve(csr, a, b, block_size=4, degree=80, check_every=10, precision=FX)
    assert out["status"] == flz.FLZ_OK and out["stats"]["filter_precision"] == FX
    ref = w[(w >= a) & (w <= b)]
    norm_a = max(abs(out["stats"]["lmin"]), abs(out["stats"]["lmax"]))
    assert out["vals"].shape == ref.shape and np.max(np.abs(out["vals"] - ref)) < 1e-10 * norm_a


def test_full_size_config2_fixed_point_filter_matches_oracle():
    # n = 1e6, r = 4, the launch shape of the benchmark's solves
    rng = np.random.Generator(np.random.PCG64(2025))
    csr = laplacian_3d_7pt(100, 100, 100, 0.5 * rng.random(100 ** 3))
    M = Mat(csr)
    m = 60
    c, e = 6.25, 6.25
    coeffs = chebyshev.filter_coefficients(-1.0, (0.2885 - c) / e, m)
    V = random_normal_block(csr.n, 4, 77)
    got = run_filter(M, c, e, coeffs, V)
    ref = chebyshev.clenshaw_apply(csr.to_scipy(), c, e, coeffs, V)
    assert np.max(np.abs(got - ref)) <= TIGHT * np.max(np.abs(V))
