"""Parity of the hot path, W = p_m((A - cI)/e) V, against the CPU oracle.

The CUDA kernels evaluate the filter either by the forward three-term
recurrence fused with the running sum or by the Clenshaw recurrence; the
oracle uses the paper's Clenshaw recurrence in plain FP64 sparse products.
All are the same polynomial, so in FP64 they differ only by rounding.

Tolerance (FP64): element by element within 1e-12 of max|V| for degrees up to
200 (the observed errors are about 1e-15), and within the a-priori bound that
follows. A perturbation of size u in step j of a Chebyshev
recurrence reaches step k multiplied by a Chebyshev polynomial of the second
kind, |U_{k-j}| <= k - j + 1 on [-1, 1]; summing over the steps and the
coefficients (|b_k| <= 2/(k pi)) bounds the error of either method by a small
multiple of m^2 u max|V| times the row-sum of |Ahat|. The tests use
32 (m + 1)^2 u (1 + max row sum of |Ahat|) max|V|.

Reduced precision: FP32 storage and arithmetic give the same bound with the
FP32 unit roundoff; BF16 storage adds the BF16 rounding of every stored
vector, bounded the same way with u = 2^-8.
"""

import numpy as np
import pytest

import __graft_entry__
import paper_2409_15053_gb300 as flz
from oracle import chebyshev
from synth import (diagonal_csr, fd4_laplacian_3d, gaussian_wells_potential, laplacian_2d, laplacian_3d_7pt,
                   powerlaw_graph_laplacian, random_normal_block)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24
UBF = 2.0 ** -8
UDF = 2.0 ** -44  # double-FP32: 48 stored bits, a few bits lost per compensated operation


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


def run_filter(M, c, e, coeffs, V, precision=flz.FLZ_PREC_FP64, rec=flz.FLZ_REC_FORWARD):
    Vd = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    Wd = torch.full_like(Vd, float("nan"))
    flz.flz_filter_apply(M.h, c, e, coeffs, len(coeffs) - 1, V.shape[1], Vd, Wd, precision, recurrence=rec)
    torch.cuda.synchronize()
    return Wd.cpu().numpy()


def bound(csr, c, e, m, V, u):
    S = csr.to_scipy()
    rowsum = np.asarray(abs(S).sum(axis=1)).ravel() + abs(c)
    return 32.0 * (m + 1) ** 2 * u * (1.0 + rowsum.max() / e) * np.max(np.abs(V))


def gershgorin_map(csr):
    S = csr.to_scipy()
    d = S.diagonal()
    rad = np.asarray(abs(S).sum(axis=1)).ravel() - np.abs(d)
    lo, hi = float(np.min(d - rad)), float(np.max(d + rad))
    return 0.5 * (lo + hi), 0.5 * (hi - lo)


RECS = [flz.FLZ_REC_FORWARD, flz.FLZ_REC_CLENSHAW]
REC_IDS = ["forward", "clenshaw"]

CASES = [
    ("lap2d_37x41", lambda: laplacian_2d(37, 41)),
    ("lap3d_pot_13x9x11", lambda: laplacian_3d_7pt(13, 9, 11, 0.5 * np.linspace(0, 1, 1287))),
    ("fd4_wells_10", lambda: fd4_laplacian_3d(10, gaussian_wells_potential(10, 5, seed=3))),
    ("graph_3000", lambda: powerlaw_graph_laplacian(3000, seed=2)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[x[0] for x in CASES])
@pytest.mark.parametrize("r", [1, 2, 3, 4, 5, 8, 16])
@pytest.mark.parametrize("rec", RECS, ids=REC_IDS)
def test_fp64_filter_matches_oracle(name, make, r, rec):
    csr = make()
    c, e = gershgorin_map(csr)
    M = Mat(csr)
    m = 37
    coeffs = chebyshev.filter_coefficients(-0.8, -0.35, m)
    V = random_normal_block(csr.n, r, 100 + r)
    got = run_filter(M, c, e, coeffs, V, rec=rec)
    ref = chebyshev.clenshaw_apply(csr.to_scipy(), c, e, coeffs, V)
    assert np.all(np.isfinite(got))
    # element by element within 1e-12 of max|V| (the a-priori rounding bound
    # below is the second, looser assertion)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(V))
    assert np.max(np.abs(got - ref)) <= bound(csr, c, e, m, V, U64)


@pytest.mark.parametrize("m", [0, 1, 2, 3, 4, 50, 200])
@pytest.mark.parametrize("rec", RECS, ids=REC_IDS)
def test_fp64_filter_degrees(m, rec):
    csr = laplacian_3d_7pt(12, 12, 12)
    M = Mat(csr)
    coeffs = chebyshev.filter_coefficients(-1.0, -0.9, m)
    V = random_normal_block(csr.n, 4, 7)
    got = run_filter(M, 6.0, 6.0, coeffs, V, rec=rec)
    ref = chebyshev.clenshaw_apply(csr.to_scipy(), 6.0, 6.0, coeffs, V)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(V))
    assert np.max(np.abs(got - ref)) <= bound(csr, 6.0, 6.0, m, V, U64)


@pytest.mark.parametrize("k", [0, 1, 2, 9, 64])
@pytest.mark.parametrize("rec", RECS, ids=REC_IDS)
def test_single_term_is_cosine_on_a_diagonal_matrix(k, rec):
    # T_k(x) = cos(k arccos x): with b = e_k the kernel must return cos(k acos d) * V
    n = 5000
    d = np.cos(np.linspace(0.0, np.pi, n))
    M = Mat(diagonal_csr(d))
    b = np.zeros(k + 1)
    b[k] = 1.0
    V = random_normal_block(n, 4, 1)
    got = run_filter(M, 0.0, 1.0, b, V, rec=rec)
    want = np.cos(k * np.arccos(d))[:, None] * V
    assert np.max(np.abs(got - want)) <= 64 * (k + 1) ** 2 * U64 * np.max(np.abs(V))


def test_laplacian_eigenvector_identity():
    nx, ny = 40, 50
    M = Mat(laplacian_2d(nx, ny))
    c, e = 4.0, 4.0
    b = chebyshev.filter_coefficients(-0.7, -0.4, 120)
    x = np.arange(1, nx + 1)[:, None]
    y = np.arange(1, ny + 1)[None, :]
    cols, want = [], []
    for (i, j) in [(1, 1), (5, 9), (17, 3), (40, 50)]:
        u = (np.sin(i * np.pi * x / (nx + 1)) * np.sin(j * np.pi * y / (ny + 1))).T.reshape(-1)
        lam = 4 - 2 * np.cos(i * np.pi / (nx + 1)) - 2 * np.cos(j * np.pi / (ny + 1))
        z = (lam - c) / e
        cols.append(u)
        want.append(np.sum(b * np.cos(np.arange(121) * np.arccos(z))) * u)
    U = np.stack(cols, axis=1)
    got = run_filter(M, c, e, b, U)
    assert np.max(np.abs(got - np.stack(want, axis=1))) < 1e-11


@pytest.mark.parametrize("precision,u", [(flz.FLZ_PREC_FP32, U32), (flz.FLZ_PREC_BF16, UBF), (flz.FLZ_PREC_DF64, UDF)])
@pytest.mark.parametrize("rec", RECS, ids=REC_IDS)
@pytest.mark.parametrize("r", [3, 4])
def test_reduced_precision_filter_within_bound(precision, u, rec, r):
    csr = laplacian_3d_7pt(16, 16, 16, 0.5 * np.linspace(0, 1, 4096))
    M = Mat(csr)
    m = 30
    coeffs = chebyshev.filter_coefficients(-1.0, -0.9, m)
    V = random_normal_block(csr.n, r, 5)
    got = run_filter(M, 6.25, 6.25, coeffs, V, precision, rec)
    ref = chebyshev.clenshaw_apply(csr.to_scipy(), 6.25, 6.25, coeffs, V)
    err = np.max(np.abs(got - ref))
    assert err <= bound(csr, 6.25, 6.25, m, V, u)
    # and it is a real approximation, not noise
    assert err < 0.5 * np.max(np.abs(ref))


def test_filter_rejects_overlapping_buffers():
    csr = laplacian_2d(10, 10)
    M = Mat(csr)
    Vd = torch.zeros((100, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(flz.FlzError) as e:
        flz.flz_filter_apply(M.h, 4.0, 4.0, np.ones(3), 2, 4, Vd, Vd)
    assert e.value.status == flz.FLZ_ERR_INVALID_ARG
    Wd = torch.zeros_like(Vd)
    with pytest.raises(flz.FlzError) as e:
        flz.flz_filter_apply(M.h, 4.0, 4.0, np.ones(3), 2, 4, Vd, Wd, recurrence=2)
    assert e.value.status == flz.FLZ_ERR_INVALID_ARG


@pytest.mark.parametrize("rec", RECS, ids=REC_IDS)
def test_full_size_config2_filter_matches_oracle(rec):
    # 100^3 grid (n = 1e6, 6.94e6 nnz), r = 4, the launch shape the solver uses
    rng = np.random.Generator(np.random.PCG64(2025))
    csr = laplacian_3d_7pt(100, 100, 100, 0.5 * rng.random(100 ** 3))
    M = Mat(csr)
    m = 60
    lmin, lmax = 0.0, 12.5
    c, e = 0.5 * (lmin + lmax), 0.5 * (lmax - lmin)
    coeffs = chebyshev.filter_coefficients(-1.0, (0.2885 - c) / e, m)
    V = random_normal_block(csr.n, 4, 77)
    got = run_filter(M, c, e, coeffs, V, rec=rec)
    ref = chebyshev.clenshaw_apply(csr.to_scipy(), c, e, coeffs, V)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(V))
    assert np.max(np.abs(got - ref)) <= bound(csr, c, e, m, V, U64)


@pytest.mark.parametrize("rec", RECS, ids=REC_IDS)
def test_rows_without_stored_diagonal(rec):
    # The filter folds -cI into the stored diagonal; rows that store no a_ii get
    # an explicit zero at creation. A symmetric matrix with most diagonals absent:
    S = laplacian_2d(23, 19).to_scipy().tolil()
    for i in range(0, 23 * 19, 3):
        S[i, i] = 0.0
    S = S.tocsr()
    S.eliminate_zeros()
    from synth.matrices import CSR
    csr = CSR(S.shape[0], S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))
    M = Mat(csr)
    n, nnz, glo, ghi = flz.flz_matrix_info(M.h)
    assert nnz == csr.nnz  # reports the caller's entries
    c, e = gershgorin_map(csr)
    coeffs = chebyshev.filter_coefficients(-0.5, 0.1, 41)
    V = random_normal_block(csr.n, 3, 9)
    got = run_filter(M, c, e, coeffs, V, rec=rec)
    ref = chebyshev.clenshaw_apply(S, c, e, coeffs, V)
    assert np.max(np.abs(got - ref)) <= bound(csr, c, e, 41, V, U64)


@pytest.mark.parametrize("r", [1, 4, 16])
@pytest.mark.parametrize("precision,u", [(flz.FLZ_PREC_FP64, U64), (flz.FLZ_PREC_FP32, U32)])
@pytest.mark.parametrize("rec", RECS, ids=REC_IDS)
def test_hub_rows_use_the_long_row_tier(r, precision, u, rec):
    # A power-law graph with i0 = 1 has hubs with thousands of entries, far
    # above the 256-entry threshold of the row-per-thread kernel.
    csr = powerlaw_graph_laplacian(20000, seed=11, i0=1)
    assert np.diff(csr.rowptr).max() > 1000
    c, e = gershgorin_map(csr)
    M = Mat(csr)
    m = 25
    coeffs = chebyshev.filter_coefficients(-0.95, -0.7, m)
    V = random_normal_block(csr.n, r, 13)
    got = run_filter(M, c, e, coeffs, V, precision, rec)
    ref = chebyshev.clenshaw_apply(csr.to_scipy(), c, e, coeffs, V)
    assert np.max(np.abs(got - ref)) <= bound(csr, c, e, m, V, u)


@pytest.mark.parametrize("r", [1, 3, 4, 16])
@pytest.mark.parametrize("rec", RECS, ids=REC_IDS)
def test_double_fp32_filter_matches_oracle(r, rec):
    csr = fd4_laplacian_3d(10, gaussian_wells_potential(10, 5, seed=3))
    c, e = gershgorin_map(csr)
    M = Mat(csr)
    m = 80
    coeffs = chebyshev.filter_coefficients(-0.9, -0.6, m)
    V = random_normal_block(csr.n, r, 40 + r)
    got = run_filter(M, c, e, coeffs, V, flz.FLZ_PREC_DF64, rec)
    ref = chebyshev.clenshaw_apply(csr.to_scipy(), c, e, coeffs, V)
    assert np.max(np.abs(got - ref)) <= bound(csr, c, e, m, V, UDF)


@pytest.mark.parametrize("r", [1, 4])
@pytest.mark.parametrize("rec", RECS, ids=REC_IDS)
def test_jackson_damped_filter_matches_oracle(r, rec):
    # The kernels take any coefficient vector; the damped one comes from the
    # library's own factors and is checked against the oracle's series.
    csr = laplacian_3d_7pt(13, 9, 11, 0.5 * np.linspace(0, 1, 1287))
    c, e = gershgorin_map(csr)
    m = 90
    coeffs = flz.flz_filter_coefficients(-0.6, -0.3, m) * flz.flz_jackson_factors(m)
    ref_coeffs = chebyshev.damped_filter_coefficients(-0.6, -0.3, m)
    assert np.max(np.abs(coeffs - ref_coeffs)) < 1e-14
    V = random_normal_block(csr.n, r, 29)
    W = run_filter(Mat(csr), c, e, coeffs, V, rec=rec)
    ref = chebyshev.clenshaw_apply(csr.to_scipy(), c, e, ref_coeffs, V)
    assert np.max(np.abs(W - ref)) < bound(csr, c, e, m, V, U64)


def _stencil_with_hub(g=20, hub_degree=400, seed=17):
    # 3D Laplacian (regular rows: the SELL-32 layout applies) plus one hub
    # vertex joined to `hub_degree` grid points (a row far above 256 entries,
    # left to the CTA-per-row kernel next to SELL).
    import scipy.sparse as sp
    from synth.matrices import CSR
    S = laplacian_3d_7pt(g, g, g, 0.5 * np.linspace(0, 1, g ** 3)).to_scipy().tolil()
    n = g ** 3
    S.resize((n + 1, n + 1))
    rng = np.random.Generator(np.random.PCG64(seed))
    nb = rng.choice(n, hub_degree, replace=False)
    w = 0.1 + 0.9 * rng.random(hub_degree)
    for j, x in zip(nb, w):
        S[n, j] = -x
        S[j, n] = -x
        S[j, j] = S[j, j] + x
    S[n, n] = w.sum()
    S = sp.csr_matrix(S)
    S.sort_indices()
    return CSR(n + 1, S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))


@pytest.mark.parametrize("rec", RECS, ids=REC_IDS)
@pytest.mark.parametrize("precision,u", [(flz.FLZ_PREC_FP64, U64), (flz.FLZ_PREC_FP32, U32), (flz.FLZ_PREC_DF64, UDF)])
@pytest.mark.parametrize("r", [1, 3, 4, 16])
def test_regular_rows_with_a_hub(r, precision, u, rec):
    csr = _stencil_with_hub()
    assert np.diff(csr.rowptr).max() > 256
    c, e = gershgorin_map(csr)
    M = Mat(csr)
    sell, entries, long_rows = flz.flz_matrix_format(M.h)
    assert sell == 1 and long_rows == 1 and csr.nnz <= entries <= 1.3 * csr.nnz
    m = 45
    coeffs = chebyshev.filter_coefficients(-0.9, -0.5, m)
    V = random_normal_block(csr.n, r, 23)
    got = run_filter(M, c, e, coeffs, V, precision, rec)
    ref = chebyshev.clenshaw_apply(csr.to_scipy(), c, e, coeffs, V)
    assert np.max(np.abs(got - ref)) <= bound(csr, c, e, m, V, u)


def test_storage_format_choice():
    # regular stencils get the SELL-32 layout; power-law graphs (rows from 2 to
    # thousands of entries) stay in CSR with their hubs in the long-row tier
    M = Mat(laplacian_3d_7pt(30, 30, 30))
    sell, entries, long_rows = flz.flz_matrix_format(M.h)
    assert sell == 1 and long_rows == 0 and entries >= M.csr.nnz
    G = Mat(powerlaw_graph_laplacian(20000, seed=11, i0=1))
    sell, entries, long_rows = flz.flz_matrix_format(G.h)
    assert sell == 0 and entries == 0 and long_rows > 0


@pytest.mark.slow
def test_full_size_power_law_graph_filter_matches_oracle():
    # The irregular workload at full size (n = 4e6, 64e6 stored entries, 9211
    # rows above 256 entries), r = 16 as the graph benchmark runs it: staged
    # CSR rows plus the CTA-per-row tier for the hubs, against the oracle's
    # Clenshaw evaluation (low degree keeps the CPU side to seconds).
    csr = powerlaw_graph_laplacian(4_000_000, seed=5)
    assert np.diff(csr.rowptr).max() > 256
    c, e = gershgorin_map(csr)
    M = Mat(csr)
    sell, _, long_rows = flz.flz_matrix_format(M.h)
    assert sell == 0 and long_rows > 1000
    m = 6
    coeffs = chebyshev.filter_coefficients(0.6, 1.0, m)
    V = random_normal_block(csr.n, 16, 61)
    got = run_filter(M, c, e, coeffs, V)
    ref = chebyshev.clenshaw_apply(csr.to_scipy(), c, e, coeffs, V)
    assert np.max(np.abs(got - ref)) <= bound(csr, c, e, m, V, U64)
