"""End-to-end parity of the GPU filtered Lanczos solver against closed forms,
the CPU oracle's dense definition, and its error statuses.

Bar: the count in [alpha, beta] is exact (with multiplicity); FP64
eigenvalues agree within 1e-10 relative to ||A||; every returned pair has
||Ax - lambda x|| / ||A|| <= tol recomputed here on the CPU; the returned
eigenvectors are orthonormal to 1e-10.
"""

import numpy as np
import pytest

import __graft_entry__
import paper_2409_15053_gb300 as flz
from oracle import dense
from synth import (fd4_laplacian_3d, gaussian_wells_potential, laplacian_2d, laplacian_3d_7pt,
                   powerlaw_graph_laplacian)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CFG1_ALPHA, CFG1_BETA = 0.9198764447231507, 1.0094761615910202


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


def lap2d_eigs(nx, ny):
    i = np.arange(1, nx + 1)[:, None]
    j = np.arange(1, ny + 1)[None, :]
    return np.sort((4 - 2 * np.cos(i * np.pi / (nx + 1)) - 2 * np.cos(j * np.pi / (ny + 1))).ravel())


def gap_interval(eigs, lo_index, count):
    a = 0.5 * (eigs[lo_index - 1] + eigs[lo_index]) if lo_index > 0 else eigs[0] - 1.0
    b = 0.5 * (eigs[lo_index + count - 1] + eigs[lo_index + count])
    return a, b


def solve(csr, alpha, beta, **kw):
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
    p = flz.flz_params_default()
    for k, v in kw.items():
        setattr(p, k, v)
    s = flz.flz_solver_create(h, p)
    flz.flz_solver_set_interval(s, alpha, beta)
    st = flz.flz_solve(s)
    out = {
        "status": st,
        "vals": flz.flz_get_eigenvalues(s),
        "res": flz.flz_get_residuals(s),
        "vecs": flz.get_eigenvectors_host(s, csr.n),
        "stats": flz.flz_get_stats(s),
    }
    flz.flz_solver_destroy(s)
    flz.flz_matrix_destroy(h)
    return out


def check_pairs(csr, out, tol, ortho=1e-10):
    S = csr.to_scipy()
    X = out["vecs"]
    lam = out["vals"]
    norm_a = max(abs(out["stats"]["lmin"]), abs(out["stats"]["lmax"]))
    R = S @ X - X * lam
    res = np.linalg.norm(R, axis=0) / norm_a
    assert np.all(res <= tol), res.max()
    G = np.abs(X.T @ X - np.eye(X.shape[1]))
    i, j = np.unravel_index(np.argmax(G), G.shape)
    assert G[i, j] < ortho, (int(i), int(j), float(lam[i]), float(lam[j]), float(G[i, j]), float(res[i]), float(res[j]))


def sliced_ortho_bound(eigs, tol, norm_a):
    # Eigenvectors from different slices come from different Krylov bases:
    # for unit x_i, x_j with residuals r_i, r_j <= tol ||A|| and eigenvalues
    # separated by g, |x_i^T x_j| <= (r_i + r_j) / g (one solve's vectors are
    # orthonormal to rounding). g = the smallest gap between distinct
    # eigenvalues of the window.
    d = np.diff(np.unique(np.round(eigs, 12)))
    return max(1e-10, 2.0 * tol * norm_a / d.min())


@pytest.mark.parametrize("rec", [flz.FLZ_REC_FORWARD, flz.FLZ_REC_CLENSHAW], ids=["forward", "clenshaw"])
@pytest.mark.parametrize("r", [1, 2])
def test_config1_window_matches_closed_form(r, rec):
    csr = laplacian_2d(50, 50)
    lam = lap2d_eigs(50, 50)
    ref = lam[(lam >= CFG1_ALPHA) & (lam <= CFG1_BETA)]
    out = solve(csr, CFG1_ALPHA, CFG1_BETA, block_size=r, degree=50, recurrence=rec)
    assert out["status"] == flz.FLZ_OK
    assert out["vals"].shape == ref.shape == (20,)
    assert np.max(np.abs(out["vals"] - ref)) < 1e-10 * 8.0
    check_pairs(csr, out, 1e-10)
    st = out["stats"]
    assert st["matvecs"] == r * 50 * st["iters"] and st["degree"] == 50 and st["converged"] == 1


def _dense_case(csr, lo_index, count, **kw):
    w = np.linalg.eigvalsh(csr.to_dense())
    a, b = gap_interval(w, lo_index, count)
    out = solve(csr, a, b, **kw)
    ref = w[(w >= a) & (w <= b)]
    assert out["status"] == flz.FLZ_OK
    assert out["vals"].shape == ref.shape
    scale = max(abs(w[0]), abs(w[-1]))
    assert np.max(np.abs(out["vals"] - ref)) < 1e-10 * scale
    check_pairs(csr, out, kw.get("tol", 1e-10))
    return out


def test_3d_laplacian_potential_vs_dense_auto_degree():
    rng = np.random.Generator(np.random.PCG64(5))
    _dense_case(laplacian_3d_7pt(12, 12, 12, 0.5 * rng.random(1728)), 0, 40, block_size=4)


def test_fd4_hamiltonian_vs_dense():
    N = 11
    _dense_case(fd4_laplacian_3d(N, gaussian_wells_potential(N, 8, seed=2)), 3, 25, block_size=4)


def test_powerlaw_graph_vs_dense():
    _dense_case(powerlaw_graph_laplacian(2000, seed=7), 40, 15, block_size=4, degree=60)


@pytest.mark.parametrize("rec", [flz.FLZ_REC_FORWARD, flz.FLZ_REC_CLENSHAW], ids=["forward", "clenshaw"])
def test_interior_window_block3_vs_dense(rec):
    rng = np.random.Generator(np.random.PCG64(8))
    _dense_case(laplacian_3d_7pt(10, 11, 12, rng.random(1320)), 500, 30, block_size=3, degree=80, recurrence=rec)


@pytest.mark.parametrize("damping,transition", [(1, 0.0), (2, 0.0), (0, 0.02)],
                         ids=["jackson", "sigma", "smoothed-step"])
def test_damped_filter_vs_dense(damping, transition):
    # Damping and the least-squares smoothed step widen the filter's
    # transition band and tame the Gibbs oscillations; the solver must still
    # return every eigenvalue of the window.
    rng = np.random.Generator(np.random.PCG64(8))
    out = _dense_case(laplacian_3d_7pt(10, 11, 12, rng.random(1320)), 500, 30, block_size=3, degree=120,
                      damping=damping, transition=transition)
    assert out["stats"]["degree"] == 120


def test_count_matches_inertia_midsize():
    rng = np.random.Generator(np.random.PCG64(9))
    csr = laplacian_3d_7pt(20, 20, 20, 0.5 * rng.random(8000))
    S = csr.to_scipy()
    # endpoints placed in gaps of the spectrum found by inertia counting
    a = 0.35
    b = 0.80
    cnt = dense.count_in_interval(S, a, b)
    out = solve(csr, a, b, block_size=4, degree=60)
    assert out["status"] == flz.FLZ_OK
    assert out["vals"].shape[0] == cnt
    check_pairs(csr, out, 1e-10)


def test_spectrum_bounds_enclose_extremes():
    csr = laplacian_2d(60, 60)
    lam = lap2d_eigs(60, 60)
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
    lo, hi = flz.flz_spectrum_bounds(h, 60, 4, 3)
    n, nnz, glo, ghi = flz.flz_matrix_info(h)
    flz.flz_matrix_destroy(h)
    assert (n, nnz) == (3600, csr.nnz)
    assert glo <= lo <= lam[0] and lam[-1] <= hi <= ghi


def test_empty_interval_status():
    csr = laplacian_2d(20, 20)
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
    s = flz.flz_solver_create(h, None)
    flz.flz_solver_set_interval(s, 9.0, 10.0)
    with pytest.raises(flz.FlzError) as e:
        flz.flz_solve(s)
    assert e.value.status == flz.FLZ_ERR_EMPTY_INTERVAL
    flz.flz_solver_destroy(s)
    flz.flz_matrix_destroy(h)


def test_not_converged_keeps_partial_results():
    csr = laplacian_2d(50, 50)
    out = solve(csr, CFG1_ALPHA, CFG1_BETA, block_size=1, degree=50, max_basis=40, check_every=40)
    assert out["status"] == flz.FLZ_ERR_NOT_CONVERGED
    assert out["stats"]["converged"] == 0 and out["stats"]["iters"] == 40
    assert out["vals"].shape[0] == out["stats"]["count"]


def test_call_order_and_capacity_errors():
    csr = laplacian_2d(20, 20)
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
    s = flz.flz_solver_create(h, None)
    with pytest.raises(flz.FlzError) as e:
        flz.flz_solve(s)
    assert e.value.status == flz.FLZ_ERR_NO_INTERVAL
    with pytest.raises(flz.FlzError) as e:
        flz.flz_get_count(s)
    assert e.value.status == flz.FLZ_ERR_NOT_SOLVED
    lam = lap2d_eigs(20, 20)
    a, b = gap_interval(lam, 0, 6)
    flz.flz_solver_set_interval(s, a, b)
    assert flz.flz_solve(s) == flz.FLZ_OK
    with pytest.raises(flz.FlzError) as e:
        flz.flz_get_eigenvalues(s, np.empty(2))
    assert e.value.status == flz.FLZ_ERR_CAPACITY
    flz.flz_solver_destroy(s)
    p = flz.flz_params_default()
    p.damping = 3
    with pytest.raises(flz.FlzError) as e:
        flz.flz_solver_create(h, p)
    assert e.value.status == flz.FLZ_ERR_INVALID_ARG
    flz.flz_matrix_destroy(h)


def test_invalid_csr_is_rejected():
    csr = laplacian_2d(6, 6)
    bad_cols = csr.col.copy()
    bad_cols[0], bad_cols[1] = bad_cols[1], bad_cols[0]  # unsorted row 0
    with pytest.raises(flz.FlzError) as e:
        flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, bad_cols, csr.val)
    assert e.value.status == flz.FLZ_ERR_BAD_CSR
    bad_ptr = csr.rowptr.copy()
    bad_ptr[-1] -= 1
    with pytest.raises(flz.FlzError) as e:
        flz.flz_matrix_create_csr(csr.n, csr.nnz, bad_ptr, csr.col, csr.val)
    assert e.value.status == flz.FLZ_ERR_BAD_CSR
    bad_val = csr.val.copy()
    bad_val[1] += 0.5  # a_01 != a_10
    with pytest.raises(flz.FlzError) as e:
        flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, bad_val)
    assert e.value.status == flz.FLZ_ERR_NOT_SYMMETRIC


def test_device_resident_csr_input():
    csr = laplacian_2d(30, 30)
    rp = torch.from_numpy(csr.rowptr).cuda()
    cl = torch.from_numpy(csr.col).cuda()
    vl = torch.from_numpy(csr.val).cuda()
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, rp, cl, vl, flz.FLZ_F64, flz.FLZ_DEVICE)
    n, nnz, glo, ghi = flz.flz_matrix_info(h)
    flz.flz_matrix_destroy(h)
    assert (n, nnz, glo, ghi) == (900, csr.nnz, 0.0, 8.0)


@pytest.mark.parametrize("precision,rec", [(flz.FLZ_PREC_FP64, flz.FLZ_REC_FORWARD), (flz.FLZ_PREC_DF64, flz.FLZ_REC_FORWARD),
                                           (flz.FLZ_PREC_FP64, flz.FLZ_REC_CLENSHAW),
                                           (flz.FLZ_PREC_DF64, flz.FLZ_REC_CLENSHAW),
                                           (flz.FLZ_PREC_FX64, flz.FLZ_REC_FORWARD)],
                         ids=["fp64-forward", "df64-forward", "fp64-clenshaw", "df64-clenshaw", "fx64-forward"])
def test_full_size_config2_matches_oracle_reference(precision, rec):
    # n = 1e6, nnz = 6.94e6, r = 4, m = 60: the benchmark's configuration,
    # against the eigenvalues the CPU oracle computed (tests/golden).
    import json
    import os
    from synth.workloads import CONFIG2
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "config2_reference.json")))
    rng = np.random.Generator(np.random.PCG64(CONFIG2["seed"]))
    g = CONFIG2["grid"]
    csr = laplacian_3d_7pt(g, g, g, CONFIG2["potential_scale"] * rng.random(g ** 3))
    out = solve(csr, CONFIG2["alpha"], CONFIG2["beta"], block_size=4, degree=CONFIG2["degree"],
                check_every=CONFIG2["check_every"], precision=precision, recurrence=rec)
    want = np.array(ref["eigenvalues"])
    assert out["status"] == flz.FLZ_OK
    assert out["vals"].shape == want.shape == (CONFIG2["count"],)
    norm_a = max(abs(out["stats"]["lmin"]), abs(out["stats"]["lmax"]))
    assert np.max(np.abs(out["vals"] - want)) < 1e-10 * norm_a
    check_pairs(csr, out, 1e-10)


@pytest.mark.parametrize("precision,tol,eig_tol", [(flz.FLZ_PREC_FP32, 1e-6, 1e-9), (flz.FLZ_PREC_BF16, 1e-2, 1e-2),
                                                   (flz.FLZ_PREC_DF64, 1e-10, 1e-10)])
def test_reduced_precision_filter(precision, tol, eig_tol):
    # FP32 / BF16: the filter runs in FP32 (or BF16 storage with FP32 sums);
    # everything else is FP64. The filtered Lanczos relation then holds only to
    # the filter's rounding, which bounds the attainable residual: about 1e-7
    # in FP32; in BF16 the stored values of 2 Ahat alone perturb A by up to
    # 2^-9 of its row sums (about 2e-3 ||A|| here), so 1e-2 is the tolerance
    # the arithmetic supports. FP32 eigenvalue errors are of the order of the
    # squared residual (FP64 Rayleigh quotients); for BF16 the bound is Kahan's,
    # |lambda - lambda_i| <= ||r|| (residual tol times ||A||). DF64: the whole
    # basis in double-FP32, FP64-class results. Count exact, residuals <= tol.
    rng = np.random.Generator(np.random.PCG64(15))
    csr = laplacian_3d_7pt(14, 14, 14, 0.5 * rng.random(14 ** 3))
    w = np.linalg.eigvalsh(csr.to_dense())
    a, b = gap_interval(w, 0, 30)
    out = solve(csr, a, b, block_size=4, degree=60, precision=precision, tol=tol, check_every=10)
    ref = w[(w >= a) & (w <= b)]
    assert out["status"] == flz.FLZ_OK
    assert out["vals"].shape == ref.shape
    norm_a = max(abs(out["stats"]["lmin"]), abs(out["stats"]["lmax"]))
    assert np.max(np.abs(out["vals"] - ref)) < eig_tol * norm_a
    check_pairs(csr, out, tol)


def solve_sliced(csr, alpha, beta, nslices, **kw):
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
    p = flz.flz_params_default()
    for k, v in kw.items():
        setattr(p, k, v)
    s = flz.flz_solver_create(h, p)
    flz.flz_solver_set_interval(s, alpha, beta)
    st = flz.flz_solve_sliced(s, nslices)
    out = {"status": st, "vals": flz.flz_get_eigenvalues(s), "res": flz.flz_get_residuals(s),
           "vecs": flz.get_eigenvectors_host(s, csr.n), "stats": flz.flz_get_stats(s)}
    flz.flz_solver_destroy(s)
    flz.flz_matrix_destroy(h)
    return out


@pytest.mark.parametrize("nslices", [2, 3])
def test_sliced_solve_matches_dense(nslices):
    rng = np.random.Generator(np.random.PCG64(21))
    csr = laplacian_3d_7pt(12, 12, 12, 0.5 * rng.random(1728))
    w = np.linalg.eigvalsh(csr.to_dense())
    a, b = gap_interval(w, 0, 45)
    out = solve_sliced(csr, a, b, nslices, block_size=4, degree=80, check_every=10)
    ref = w[(w >= a) & (w <= b)]
    assert out["status"] == flz.FLZ_OK
    assert out["vals"].shape == ref.shape
    assert np.all(np.diff(out["vals"]) >= 0)
    norm_a = max(abs(out["stats"]["lmin"]), abs(out["stats"]["lmax"]))
    assert np.max(np.abs(out["vals"] - ref)) < 1e-10 * norm_a
    check_pairs(csr, out, 1e-10, sliced_ortho_bound(ref, 1e-10, norm_a))


def test_slice_endpoint_on_a_double_eigenvalue():
    # A diagonal matrix whose double eigenvalue 0.5 sits exactly on the shared
    # endpoint of two slices of [0.1, 0.9]: both slices see the whole
    # eigenspace; the merged result must hold it twice, not four times, with
    # orthonormal eigenvectors.
    d = np.concatenate([np.linspace(0.0, 1.0, 201), [0.5]])
    d = np.sort(d)
    from synth import diagonal_csr
    csr = diagonal_csr(d)
    ref = d[(d >= 0.1) & (d <= 0.9)]
    out = solve_sliced(csr, 0.1, 0.9, 2, block_size=2, degree=60, check_every=10, lmin=-0.001, lmax=1.001)
    assert out["status"] == flz.FLZ_OK
    assert out["vals"].shape == ref.shape
    assert np.max(np.abs(out["vals"] - ref)) < 1e-10
    check_pairs(csr, out, 1e-10, sliced_ortho_bound(ref, 1e-10, 1.001))
    # the two copies of 0.5 span the eigenspace: orthonormal to rounding
    X = out["vecs"]
    k = np.nonzero(np.abs(out["vals"] - 0.5) < 1e-9)[0]
    assert k.shape == (2,)
    assert np.max(np.abs(X[:, k].T @ X[:, k] - np.eye(2))) < 1e-12


def test_sliced_rejects_bad_count():
    csr = laplacian_2d(10, 10)
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
    s = flz.flz_solver_create(h, None)
    flz.flz_solver_set_interval(s, 0.1, 1.0)
    with pytest.raises(flz.FlzError) as e:
        flz.flz_solve_sliced(s, 0)
    assert e.value.status == flz.FLZ_ERR_INVALID_ARG
    flz.flz_solver_destroy(s)
    flz.flz_matrix_destroy(h)


def test_full_size_fd4_hamiltonian_fp64_df64_and_fixed_point():
    # The 120^3 4th-order FD Hamiltonian with 64 Gaussian wells (n = 1.728e6,
    # nnz = 22.2e6), all eigenpairs in [-6, 0] (the wells' bound states): at
    # this size no dense or oracle count is affordable, so the checks are the
    # properties that hold at any size -- residuals recomputed here, orthonormal
    # eigenvectors (k orthonormal vectors with residuals <= tol ||A|| certify k
    # eigenvalues within tol ||A|| of the computed ones) -- and the agreement of
    # three independent arithmetics: FP64, double-FP32 and the 64-bit fixed-point
    # filter must return the same count and eigenvalues. Scaled-down instances are checked against dense
    # eigensolves (test_fd4_hamiltonian_vs_dense).
    from synth.workloads import CONFIG3
    N = CONFIG3["grid"]
    csr = fd4_laplacian_3d(N, gaussian_wells_potential(N, CONFIG3["wells"], seed=CONFIG3["seed"]))
    outs = {}
    for prec in (flz.FLZ_PREC_FP64, flz.FLZ_PREC_DF64, flz.FLZ_PREC_FX64):
        outs[prec] = solve(csr, CONFIG3["alpha"], 0.0, block_size=4, degree=300, check_every=10, precision=prec)
        assert outs[prec]["status"] == flz.FLZ_OK
    a, b, f = outs[flz.FLZ_PREC_FP64], outs[flz.FLZ_PREC_DF64], outs[flz.FLZ_PREC_FX64]
    assert f["stats"]["filter_precision"] == flz.FLZ_PREC_FX64
    assert a["vals"].shape == b["vals"].shape == f["vals"].shape and a["vals"].shape[0] > 40
    norm_a = max(abs(a["stats"]["lmin"]), abs(a["stats"]["lmax"]))
    assert np.max(np.abs(a["vals"] - b["vals"])) < 1e-10 * norm_a
    assert np.max(np.abs(a["vals"] - f["vals"])) < 1e-10 * norm_a
    check_pairs(csr, a, 1e-10)
    check_pairs(csr, b, 1e-10)
    check_pairs(csr, f, 1e-10)


def test_multiple_eigenvalues_stay_orthonormal_across_walk_chunks():
    # Triple eigenvalues (a diagonal matrix, each value three times): the
    # convergence walk forms Ritz vectors 16 at a time, so some triples are
    # split between two chunks; their eigenvectors must still be orthonormal.
    from synth import diagonal_csr
    d = np.repeat(np.linspace(0.0, 1.0, 101), 3)
    csr = diagonal_csr(d)
    a, b = 0.2025, 0.4975  # 29 distinct values (0.21 ... 0.49), 87 eigenvalues, endpoints in gaps
    ref = d[(d >= a) & (d <= b)]
    out = solve(csr, a, b, block_size=3, degree=80, check_every=10, lmin=-0.001, lmax=1.001)
    assert out["status"] == flz.FLZ_OK
    assert out["vals"].shape == ref.shape == (87,)
    assert np.max(np.abs(out["vals"] - ref)) < 1e-10
    check_pairs(csr, out, 1e-10)


def test_interval_covering_the_whole_spectrum():
    # Degenerate window: [alpha, beta] contains every eigenvalue, so the filter
    # is the identity on the spectrum and the Krylov space must exhaust R^n:
    # all 64 eigenvalues of the 8 x 8 Laplacian, with their multiplicities.
    csr = laplacian_2d(8, 8)
    w = lap2d_eigs(8, 8)
    out = solve(csr, -1.0, 9.0, block_size=4, degree=20, check_every=2)
    assert out["status"] == flz.FLZ_OK
    assert out["vals"].shape == (64,)
    assert np.max(np.abs(out["vals"] - w)) < 1e-10 * 8.0
    check_pairs(csr, out, 1e-10)


@pytest.mark.parametrize("n", [1, 2, 5])
def test_tiny_matrices(n):
    # n = 1, 2, 5 with r = 1: the whole-space Krylov basis is reached in n steps.
    from synth import diagonal_csr
    d = np.arange(1.0, n + 1.0)
    csr = diagonal_csr(d)
    out = solve(csr, 0.5, n + 0.5, block_size=1, degree=10, check_every=1)
    assert out["status"] == flz.FLZ_OK
    assert np.max(np.abs(out["vals"] - d)) < 1e-10 * n
    X = out["vecs"]
    assert np.max(np.abs(np.abs(X) - np.eye(n))) < 1e-8


def test_block_wider_than_the_matrix_is_rejected():
    from synth import diagonal_csr
    csr = diagonal_csr(np.arange(1.0, 4.0))
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
    p = flz.flz_params_default()
    p.block_size = 4
    with pytest.raises(flz.FlzError) as e:
        flz.flz_solver_create(h, p)  # r > n is refused when the solver is created
    assert e.value.status == flz.FLZ_ERR_INVALID_ARG
    flz.flz_matrix_destroy(h)


@pytest.mark.parametrize("precision", [flz.FLZ_PREC_FP64, flz.FLZ_PREC_FX64], ids=["fp64", "fx64"])
def test_scaled_down_table2_stand_in_vs_dense(precision):
    # The Table 2 stand-in's generator at radius 9 (n = 3071, 119 entries per
    # row, 366 rows above 256 entries from the non-local blocks): r = 3 as in
    # the paper, CSR with the long-row tier; the negative eigenvalues (the
    # occupied states of the stand-in) against a dense eigensolve.
    from synth import parsec_like_hamiltonian
    csr = parsec_like_hamiltonian(radius=9, heavy=8, light=6, seed=3)
    lens = np.diff(csr.rowptr)
    assert (lens > 256).sum() > 100
    w = np.linalg.eigvalsh(csr.to_dense())
    k = int((w < 0).sum())
    a, b = w[0] - 1.0, 0.5 * (w[k - 1] + w[k])
    out = solve(csr, a, b, block_size=3, degree=80, check_every=10, precision=precision)
    ref = w[(w >= a) & (w <= b)]
    assert out["status"] == flz.FLZ_OK
    assert out["vals"].shape == ref.shape
    norm_a = max(abs(out["stats"]["lmin"]), abs(out["stats"]["lmax"]))
    assert np.max(np.abs(out["vals"] - ref)) < 1e-10 * norm_a
    check_pairs(csr, out, 1e-10)


def test_fd4_hamiltonian_count_matches_inertia_midsize():
    # config 3's generator at 18^3 (n = 5832, beyond the dense sizes): the
    # count in [-6, -0.3] by two LDL^T inertia counts (Sylvester)
    csr = fd4_laplacian_3d(18, gaussian_wells_potential(18, 8, seed=4))
    cnt = dense.count_in_interval(csr.to_scipy(), -6.0, -0.3)
    assert cnt >= 5
    for precision in (flz.FLZ_PREC_FP64, flz.FLZ_PREC_FX64):
        out = solve(csr, -6.0, -0.3, block_size=4, degree=120, check_every=10, precision=precision)
        assert out["status"] == flz.FLZ_OK
        assert out["vals"].shape[0] == cnt
        check_pairs(csr, out, 1e-10)


def test_warm_started_sequence_of_perturbed_potentials():
    # Self-consistent-field-like sequence on config 2's generator at 15^3: the
    # potential moves a little each step; each solve starts from the previous
    # step's eigenvectors. Counts and eigenvalues against dense eigensolves;
    # the warm starts must take fewer block steps than random starts in all.
    g = 15
    rng = np.random.Generator(np.random.PCG64(2025))
    v0 = 0.5 * rng.random(g ** 3)
    dv = rng.random(g ** 3) - 0.5
    prev = None
    steps_cold, steps_warm = 0, 0
    for t in range(4):
        csr = laplacian_3d_7pt(g, g, g, v0 + 0.02 * t * dv)
        w = np.linalg.eigvalsh(csr.to_dense())
        win = np.arange(35, 46)
        k = int(win[np.argmax(w[win + 1] - w[win])])
        beta = 0.5 * (w[k] + w[k + 1])
        want = w[w <= beta]
        h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
        try:
            outs = {}
            for mode in ("cold", "warm"):
                p = flz.flz_params_default()
                p.block_size = 4
                p.degree = 60
                p.check_every = 5
                p.precision = flz.FLZ_PREC_FX64
                s = flz.flz_solver_create(h, p)
                try:
                    flz.flz_solver_set_interval(s, 0.0, beta)
                    if mode == "warm" and prev is not None:
                        flz.flz_solver_set_start_vectors(s, prev)
                    assert flz.flz_solve(s) == flz.FLZ_OK
                    outs[mode] = (flz.flz_get_eigenvalues(s), flz.flz_get_stats(s)["iters"],
                                  flz.get_eigenvectors_host(s, csr.n))
                finally:
                    flz.flz_solver_destroy(s)
        finally:
            flz.flz_matrix_destroy(h)
        for mode in ("cold", "warm"):
            vals = outs[mode][0]
            assert vals.shape == want.shape
            assert np.max(np.abs(vals - want)) < 1e-10 * 12.5
        if t > 0:
            steps_cold += outs["cold"][1]
            steps_warm += outs["warm"][1]
        prev = outs["warm"][2]
    assert steps_warm < steps_cold, (steps_warm, steps_cold)


def test_subspace_started_sequence_of_perturbed_potentials():
    # The same kind of sequence at 20^3 with params.start_mode SUBSPACE: each
    # solve after the first is filtered subspace iteration on the previous
    # eigenvectors. Counts and eigenvalues against dense eigensolves,
    # residuals recomputed here, orthonormal eigenvectors; no block Lanczos
    # steps, and fewer products of A with a vector than the random start.
    g = 20
    rng = np.random.Generator(np.random.PCG64(2025))
    v0 = 0.5 * rng.random(g ** 3)
    dv = rng.random(g ** 3) - 0.5
    prev = None
    for t in range(4):
        csr = laplacian_3d_7pt(g, g, g, v0 + 0.02 * t * dv)
        w = np.linalg.eigvalsh(csr.to_dense())
        win = np.arange(55, 70)
        k = int(win[np.argmax(w[win + 1] - w[win])])
        beta = 0.5 * (w[k] + w[k + 1])
        want = w[w <= beta]
        h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
        try:
            outs = {}
            for mode in ("cold", "subspace"):
                if mode == "subspace" and prev is None:
                    continue
                p = flz.flz_params_default()
                p.block_size = 4
                p.degree = 60
                p.check_every = 5
                p.precision = flz.FLZ_PREC_FX64
                p.start_mode = flz.FLZ_START_SUBSPACE
                s = flz.flz_solver_create(h, p)
                try:
                    flz.flz_solver_set_interval(s, 0.0, beta)
                    if mode == "subspace":
                        flz.flz_solver_set_start_vectors(s, prev)
                    assert flz.flz_solve(s) == flz.FLZ_OK
                    outs[mode] = (flz.flz_get_eigenvalues(s), flz.flz_get_stats(s), flz.get_eigenvectors_host(s, csr.n))
                finally:
                    flz.flz_solver_destroy(s)
        finally:
            flz.flz_matrix_destroy(h)
        for mode, (vals, st, X) in outs.items():
            assert vals.shape == want.shape, (mode, vals.shape, want.shape)
            assert np.max(np.abs(vals - want)) < 1e-10 * 12.5
            R = csr.to_scipy() @ X - X * vals
            assert np.max(np.linalg.norm(R, axis=0)) / max(abs(st["lmin"]), abs(st["lmax"])) <= 1e-10
            assert np.max(np.abs(X.T @ X - np.eye(X.shape[1]))) < 1e-10
        if t > 0:
            cold, sub = outs["cold"][1], outs["subspace"][1]
            assert sub["start_used"] == 2 and sub["iters"] == 0 and sub["refine_sweeps"] >= 1, \
                (t, sub["start_used"], sub["refine_sweeps"], sub["sweep_matvecs"], cold["matvecs"])
            assert sub["sweep_matvecs"] < cold["matvecs"], (sub["sweep_matvecs"], cold["matvecs"])
        prev = outs["subspace" if t > 0 else "cold"][2]


def test_subspace_start_falls_back_to_lanczos_when_the_block_is_too_small():
    # five start vectors for a window of about 40 eigenvalues: the subspace
    # block (32 columns) cannot hold the window and its guard pairs, so the
    # solve continues as filtered Lanczos from those vectors and stays correct
    g = 16
    rng = np.random.Generator(np.random.PCG64(8))
    csr = laplacian_3d_7pt(g, g, g, 0.5 * rng.random(g ** 3))
    w = np.linalg.eigvalsh(csr.to_dense())
    beta = 0.5 * (w[39] + w[40])
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
    try:
        p = flz.flz_params_default()
        p.block_size = 4
        p.degree = 60
        p.check_every = 5
        p.precision = flz.FLZ_PREC_FX64
        p.start_mode = flz.FLZ_START_SUBSPACE
        s = flz.flz_solver_create(h, p)
        try:
            flz.flz_solver_set_interval(s, 0.0, beta)
            _, V = np.linalg.eigh(csr.to_dense())
            flz.flz_solver_set_start_vectors(s, np.asfortranarray(V[:, :5]))
            assert flz.flz_solve(s) == flz.FLZ_OK
            st = flz.flz_get_stats(s)
            assert st["start_used"] == 1 and st["iters"] > 0
            vals = flz.flz_get_eigenvalues(s)
            assert vals.shape == (40,) and np.max(np.abs(vals - w[:40])) < 1e-10 * 12.5
        finally:
            flz.flz_solver_destroy(s)
    finally:
        flz.flz_matrix_destroy(h)


def test_start_vectors_are_validated_and_cleared():
    A = laplacian_3d_7pt(8, 8, 8)
    h = flz.flz_matrix_create_csr(A.n, A.nnz, A.rowptr, A.col, A.val)
    try:
        s = flz.flz_solver_create(h, None)
        try:
            # null vectors with cols > 0, and a leading dimension below n
            assert flz.lib().flz_solver_set_start_vectors(s, None, A.n, 3, flz.FLZ_HOST) == flz.FLZ_ERR_INVALID_ARG
            X = np.asfortranarray(np.random.default_rng(0).standard_normal((A.n, 5)))
            assert flz.lib().flz_solver_set_start_vectors(s, X.ctypes.data, A.n - 1, 5,
                                                          flz.FLZ_HOST) == flz.FLZ_ERR_INVALID_ARG
            flz.flz_solver_set_start_vectors(s, X)
            flz.flz_solver_set_interval(s, 0.0, 0.6)
            assert flz.flz_solve(s) == flz.FLZ_OK
            flz.flz_solver_set_start_vectors(s, None)
            assert flz.flz_solve(s) == flz.FLZ_OK
        finally:
            flz.flz_solver_destroy(s)
    finally:
        flz.flz_matrix_destroy(h)
