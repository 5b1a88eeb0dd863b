"""The mixed-precision form: FP32 / BF16 filter, FP64 everything else, then
refinement (params.refine = 1) to residual <= 1e-8.

A reduced-precision filtered Lanczos solve stalls at its rounding floor
(about 1e-7 relative residual in FP32, 1e-4 in BF16). The refinement runs
filtered subspace iteration with the fixed-point filter and Rayleigh-Ritz on
A in FP64 on the wanted, guard and extra Ritz pairs. Bar, as for FP64 solves:
the count in [alpha, beta] exact, eigenvalues within 1e-10 ||A|| of a dense
eigensolve (or the oracle's reference), residuals <= 1e-8 recomputed here on
the CPU, orthonormal eigenvectors.
"""

import json
import os

import numpy as np
import pytest

import __graft_entry__
import paper_2409_15053_gb300 as flz
from synth import fd4_laplacian_3d, gaussian_wells_potential, laplacian_3d_7pt

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-8


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


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


def check(csr, out, want, tol=TOL):
    assert out["status"] == flz.FLZ_OK
    st = out["stats"]
    assert st["refine_sweeps"] >= 1
    norm_a = max(abs(st["lmin"]), abs(st["lmax"]))
    assert out["vals"].shape == want.shape, (out["vals"].shape, want.shape)
    assert np.max(np.abs(out["vals"] - want)) < 1e-10 * norm_a
    X = out["vecs"]
    R = csr.to_scipy() @ X - X * out["vals"]
    res = np.linalg.norm(R, axis=0) / norm_a
    assert np.all(res <= tol), res.max()
    assert np.max(np.abs(X.T @ X - np.eye(X.shape[1]))) < 1e-10


def window(w, lo, count):
    a = 0.5 * (w[lo - 1] + w[lo]) if lo > 0 else w[0] - 1.0
    b = 0.5 * (w[lo + count - 1] + w[lo + count])
    return a, b


@pytest.mark.parametrize("precision", [flz.FLZ_PREC_FP32, flz.FLZ_PREC_BF16], ids=["fp32", "bf16"])
def test_lowest_pairs_of_a_3d_hamiltonian(precision):
    rng = np.random.Generator(np.random.PCG64(15))
    csr = laplacian_3d_7pt(14, 14, 14, 0.5 * rng.random(14 ** 3))
    w = np.linalg.eigvalsh(csr.to_dense())
    a, b = window(w, 0, 30)
    out = solve(csr, a, b, block_size=4, degree=60, check_every=10, precision=precision, refine=1, tol=TOL)
    check(csr, out, w[(w >= a) & (w <= b)])


def test_fd4_hamiltonian_bound_states():
    csr = fd4_laplacian_3d(11, gaussian_wells_potential(11, 6, seed=9))
    w = np.linalg.eigvalsh(csr.to_dense())
    a, b = w[0] - 1.0, 0.5 * (w[24] + w[25])
    out = solve(csr, a, b, block_size=4, degree=80, check_every=10, precision=flz.FLZ_PREC_FP32, refine=1, tol=TOL)
    check(csr, out, w[(w >= a) & (w <= b)])


def test_top_of_a_3d_hamiltonian():
    # a window at the top of the spectrum: the damping polynomial is mirrored
    rng = np.random.Generator(np.random.PCG64(31))
    csr = laplacian_3d_7pt(13, 13, 13, 0.5 * rng.random(13 ** 3))
    w = np.linalg.eigvalsh(csr.to_dense())
    a, b = 0.5 * (w[-26] + w[-25]), w[-1] + 1.0
    out = solve(csr, a, b, block_size=4, degree=60, check_every=10, precision=flz.FLZ_PREC_FP32, refine=1, tol=TOL)
    check(csr, out, w[(w >= a) & (w <= b)])


def test_interior_window_uses_the_solve_filter():
    rng = np.random.Generator(np.random.PCG64(21))
    csr = laplacian_3d_7pt(12, 12, 12, 0.5 * rng.random(12 ** 3))
    w = np.linalg.eigvalsh(csr.to_dense())
    a, b = window(w, 200, 20)
    out = solve(csr, a, b, block_size=4, degree=120, check_every=10, precision=flz.FLZ_PREC_FP32, refine=1, tol=TOL)
    check(csr, out, w[(w >= a) & (w <= b)])
    assert out["stats"]["refine_degree"] in (60, 120)  # the solve's filter (half its degree in the first sweep)


def test_refine_is_rejected_out_of_range():
    csr = laplacian_3d_7pt(6, 6, 6)
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
    try:
        p = flz.flz_params_default()
        p.refine = 2
        with pytest.raises(flz.FlzError) as e:
            flz.flz_solver_create(h, p)
        assert e.value.status == flz.FLZ_ERR_INVALID_ARG
    finally:
        flz.flz_matrix_destroy(h)


def test_full_size_config2_fp32_filter_refined_to_1e8():
    # n = 1e6: the benchmark's workload with the FP32 filter, against the oracle's eigenvalues
    from synth.workloads import CONFIG2
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "config2_reference.json")))
    rng = np.random.Generator(np.random.PCG64(CONFIG2["seed"]))
    g = CONFIG2["grid"]
    csr = laplacian_3d_7pt(g, g, g, CONFIG2["potential_scale"] * rng.random(g ** 3))
    out = solve(csr, CONFIG2["alpha"], CONFIG2["beta"], block_size=4, degree=100, check_every=10,
                precision=flz.FLZ_PREC_FP32, refine=1, tol=TOL)
    check(csr, out, np.array(ref["eigenvalues"]))


def test_full_size_config3_bound_states_fp32_refined_to_1e8():
    # the 120^3 4th-order FD Hamiltonian with 64 wells, window [-6, -0.2]: the
    # refined FP32 solve against the FP64-class (fixed-point filter) solve of the
    # same window -- same count and eigenvalues -- and residuals recomputed here
    from synth.workloads import CONFIG3
    N = CONFIG3["grid"]
    csr = fd4_laplacian_3d(N, gaussian_wells_potential(N, CONFIG3["wells"], seed=CONFIG3["seed"]))
    ref = solve(csr, CONFIG3["alpha"], -0.2, block_size=4, degree=200, check_every=10, precision=flz.FLZ_PREC_FX64)
    assert ref["status"] == flz.FLZ_OK and ref["vals"].shape[0] > 40
    out = solve(csr, CONFIG3["alpha"], -0.2, block_size=4, degree=200, check_every=10,
                precision=flz.FLZ_PREC_FP32, refine=1, tol=TOL)
    check(csr, out, ref["vals"])
