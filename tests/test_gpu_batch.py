"""Batches of independent problems (uneven 2D/3D Laplacians with potentials,
each with its own interval) solved in lockstep, against dense eigensolves of
every problem: exact counts, eigenvalues within 1e-10 ||A|| (FP64 filter) and
residuals recomputed on the CPU."""

import numpy as np
import pytest

import __graft_entry__
import paper_2409_15053_gb300 as flz
from synth import laplacian_2d, laplacian_3d_7pt, uneven_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


def gap_interval(w, lo, cnt):
    a = 0.5 * (w[lo - 1] + w[lo]) if lo > 0 else w[0] - 1.0
    b = 0.5 * (w[lo + cnt - 1] + w[lo + cnt])
    return a, b


def run_batch(csrs, intervals, **kw):
    hs = [flz.flz_matrix_create_csr(c.n, c.nnz, c.rowptr, c.col, c.val) for c in csrs]
    p = flz.flz_params_default()
    for k, v in kw.items():
        setattr(p, k, v)
    b = flz.flz_batch_create(hs, [a for a, _ in intervals], [z for _, z in intervals], p)
    st = flz.flz_batch_solve(b)
    out = []
    for i, c in enumerate(csrs):
        assert flz.flz_batch_get_count(b, i) == flz.flz_batch_get_eigenvalues(b, i).shape[0]
        out.append({"vals": flz.flz_batch_get_eigenvalues(b, i), "res": flz.flz_batch_get_residuals(b, i),
                    "vecs": flz.batch_eigenvectors_host(b, i, c.n), "stats": flz.flz_batch_get_stats(b, i)})
    flz.flz_batch_destroy(b)
    for h in hs:
        flz.flz_matrix_destroy(h)
    return st, out


def check(csrs, intervals, out, tol):
    for c, (a, z), o in zip(csrs, intervals, out):
        w = np.linalg.eigvalsh(c.to_dense())
        ref = w[(w >= a) & (w <= z)]
        assert o["vals"].shape == ref.shape, (o["vals"].shape, ref.shape, o["stats"])
        norm_a = max(abs(o["stats"]["lmin"]), abs(o["stats"]["lmax"]))
        assert np.max(np.abs(o["vals"] - ref)) < 1e-10 * norm_a
        X = o["vecs"]
        R = c.to_scipy() @ X - X * o["vals"]
        assert np.max(np.linalg.norm(R, axis=0)) / norm_a <= tol
        assert np.max(np.abs(X.T @ X - np.eye(X.shape[1]))) < 1e-10


def small_batch(seed, count):
    rng = np.random.Generator(np.random.PCG64(seed))
    csrs, intervals = [], []
    for i in range(count):
        if i % 2 == 0:
            s = int(rng.integers(9, 14))
            c = laplacian_3d_7pt(s, s, s, rng.random(s ** 3))
        else:
            s = int(rng.integers(25, 45))
            c = laplacian_2d(s, s, rng.random(s * s))
        w = np.linalg.eigvalsh(c.to_dense())
        cnt = int(rng.integers(10, 25))
        lo = int(rng.integers(0, 40))
        csrs.append(c)
        intervals.append(gap_interval(w, lo, cnt))
    return csrs, intervals


@pytest.mark.parametrize("ortho", [flz.FLZ_ORTHO_TENSOR, flz.FLZ_ORTHO_CUDA_CORES], ids=["tensor", "cuda-cores"])
@pytest.mark.parametrize("r", [4, 8])
def test_batch_fp64_matches_dense(r, ortho):
    # reorthogonalization per problem on the tensor cores (exact digit
    # products), or segmented over the concatenation on the CUDA cores
    csrs, intervals = small_batch(3, 6)
    st, out = run_batch(csrs, intervals, block_size=r, degree=40, check_every=5, ortho=ortho)
    assert st == flz.FLZ_OK
    assert all(o["stats"]["ortho"] == ortho for o in out)
    check(csrs, intervals, out, 1e-10)


def test_batch_tensor_core_basis_grows_past_its_first_capacity():
    # r = 16 and degree 8: the digit copies start at 256 columns and must
    # grow (keeping their digits) before these problems converge
    csrs, intervals = small_batch(13, 3)
    st, out = run_batch(csrs, intervals, block_size=16, degree=8, check_every=5, ortho=flz.FLZ_ORTHO_TENSOR)
    assert st == flz.FLZ_OK
    assert max(o["stats"]["basis_vectors"] for o in out) > 256
    check(csrs, intervals, out, 1e-10)


@pytest.mark.parametrize("r,m,rows", [(4, 40, 256), (4, 41, 128), (4, 42, 256), (8, 40, 128), (16, 40, 256),
                                      (16, 41, 128)])
def test_batch_fixed_point_filter_matches_dense(r, m, rows):
    # the 64-bit fixed-point filter over the concatenation: per-problem maps,
    # coefficient tables and sum scalings in one kernel per degree; degrees
    # 40, 41, 42 end with 3, 1 and 2 running-sum terms added at the last
    # step; both tile shapes (128 and 256 rows per CTA)
    csrs, intervals = small_batch(3, 6)
    st, out = run_batch(csrs, intervals, block_size=r, degree=m, check_every=5, precision=flz.FLZ_PREC_FX64,
                        tile_rows=rows)
    assert st == flz.FLZ_OK
    assert all(o["stats"]["filter_precision"] == flz.FLZ_PREC_FX64 for o in out)
    assert all(o["stats"]["tile_rows"] == rows for o in out)
    check(csrs, intervals, out, 1e-10)


@pytest.mark.parametrize("r,m", [(4, 40), (4, 41), (16, 42)])
def test_batch_persistent_degree_loop_matches_dense(r, m):
    # every degree of a filter application in one cooperative launch, the
    # CTAs meeting at a bounded grid barrier between degrees
    csrs, intervals = small_batch(3, 6)
    st, out = run_batch(csrs, intervals, block_size=r, degree=m, check_every=5, precision=flz.FLZ_PREC_FX64,
                        persistent=1)
    assert st == flz.FLZ_OK
    assert all(o["stats"]["filter_precision"] == flz.FLZ_PREC_FX64 for o in out)
    check(csrs, intervals, out, 1e-10)


def test_batch_persistent_loop_with_cuda_core_reorthogonalization_and_auto_degrees():
    csrs, intervals = small_batch(5, 4)
    st, out = run_batch(csrs, intervals, block_size=4, degree=0, check_every=5, precision=flz.FLZ_PREC_FX64,
                        persistent=1, ortho=flz.FLZ_ORTHO_CUDA_CORES)
    assert st == flz.FLZ_OK
    check(csrs, intervals, out, 1e-10)


def test_batch_fixed_point_filter_with_per_problem_degrees():
    # automatic degrees differ between problems: each problem's rows stop at
    # its own last degree (the running sum becomes W there) while the others go on
    csrs, intervals = small_batch(5, 4)
    st, out = run_batch(csrs, intervals, block_size=4, degree=0, check_every=5, precision=flz.FLZ_PREC_FX64)
    assert st == flz.FLZ_OK
    assert len({o["stats"]["degree"] for o in out}) > 1
    assert all(o["stats"]["filter_precision"] == flz.FLZ_PREC_FX64 for o in out)
    check(csrs, intervals, out, 1e-10)


def test_batch_fixed_point_request_falls_back_to_fp64_for_irregular_rows():
    # power-law graphs: the SELL-32 padding exceeds 30 %, the fixed-point
    # layout is not built and the batch filters in FP64
    from synth import powerlaw_graph_laplacian
    csrs, intervals = [], []
    for seed in (7, 8):
        c = powerlaw_graph_laplacian(1500, seed=seed)
        w = np.linalg.eigvalsh(c.to_dense())
        csrs.append(c)
        intervals.append(gap_interval(w, 30, 12))
    st, out = run_batch(csrs, intervals, block_size=4, degree=60, check_every=5, precision=flz.FLZ_PREC_FX64)
    assert st == flz.FLZ_OK
    assert all(o["stats"]["filter_precision"] == flz.FLZ_PREC_FP64 for o in out)
    check(csrs, intervals, out, 1e-10)


def low_end_batch(seed, count):
    # windows [w_0 - 1, gap midpoint] at the bottom of each spectrum, as in the
    # batch benchmark's workload
    rng = np.random.Generator(np.random.PCG64(seed))
    csrs, intervals = [], []
    for i in range(count):
        s = int(rng.integers(11, 15)) if i % 2 == 0 else int(rng.integers(30, 45))
        c = laplacian_3d_7pt(s, s, s, rng.random(s ** 3)) if i % 2 == 0 else laplacian_2d(s, s, rng.random(s * s))
        w = np.linalg.eigvalsh(c.to_dense())
        csrs.append(c)
        intervals.append(gap_interval(w, 0, int(rng.integers(10, 25))))
    return csrs, intervals


@pytest.mark.parametrize("precision", [flz.FLZ_PREC_FP32, flz.FLZ_PREC_BF16], ids=["fp32", "bf16"])
def test_batch_reduced_precision_filter_refined_to_1e8(precision):
    # the lockstep phase with an FP32 / BF16 filter stops at its floor, then
    # every problem's pairs are refined to 1e-8 by filtered subspace iteration
    # with the fixed-point filter and Rayleigh-Ritz on its own matrix
    csrs, intervals = low_end_batch(3, 6)
    st, out = run_batch(csrs, intervals, block_size=4, degree=40, check_every=5, precision=precision, refine=1,
                        tol=1e-8)
    assert st == flz.FLZ_OK
    assert all(o["stats"]["refine_sweeps"] >= 1 for o in out)
    check(csrs, intervals, out, 1e-8)


def test_batch_fp32_filter_refined_on_interior_windows():
    # interior windows: the refinement sweeps with each problem's own (flat) filter
    csrs, intervals = small_batch(3, 6)
    st, out = run_batch(csrs, intervals, block_size=4, degree=80, check_every=5, precision=flz.FLZ_PREC_FP32,
                        refine=1, tol=1e-8)
    assert st == flz.FLZ_OK
    assert all(o["stats"]["refine_sweeps"] >= 1 for o in out)
    check(csrs, intervals, out, 1e-8)


def test_batch_double_fp32_filter_matches_dense():
    # the double-FP32 filter (FP32 pipes, FP64-class accuracy) with the batch's FP64 basis
    csrs, intervals = small_batch(11, 5)
    st, out = run_batch(csrs, intervals, block_size=4, degree=50, check_every=5, precision=flz.FLZ_PREC_DF64)
    assert st == flz.FLZ_OK
    check(csrs, intervals, out, 1e-10)


@pytest.mark.parametrize("precision", [flz.FLZ_PREC_FP64, flz.FLZ_PREC_FX64], ids=["fp64", "fx64"])
def test_batch_autotuned_block_width_and_auto_degree(precision):
    # the autotuner picks r (and, for the fixed-point filter, 128 or 256 rows per CTA)
    csrs, intervals = small_batch(5, 4)
    st, out = run_batch(csrs, intervals, block_size=0, degree=0, check_every=5, precision=precision)
    assert st == flz.FLZ_OK
    assert all(o["stats"]["block_size"] in (4, 8, 16) for o in out)
    want_rows = (128, 256) if precision == flz.FLZ_PREC_FX64 else (0,)
    assert all(o["stats"]["tile_rows"] in want_rows for o in out)
    check(csrs, intervals, out, 1e-10)


def test_batch_rejects_a_tile_shape_it_has_no_kernel_for():
    c = laplacian_2d(10, 10)
    h = flz.flz_matrix_create_csr(c.n, c.nnz, c.rowptr, c.col, c.val)
    p = flz.flz_params_default()
    p.tile_rows = 192
    with pytest.raises(flz.FlzError) as e:
        flz.flz_batch_create([h], [0.0], [1.0], p)
    assert e.value.status == flz.FLZ_ERR_INVALID_ARG
    flz.flz_matrix_destroy(h)


def test_batch_of_one_matches_single_solver():
    csrs, intervals = small_batch(7, 1)
    st, out = run_batch(csrs, intervals, block_size=4, degree=50, check_every=5)
    assert st == flz.FLZ_OK
    check(csrs, intervals, out, 1e-10)


def test_batch_rejects_bad_arguments():
    c = laplacian_2d(10, 10)
    h = flz.flz_matrix_create_csr(c.n, c.nnz, c.rowptr, c.col, c.val)
    p = flz.flz_params_default()
    p.block_size = 3
    with pytest.raises(flz.FlzError) as e:
        flz.flz_batch_create([h], [0.0], [1.0], p)
    assert e.value.status == flz.FLZ_ERR_INVALID_ARG
    p.block_size = 4
    with pytest.raises(flz.FlzError) as e:
        flz.flz_batch_create([h], [1.0], [0.5], p)
    assert e.value.status == flz.FLZ_ERR_INVALID_ARG
    flz.flz_matrix_destroy(h)


@pytest.mark.parametrize("precision,tol,refine,extra", [
    (flz.FLZ_PREC_FP32, 1e-6, 0, {}), (flz.FLZ_PREC_FP64, 1e-10, 0, {}), (flz.FLZ_PREC_FX64, 1e-10, 0, {}),
    (flz.FLZ_PREC_FP32, 1e-8, 1, {}), (flz.FLZ_PREC_FX64, 1e-10, 0, {"persistent": 1}),
    (flz.FLZ_PREC_FX64, 1e-10, 0, {"tile_rows": 128})],
    ids=["fp32", "fp64", "fx64", "fp32-refined", "fx64-persistent", "fx64-128-rows"])
def test_full_size_batch64_matches_oracle_reference(precision, tol, refine, extra):
    # 64 problems, n log-uniform in [1e4, 2e5] (sum ~4.7e6), autotuned r,
    # degree 60: the batched launch shape the benchmark times, against the
    # eigenvalues the CPU oracle computed for every problem (tests/golden).
    # Counts exact; every eigenvalue within tol ||A|| of the oracle's (each
    # Rayleigh quotient with residual <= tol lies within tol ||A|| of an
    # eigenvalue, and the counts pin which); residuals recomputed here.
    import json
    import os
    from synth.workloads import BATCH64
    from synth import csr_checksum
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "batch64_reference.json")))["problems"]
    items = uneven_batch(BATCH64["count"], seed=BATCH64["seed"], n_lo=BATCH64["n_lo"], n_hi=BATCH64["n_hi"])
    csrs = [c for c, _, _ in items]
    assert [csr_checksum(c) for c in csrs] == [p["matrix_checksum"] for p in ref]
    intervals = [(p["alpha"], p["beta"]) for p in ref]
    st, out = run_batch(csrs, intervals, block_size=0, degree=60, check_every=5, precision=precision, tol=tol,
                        refine=refine, **extra)
    assert st == flz.FLZ_OK
    for c, p, o in zip(csrs, ref, out):
        want = np.array(p["eigenvalues"])
        assert o["vals"].shape == want.shape, (p["index"], o["vals"].shape, want.shape)
        norm_a = max(abs(o["stats"]["lmin"]), abs(o["stats"]["lmax"]))
        assert np.max(np.abs(o["vals"] - want)) <= tol * norm_a
        X = o["vecs"]
        R = c.to_scipy() @ X - X * o["vals"]
        assert np.max(np.linalg.norm(R, axis=0)) / norm_a <= tol
        assert np.max(np.abs(X.T @ X - np.eye(X.shape[1]))) < 1e-10
