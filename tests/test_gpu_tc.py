"""Full reorthogonalization on the tensor cores (Section 3.2.2, classical
Gram-Schmidt twice) against exact arithmetic and the FP64 path.

The tensor-core path rounds the basis to the 2^-62 grid and W (or a
coefficient matrix H) to 62 fractional bits of each column's scale, splits
both into eight base-256 digits and sums the digit products exactly. The
references are the oracle's exact products of the UNROUNDED FP64 inputs
(oracle/reorth.py); the tests bound the difference by that number format's
error model, written out below, and compare with the FP64 CUDA-core path.

The first tests check the shared-memory descriptor layouts of one tcgen05
MMA on small integer tiles; they run first so that a layout mismatch stops
the run before the projection kernels (which rely on the same layouts).
"""

import numpy as np
import pytest

import paper_2409_15053_gb300 as flz
from oracle import reorth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")


def bf16_bits(x):
    """uint16 bfloat16 bit patterns of small integers (exact)."""
    f = np.asarray(x, dtype=np.float32)
    return (f.view(np.uint32) >> 16).astype(np.uint16)


def image(mat, lead_stride, strided_stride, k_major, nbytes):
    """Shared-memory image of a (rows x 16) operand as 8 x 16-byte core matrices.

    k_major: core-matrix rows are operand rows (16 bytes = 8 consecutive K);
    otherwise core-matrix rows are K indices (16 bytes = 8 consecutive rows).
    lead_stride: bytes between core matrices adjacent along K;
    strided_stride: bytes between core matrices adjacent along the rows.
    """
    img = np.zeros(nbytes // 2, dtype=np.uint16)
    bits = bf16_bits(mat)
    rows, K = mat.shape
    for m in range(rows):
        for k in range(K):
            if k_major:
                off = (m // 8) * strided_stride + (k // 8) * lead_stride + (m % 8) * 16 + (k % 8) * 2
            else:
                off = (m // 8) * strided_stride + (k // 8) * lead_stride + (k % 8) * 16 + (m % 8) * 2
            img[off // 2] = bits[m, k]
    return img


def probe(A, B, a_mn_major, a_lbo, a_sbo, b_lbo, b_sbo, a_bytes, b_bytes):
    a_img = image(A, a_lbo, a_sbo, not a_mn_major, a_bytes)
    b_img = image(B, b_lbo, b_sbo, True, b_bytes)
    return flz.flz_tc_mma_probe(a_img, b_img, B.shape[0], a_mn_major, a_lbo, a_sbo, b_lbo, b_sbo)


@pytest.mark.parametrize("np_", [32, 16])
def test_mma_layout_of_the_projection(np_):
    # projection: A K-major (digit x column rows, 16 strips 2048 B apart, row
    # octets 128 B apart), B K-major (W columns x digits, octets 128 B apart,
    # column blocks 4096 B apart)
    rng = np.random.default_rng(np_)
    A = rng.integers(-9, 10, size=(128, 16)).astype(np.float32)
    B = rng.integers(-9, 10, size=(np_, 16)).astype(np.float32)
    D = probe(A, B, 0, 128, 2048, 128, 4096, 32768, (np_ // 8) * 4096)
    want = A @ B.T
    if not np.array_equal(D, want):
        # diagnosis: the same images with the two stride fields exchanged
        a_img = image(A, 128, 2048, True, 32768)
        b_img = image(B, 128, 4096, True, (np_ // 8) * 4096)
        Ds = flz.flz_tc_mma_probe(a_img, b_img, np_, 0, 2048, 128, 4096, 128)
        pytest.fail(f"max diff {np.max(np.abs(D - want))}; exchanged fields match: {np.array_equal(Ds, want)}")


@pytest.mark.parametrize("np_", [32, 16])
def test_mma_layout_of_the_update(np_):
    # update: A MN-major (row octets 128 B apart along M, column halves 2048 B
    # apart along K), B K-major (column halves 128 B apart, j blocks 256 B apart)
    rng = np.random.default_rng(100 + np_)
    A = rng.integers(-9, 10, size=(128, 16)).astype(np.float32)
    B = rng.integers(-9, 10, size=(np_, 16)).astype(np.float32)
    D = probe(A, B, 1, 2048, 128, 128, 256, 4096, (np_ // 8) * 256)
    want = A @ B.T
    if not np.array_equal(D, want):
        a_img = image(A, 2048, 128, False, 4096)
        b_img = image(B, 128, 256, True, (np_ // 8) * 256)
        Ds = flz.flz_tc_mma_probe(a_img, b_img, np_, 1, 128, 2048, 128, 256)
        pytest.fail(f"max diff {np.max(np.abs(D - want))}; exchanged A fields match: {np.array_equal(Ds, want)}")


@pytest.mark.parametrize("np_", [64, 128])
def test_mma_layout_with_wide_n(np_):
    # N = 64 and 128 (blocks of 5..16 columns): more column blocks along N
    rng = np.random.default_rng(200 + np_)
    A = rng.integers(-9, 10, size=(128, 16)).astype(np.float32)
    B = rng.integers(-9, 10, size=(np_, 16)).astype(np.float32)
    D = probe(A, B, 0, 128, 2048, 128, 256, 32768, (np_ // 8) * 256)
    assert np.array_equal(D, A @ B.T)
    D = probe(A, B, 1, 2048, 128, 128, 256, 4096, (np_ // 8) * 256)
    assert np.array_equal(D, A @ B.T)


def test_mma_holds_exact_integer_sums():
    # digits up to the bound the kernels use: products up to 2^14, sums of 16
    A = np.full((128, 16), -128.0, dtype=np.float32)
    B = np.full((32, 16), -128.0, dtype=np.float32)
    A[1::2] = 127.0
    D = probe(A, B, 0, 128, 2048, 128, 4096, 32768, 4 * 4096)
    assert np.array_equal(D, A @ B.T)


# ---------------------------------------------------------------------------
def orthonormal_blocks(n, nb, r, seed):
    """An orthonormal FP64 basis (Householder QR of a normal matrix), as is and as nb row-major n x r blocks."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, nb * r)))
    blocks = np.ascontiguousarray(Q.reshape(n, nb, r).transpose(1, 0, 2))  # nb x n x r
    return Q, blocks


U = 2.0**-53        # FP64 unit roundoff
GRID = 2.0**-62     # spacing of the basis grid
TOP_DROPPED = 2.0**-66  # digit pairs s + t >= 9 an update leaves out, per basis column, times the column scale


def column_scale(X):
    """2^E per column, E the least integer with max |column| < 2^E (1 for a zero column)."""
    m = np.max(np.abs(X), axis=0)
    return np.where(m > 0, np.ldexp(1.0, np.frexp(m)[1]), 1.0)


def projection_error_bound(Q, W):
    """|C_tc - Q^T W| elementwise: the basis rounded to the 2^-62 grid (|dq| <= 2^-63), each W column
    rounded to 62 fractional bits of its scale 2^E (|dw| <= 2^(E-63)), their product, and the FP64
    recombination of the 15 exact digit-diagonal sums (at most 16 roundings of partial sums bounded
    by sum |q| |w|)."""
    n = Q.shape[0]
    dw = column_scale(W) * 2.0**-63
    aQ, aW = np.abs(Q), np.abs(W)
    grid = GRID / 2 * aW.sum(axis=0)[None, :] + aQ.sum(axis=0)[:, None] * dw[None, :] + n * GRID / 2 * dw[None, :]
    return grid + 16 * U * ((aQ + GRID).T @ (aW + dw[None, :]))


def combination_error_bound(Q, H):
    """|X_tc - Q H| elementwise: the basis grid (2^-63 per value), each H column rounded to 62 fractional
    bits of its scale 2^F, the digit pairs below 2^-64 of the scale the kernel leaves out, and per window
    of 256 basis columns three FP64 roundings of partial sums bounded by |Q| |H|."""
    K = Q.shape[1]
    windows = (K + 255) // 256
    dh = column_scale(H) * 2.0**-63
    aQ, aH = np.abs(Q), np.abs(H)
    grid = GRID / 2 * aH.sum(axis=0)[None, :] + aQ.sum(axis=1)[:, None] * dh[None, :] + K * GRID / 2 * dh[None, :]
    dropped = K * TOP_DROPPED * column_scale(H)[None, :]
    return grid + dropped + 3 * windows * U * ((aQ + GRID) @ (aH + dh[None, :]))


@pytest.mark.parametrize("n,nb,r", [(4000, 6, 4), (2777, 13, 3), (1000, 9, 2), (513, 20, 1), (3000, 75, 4),
                                    (3000, 5, 8), (1500, 7, 6), (2000, 3, 16), (700, 2, 13)])
def test_projection_within_the_fixed_point_error_bound(n, nb, r):
    Q, blocks = orthonormal_blocks(n, nb, r, n + nb)
    rng = np.random.default_rng(7)
    W = rng.standard_normal((n, r)) * np.resize(np.array([1.0, 1e-3, 37.0, 2.0**-40]), r)
    Qd = torch.from_numpy(blocks).cuda()
    Wd = torch.from_numpy(W).cuda()
    C = torch.zeros(nb * r, r, dtype=torch.float64, device="cuda")
    C64 = torch.zeros_like(C)
    flz.flz_basis_project(n, nb, r, Qd, Wd, C, flz.FLZ_ORTHO_TENSOR)
    flz.flz_basis_project(n, nb, r, Qd, Wd, C64, flz.FLZ_ORTHO_CUDA_CORES)
    assert np.array_equal(blocks, Qd.cpu().numpy())  # the caller's basis is not modified
    exact = reorth.exact_projection(Q, W)
    err_tc = np.abs(C.cpu().numpy() - exact)
    bound = projection_error_bound(Q, W)
    assert np.all(err_tc <= bound), float(np.max(err_tc / bound))
    # and the bound is tighter than the FP64 inner products' own (n-term rounding)
    assert np.all(bound <= n * U * (np.abs(Q).T @ np.abs(W)) + 64 * U * np.abs(exact) + 2.0**-1000)
    scale = np.linalg.norm(Q, axis=0)[:, None] * np.linalg.norm(W, axis=0)[None, :]
    err_64 = np.max(np.abs(C64.cpu().numpy() - exact) / scale)
    assert np.max(err_tc / scale) <= max(err_64, 2.0**-52)


@pytest.mark.parametrize("n,nb,r,s", [(3000, 6, 4, 4), (2777, 13, 3, 16), (1000, 90, 4, 9), (513, 20, 1, 1),
                                      (700, 2, 13, 5)])
def test_combination_within_the_fixed_point_error_bound(n, nb, r, s):
    # X = Q H, the Ritz vectors' product (Section 2.3), on the update kernel
    Q, blocks = orthonormal_blocks(n, nb, r, 5 * n + nb)
    rng = np.random.default_rng(13)
    K = nb * r
    H = rng.standard_normal((K, s)) * np.resize(np.array([1.0, 3e-4, 20.0, 2.0**-30]), s)
    Qd = torch.from_numpy(blocks).cuda()
    Hd = torch.from_numpy(np.ascontiguousarray(H)).cuda()
    X = torch.full((n, s), 7.0, dtype=torch.float64, device="cuda")  # overwritten, not accumulated into
    X64 = torch.zeros_like(X)
    flz.flz_basis_multiply(n, nb, r, Qd, Hd, s, X, flz.FLZ_ORTHO_TENSOR)
    flz.flz_basis_multiply(n, nb, r, Qd, Hd, s, X64, flz.FLZ_ORTHO_CUDA_CORES)
    exact = reorth.exact_combination(Q, H)
    err_tc = np.abs(X.cpu().numpy() - exact)
    bound = combination_error_bound(Q, H)
    assert np.all(err_tc <= bound), float(np.max(err_tc / bound))
    err_64 = np.abs(X64.cpu().numpy() - exact)
    assert np.all(err_64 <= K * U * (np.abs(Q) @ np.abs(H)) + 2.0**-1000)


@pytest.mark.parametrize("n,nb,r", [(4000, 6, 4), (2777, 13, 3), (3000, 75, 4), (300, 1, 2), (8, 1, 1),
                                    (3000, 20, 8), (2000, 20, 16), (1000, 9, 11)])
def test_orthogonalize_matches_fp64_and_leaves_w_orthogonal(n, nb, r):
    Q, blocks = orthonormal_blocks(n, nb, r, 3 * n + nb)
    rng = np.random.default_rng(11)
    # W with a large component in span(Q): the second pass must clean it up
    W = Q @ rng.standard_normal((nb * r, r)) * 1e3 + rng.standard_normal((n, r))
    W = np.ascontiguousarray(W)
    Qd = torch.from_numpy(blocks).cuda()
    out = {}
    for method in (flz.FLZ_ORTHO_TENSOR, flz.FLZ_ORTHO_CUDA_CORES):
        Wd = torch.from_numpy(W.copy()).cuda()
        C = torch.zeros(nb * r, r, dtype=torch.float64, device="cuda")
        flz.flz_basis_orthogonalize(n, nb, r, Qd, Wd, C, method)
        out[method] = (Wd.cpu().numpy(), C.cpu().numpy())
    Wt, Ct = out[flz.FLZ_ORTHO_TENSOR]
    W6, C6 = out[flz.FLZ_ORTHO_CUDA_CORES]
    nw = np.linalg.norm(Wt, axis=0)
    assert np.max(np.abs(Q.T @ Wt) / nw) < 1e-14
    assert np.max(np.abs(Wt - W6)) < 1e-12 * np.max(np.abs(W))
    assert np.max(np.abs(Ct - C6)) < 1e-12 * np.max(np.abs(C6))


def test_full_size_projection_grid():
    # the benchmark's row count: many CTAs per group set, 256-row ranges
    n, nb, r = 1_000_000, 30, 4
    g = torch.Generator(device="cuda").manual_seed(5)
    Q = torch.randn(n, nb * r, dtype=torch.float64, device="cuda", generator=g)
    Q, _ = torch.linalg.qr(Q)
    blocks = Q.reshape(n, nb, r).permute(1, 0, 2).contiguous()
    W = torch.randn(n, r, dtype=torch.float64, device="cuda", generator=g) + Q[:, :r] * 50.0
    C = torch.zeros(nb * r, r, dtype=torch.float64, device="cuda")
    C64 = torch.zeros_like(C)
    Wt = W.clone()
    flz.flz_basis_orthogonalize(n, nb, r, blocks, Wt, C, flz.FLZ_ORTHO_TENSOR)
    W6 = W.clone()
    flz.flz_basis_orthogonalize(n, nb, r, blocks, W6, C64, flz.FLZ_ORTHO_CUDA_CORES)
    torch.cuda.synchronize()
    proj = (Q.T @ Wt) / torch.linalg.norm(Wt, dim=0)
    assert float(proj.abs().max()) < 1e-14
    assert float((Wt - W6).abs().max()) < 1e-11 * float(W.abs().max())
    assert float((C - C64).abs().max()) < 1e-11 * float(C64.abs().max())


# ---------------------------------------------------------------------------
def test_solver_on_the_tensor_cores_matches_the_fp64_path():
    from synth import laplacian_3d_7pt
    A = laplacian_3d_7pt(24, 24, 24)
    h = flz.flz_matrix_create_csr(A.n, A.nnz, A.rowptr, A.col, A.val)
    try:
        vals = {}
        for ortho in (flz.FLZ_ORTHO_TENSOR, flz.FLZ_ORTHO_CUDA_CORES, flz.FLZ_ORTHO_AUTO):
            p = flz.flz_params_default()
            p.block_size = 4
            p.degree = 60
            p.check_every = 10
            p.ortho = ortho
            s = flz.flz_solver_create(h, p)
            try:
                flz.flz_solver_set_interval(s, 0.0, 0.436)
                assert flz.flz_solve(s) == flz.FLZ_OK
                st = flz.flz_get_stats(s)
                vals[ortho] = (flz.flz_get_eigenvalues(s), flz.flz_get_residuals(s), st["ortho"])
                if ortho == flz.FLZ_ORTHO_TENSOR:
                    # Ritz vectors formed on the tensor cores: orthonormal eigenvectors of A
                    X = flz.get_eigenvectors_host(s, A.n)
                    lam = vals[ortho][0]
                    R = A.to_scipy() @ X - X * lam
                    assert np.max(np.linalg.norm(R, axis=0)) < 1e-10 * 12.0
                    assert np.max(np.abs(X.T @ X - np.eye(X.shape[1]))) < 1e-12
            finally:
                flz.flz_solver_destroy(s)
        t, c, a = vals[flz.FLZ_ORTHO_TENSOR], vals[flz.FLZ_ORTHO_CUDA_CORES], vals[flz.FLZ_ORTHO_AUTO]
        assert t[2] == flz.FLZ_ORTHO_TENSOR and c[2] == flz.FLZ_ORTHO_CUDA_CORES
        assert a[2] == flz.FLZ_ORTHO_TENSOR  # AUTO picks the tensor cores for r <= 4
        assert t[0].shape == c[0].shape and t[0].shape[0] > 20
        assert np.max(np.abs(t[0] - c[0])) < 1e-12
        assert np.max(t[1]) < 1e-10
        # closed form: 6 - 2 sum cos(k pi / 25)
        k = np.arange(1, 25)
        lam = np.sort((6 - 2 * (np.cos(k[:, None, None] * np.pi / 25) + np.cos(k[None, :, None] * np.pi / 25) +
                                np.cos(k[None, None, :] * np.pi / 25))).ravel())
        want = lam[(lam >= 0.0) & (lam <= 0.436)]
        assert t[0].shape == want.shape and np.max(np.abs(t[0] - want)) < 1e-12
    finally:
        flz.flz_matrix_destroy(h)


def test_wide_blocks_and_double_fp32_paths():
    # r = 8 and 16 take the tensor cores under AUTO and match the CUDA cores;
    # the double-FP32 precision keeps its own basis on the FP32 pipes
    from synth import laplacian_2d
    A = laplacian_2d(60, 60)
    h = flz.flz_matrix_create_csr(A.n, A.nnz, A.rowptr, A.col, A.val)
    try:
        for r in (8, 16):
            out = {}
            for ortho in (flz.FLZ_ORTHO_AUTO, flz.FLZ_ORTHO_CUDA_CORES):
                p = flz.flz_params_default()
                p.block_size = r
                p.degree = 40
                p.ortho = ortho
                s = flz.flz_solver_create(h, p)
                try:
                    flz.flz_solver_set_interval(s, 0.0, 0.3)
                    assert flz.flz_solve(s) == flz.FLZ_OK
                    out[ortho] = (flz.flz_get_eigenvalues(s), flz.flz_get_stats(s)["ortho"],
                                  flz.flz_get_residuals(s))
                finally:
                    flz.flz_solver_destroy(s)
            assert out[flz.FLZ_ORTHO_AUTO][1] == flz.FLZ_ORTHO_TENSOR
            assert out[flz.FLZ_ORTHO_CUDA_CORES][1] == flz.FLZ_ORTHO_CUDA_CORES
            a, c = out[flz.FLZ_ORTHO_AUTO][0], out[flz.FLZ_ORTHO_CUDA_CORES][0]
            assert a.shape == c.shape and np.max(np.abs(a - c)) < 1e-12
            assert np.max(out[flz.FLZ_ORTHO_AUTO][2]) < 1e-10
        p = flz.flz_params_default()
        p.block_size = 4
        p.degree = 40
        p.precision = flz.FLZ_PREC_DF64
        s = flz.flz_solver_create(h, p)
        try:
            flz.flz_solver_set_interval(s, 0.0, 0.3)
            assert flz.flz_solve(s) == flz.FLZ_OK
            assert flz.flz_get_stats(s)["ortho"] == flz.FLZ_ORTHO_CUDA_CORES
        finally:
            flz.flz_solver_destroy(s)
        p.ortho = flz.FLZ_ORTHO_TENSOR
        with pytest.raises(flz.FlzError) as e:
            flz.flz_solver_create(h, p)
        assert e.value.status == flz.FLZ_ERR_INVALID_ARG
    finally:
        flz.flz_matrix_destroy(h)
