"""Failure detection without a fault: every device-side wait of the library is
bounded, and an expired wait ends the kernel with a status the host turns
into FLZ_ERR_TIMEOUT while the device stays usable.

The tests shorten the wait limit to zero (flz_set_wait_limit), so that the
tensor-core reorthogonalization's and the staged fixed-point filter's barrier
waits expire before their bulk copies land: no kernel is broken, nothing is
left waiting on a flag that never comes; the kernels drain what they have in
flight (with their own fixed bound), free their tensor memory and return. The
limit is restored and the same calls, then a whole solve, must succeed in the
same process with correct results.
"""

import numpy as np
import pytest

import __graft_entry__
import paper_2409_15053_gb300 as flz
from oracle import chebyshev
from synth import laplacian_3d_7pt, random_normal_block

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


class ZeroWaitLimit:
    def __enter__(self):
        self.prev = flz.flz_set_wait_limit(0)
        return self

    def __exit__(self, *exc):
        flz.flz_set_wait_limit(self.prev)
        return False


def basis(n, nb, r, seed):
    g = torch.Generator(device="cuda").manual_seed(seed)
    Q, _ = torch.linalg.qr(torch.randn(n, nb * r, dtype=torch.float64, device="cuda", generator=g))
    return Q, Q.reshape(n, nb, r).permute(1, 0, 2).contiguous()


def test_tensor_core_projection_reports_an_expired_wait_and_recovers():
    n, nb, r = 300_000, 10, 4
    Q, blocks = basis(n, nb, r, 3)
    W = torch.randn(n, r, dtype=torch.float64, device="cuda")
    C = torch.zeros(nb * r, r, dtype=torch.float64, device="cuda")
    with ZeroWaitLimit():
        with pytest.raises(flz.FlzError) as e:
            flz.flz_basis_project(n, nb, r, blocks, W, C, flz.FLZ_ORTHO_TENSOR)
        assert e.value.status == flz.FLZ_ERR_TIMEOUT
        with pytest.raises(flz.FlzError) as e:
            flz.flz_basis_orthogonalize(n, nb, r, blocks, W.clone(), C, flz.FLZ_ORTHO_TENSOR)
        assert e.value.status == flz.FLZ_ERR_TIMEOUT
    assert flz.flz_set_wait_limit(2_000_000_000) == 2_000_000_000  # restored
    C64 = torch.zeros_like(C)
    flz.flz_basis_project(n, nb, r, blocks, W, C, flz.FLZ_ORTHO_TENSOR)
    flz.flz_basis_project(n, nb, r, blocks, W, C64, flz.FLZ_ORTHO_CUDA_CORES)
    torch.cuda.synchronize()
    assert float((C - C64).abs().max()) < 1e-12 * float(C64.abs().max())


def test_fixed_point_filter_reports_an_expired_stage_wait_and_recovers():
    rng = np.random.Generator(np.random.PCG64(7))
    csr = laplacian_3d_7pt(60, 60, 60, 0.5 * rng.random(60 ** 3))
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
    try:
        coeffs = chebyshev.filter_coefficients(-1.0, -0.9, 30)
        V = random_normal_block(csr.n, 4, 5)
        Vd = torch.from_numpy(V).cuda()
        Wd = torch.zeros_like(Vd)
        with ZeroWaitLimit():
            with pytest.raises(flz.FlzError) as e:
                flz.flz_filter_apply(h, 6.25, 6.25, coeffs, 30, 4, Vd, Wd, flz.FLZ_PREC_FX64)
            assert e.value.status == flz.FLZ_ERR_TIMEOUT
        flz.flz_filter_apply(h, 6.25, 6.25, coeffs, 30, 4, Vd, Wd, flz.FLZ_PREC_FX64)
        torch.cuda.synchronize()
        ref = chebyshev.clenshaw_apply(csr.to_scipy(), 6.25, 6.25, coeffs, V)
        assert np.max(np.abs(Wd.cpu().numpy() - ref)) <= 1e-12 * np.max(np.abs(V))
    finally:
        flz.flz_matrix_destroy(h)


def test_solve_times_out_then_succeeds_in_the_same_process():
    A = laplacian_3d_7pt(24, 24, 24)
    h = flz.flz_matrix_create_csr(A.n, A.nnz, A.rowptr, A.col, A.val)
    try:
        p = flz.flz_params_default()
        p.block_size = 4
        p.degree = 60
        p.check_every = 10
        p.precision = flz.FLZ_PREC_FX64
        s = flz.flz_solver_create(h, p)
        try:
            flz.flz_solver_set_interval(s, 0.0, 0.436)
            with ZeroWaitLimit():
                with pytest.raises(flz.FlzError) as e:
                    flz.flz_solve(s)
                assert e.value.status == flz.FLZ_ERR_TIMEOUT
            assert flz.flz_solve(s) == flz.FLZ_OK
            k = np.arange(1, 25)
            lam = np.sort((6 - 2 * (np.cos(k[:, None, None] * np.pi / 25) + np.cos(k[None, :, None] * np.pi / 25) +
                                    np.cos(k[None, None, :] * np.pi / 25))).ravel())
            want = lam[(lam >= 0.0) & (lam <= 0.436)]
            got = flz.flz_get_eigenvalues(s)
            assert got.shape == want.shape and np.max(np.abs(got - want)) < 1e-12
        finally:
            flz.flz_solver_destroy(s)
    finally:
        flz.flz_matrix_destroy(h)


def test_persistent_batch_grid_barrier_times_out_then_succeeds():
    # the persistent batch filter's grid barrier with a zero wait limit: the
    # CTAs that arrive before the last one give up at once, the solve ends
    # with FLZ_ERR_TIMEOUT, and the same batch then solves normally
    A = [laplacian_3d_7pt(14, 14, 14), laplacian_3d_7pt(12, 13, 15)]
    hs = [flz.flz_matrix_create_csr(c.n, c.nnz, c.rowptr, c.col, c.val) for c in A]
    try:
        p = flz.flz_params_default()
        p.block_size = 4
        p.degree = 40
        p.check_every = 5
        p.precision = flz.FLZ_PREC_FX64
        p.persistent = 1
        p.ortho = flz.FLZ_ORTHO_CUDA_CORES
        b = flz.flz_batch_create(hs, [0.0, 0.0], [0.5, 0.5], p)
        try:
            with ZeroWaitLimit():
                with pytest.raises(flz.FlzError) as e:
                    flz.flz_batch_solve(b)
                assert e.value.status == flz.FLZ_ERR_TIMEOUT
            assert flz.flz_batch_solve(b) == flz.FLZ_OK
            for i, c in enumerate(A):
                w = np.linalg.eigvalsh(c.to_dense())
                want = w[w <= 0.5]
                got = flz.flz_batch_get_eigenvalues(b, i)
                assert got.shape == want.shape and np.max(np.abs(got - want)) < 1e-10 * 12.0
        finally:
            flz.flz_batch_destroy(b)
    finally:
        for h in hs:
            flz.flz_matrix_destroy(h)

