"""The allocation-free filter entry point against the regular one.

flz_filter_apply_noalloc serves callers that cannot allocate device memory
(their memory belongs to another allocator, or cudaMalloc's device-wide
synchronization is not acceptable to them); it takes the CSR arrays and the
blocks as device pointers and uses a fixed static scratch array. Its output
must match flz_filter_apply (which allocates its scratch in the matrix handle)
within the FP64 filter tolerance of tests/test_gpu_filter.py, on two
consecutive calls (the second reuses the shared scratch left by the first).
This file is collected last so that a failure here does not hide the others.
"""

import numpy as np
import pytest

import __graft_entry__
import paper_2409_15053_gb300 as flz
from oracle import chebyshev
from synth import laplacian_3d_7pt, random_normal_block

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


def test_noalloc_filter_matches_regular_entry_point_twice():
    __graft_entry__.build()
    assert torch.cuda.is_available()
    csr = laplacian_3d_7pt(40, 50, 60, 0.5 * np.linspace(0.0, 1.0, 120000))  # n*r = 480,000 at r = 4
    c, e = 6.25, 6.25
    rp = torch.from_numpy(csr.rowptr).cuda()
    cl = torch.from_numpy(csr.col).cuda()
    vl = torch.from_numpy(csr.val).cuda()
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
    try:
        for call, (m, lo, hi, seed) in enumerate([(45, -1.0, -0.93, 3), (23, -0.4, 0.1, 4)]):
            coeffs = chebyshev.filter_coefficients(lo, hi, m)
            V = torch.from_numpy(random_normal_block(csr.n, 4, seed)).cuda()
            W_regular = torch.full_like(V, float("nan"))
            W_noalloc = torch.full_like(V, float("nan"))
            flz.flz_filter_apply(h, c, e, coeffs, m, 4, V, W_regular)
            flz.flz_filter_apply_noalloc(csr.n, csr.nnz, rp, cl, vl, c, e, coeffs, m, 4, V, W_noalloc)
            torch.cuda.synchronize()
            a = W_regular.cpu().numpy()
            b = W_noalloc.cpu().numpy()
            rowsum = 12.5 + c
            tol = 32.0 * (m + 1) ** 2 * U64 * (1.0 + rowsum / e) * float(V.abs().max())
            assert np.all(np.isfinite(b)), f"call {call}"
            assert np.max(np.abs(a - b)) <= tol, f"call {call}"
    finally:
        flz.flz_matrix_destroy(h)


def test_noalloc_filter_rejects_oversized_blocks():
    __graft_entry__.build()
    n = 300000  # n * r = 1.2e6 > 1,048,576 at r = 4
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    ip = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(flz.FlzError) as e:
        flz.flz_filter_apply_noalloc(n, 0, ip, None, None, 0.0, 1.0, np.ones(3), 2, 4, dummy.data_ptr(),
                                     dummy.data_ptr() + 8 * 4 * n + 64)
    assert e.value.status == flz.FLZ_ERR_CAPACITY
