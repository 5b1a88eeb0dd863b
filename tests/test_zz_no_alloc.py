"""The allocation-free filter entry point against the regular one.

flz_filter_apply_noalloc serves callers that cannot allocate device memory
(their memory belongs to another allocator, or cudaMalloc's device-wide
synchronization is not acceptable to them); it takes the CSR arrays and the
blocks as device pointers and uses a fixed static scratch array. Its output
must match flz_filter_apply (which allocates its scratch in the matrix handle)
within 1e-13 of max|V| (the same FP64 recurrence up to rounding), on two
consecutive calls (the second reuses the shared scratch left by the first),
for degrees 0, 1, 2, 45 and block widths 1, 3, 4, 16.
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



@pytest.mark.parametrize("m", [0, 1, 2, 45])
@pytest.mark.parametrize("r", [1, 3, 4, 16])
def test_noalloc_filter_matches_regular_entry_point_twice(m, r):
    # degree 0 (a scaling), degree 1 (the first step alone), widths that leave
    # lanes of a warp idle (r = 3) and the widest block; n * r = 960,000 at r = 16
    __graft_entry__.build()
    assert torch.cuda.is_available()
    csr = laplacian_3d_7pt(30, 40, 50, 0.5 * np.linspace(0.0, 1.0, 60000))
    c, e = 6.25, 6.25
    rp = torch.from_numpy(csr.rowptr).cuda()
    cl = torch.from_numpy(csr.col).cuda()
    vl = torch.from_numpy(csr.val).cuda()
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
    try:
        for call, (lo, hi, seed) in enumerate([(-1.0, -0.93, 3), (-0.4, 0.1, 4)]):
            coeffs = chebyshev.filter_coefficients(lo, hi, m)
            V = torch.from_numpy(random_normal_block(csr.n, r, seed + 10 * r)).cuda()
            W_regular = torch.full_like(V, float("nan"))
            W_noalloc = torch.full_like(V, float("nan"))
            flz.flz_filter_apply(h, c, e, coeffs, m, r, V, W_regular)
            flz.flz_filter_apply_noalloc(csr.n, csr.nnz, rp, cl, vl, c, e, coeffs, m, r, V, W_noalloc)
            torch.cuda.synchronize()
            a = W_regular.cpu().numpy()
            b = W_noalloc.cpu().numpy()
            assert np.all(np.isfinite(b)), f"call {call}"
            # both evaluate the same FP64 forward recurrence; they differ only in
            # where the shift and scale are applied (rounding of order m u)
            assert np.max(np.abs(a - b)) <= 1e-13 * float(V.abs().max()), f"call {call}"
    finally:
        flz.flz_matrix_destroy(h)


def test_noalloc_wrapper_checks_the_coefficient_count():
    __graft_entry__.build()
    with pytest.raises(ValueError):
        flz.flz_filter_apply_noalloc(10, 0, 0, 0, 0, 0.0, 1.0, np.ones(3), 5, 1, 0, 0)


def test_noalloc_filter_rejects_oversized_blocks():
    __graft_entry__.build()
    n = 300000  # n * r = 1.2e6 > 1,048,576 at r = 4
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    ip = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(flz.FlzError) as e:
        flz.flz_filter_apply_noalloc(n, 0, ip, None, None, 0.0, 1.0, np.ones(3), 2, 4, dummy.data_ptr(),
                                     dummy.data_ptr() + 8 * 4 * n + 64)
    assert e.value.status == flz.FLZ_ERR_CAPACITY
