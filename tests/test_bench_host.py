"""The benchmark's roofline arithmetic on the CPU.

The algorithmic bytes of a degree step and of the reorthogonalization phase
decide the reported HBM fractions, so they are checked here against byte
counts worked out by hand for the 100^3 workload (n = 1,000,000,
nnz = 6,940,000, r = 4):

- forward step, 8-byte values: the CSR once (8-byte values, 4-byte columns,
  4 (n + 1) bytes of row pointers) = 87,280,004 bytes, plus per element of the
  n x r block a gather of Y_k, a read of Y_{k-1}, a write of Y_{k+1} and a read
  and a write of the sum, 5 x 8 bytes = 160,000,000 bytes: 247,280,004;
- FP32 storage: 4-byte values (59,520,004 bytes of CSR) and 5 x 4 bytes per
  element (80,000,000): 139,520,004;
- Clenshaw: V, B_{k+1} and B_{k+2} read, B_k written, 4 x 8 bytes per element:
  87,280,004 + 128,000,000 = 215,280,004;
- the reorthogonalization of 90 block steps reads the 16-byte digit copy of a
  basis of 4 (j + 1) columns four times at step j: 4 x 16 x 1e6 x 16,380
  columns = 1.04832e12 bytes.
"""

import math

import bench

N, NNZ, R = 1_000_000, 6_940_000, 4


def test_forward_step_bytes():
    assert bench.filter_bytes_per_launch(N, NNZ, R) == 247_280_004


def test_fp32_step_bytes():
    s_val, s_vec, s_acc = bench.ELEMENT_BYTES["fp32"]
    assert bench.filter_bytes_per_launch(N, NNZ, R, s_val, s_vec, s_acc) == 139_520_004


def test_clenshaw_step_bytes():
    assert bench.filter_bytes_per_launch(N, NNZ, R, recurrence="clenshaw") == 215_280_004


def test_bf16_storage_keeps_fp32_sums():
    # 2-byte values and vectors, 4-byte running sum: 6 bytes per stored entry,
    # 3 x 2 + 2 x 4 = 14 bytes per element
    s_val, s_vec, s_acc = bench.ELEMENT_BYTES["bf16"]
    assert bench.filter_bytes_per_launch(N, NNZ, R, s_val, s_vec, s_acc) == 6 * NNZ + 4 * (N + 1) + 14 * N * R


def test_reorthogonalization_phase_bytes_and_rate():
    st = {"iters": 90, "ortho": 2, "ms_orth": 221.0}
    out = bench.ortho_summary(st, N, R, 6788.3)
    assert out["path"] == "tensor"
    assert out["basis_bytes_read"] == 4 * 16 * N * 16_380 == 1_048_320_000_000
    assert math.isclose(out["achieved_gbs"], 1.04832e12 / 0.221 / 1e9)
    assert math.isclose(out["hbm_frac"], out["achieved_gbs"] / 6788.3)


def test_cuda_core_reorthogonalization_reads_the_fp64_basis():
    st = {"iters": 10, "ortho": 1, "ms_orth": 0.0}
    out = bench.ortho_summary(st, N, R, 6788.3)
    assert out["path"] == "cuda_cores"
    assert out["basis_bytes_read"] == 4 * 8 * N * (4 * 10 * 11 // 2)
    assert out["achieved_gbs"] is None and out["hbm_frac"] is None
