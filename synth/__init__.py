"""Seeded synthetic inputs shared by the tests, the benchmark and the CPU oracle's tests.

This package builds matrices and random blocks only. It holds none of the
filtered Lanczos arithmetic (no Chebyshev coefficients, no recurrences, no
Lanczos steps); both the CUDA path and the oracle receive its outputs as plain
arrays.

Every generator draws only from ``numpy.random.Generator(PCG64(seed))`` through
``random()`` (uniform doubles) and ``integers()``, whose output streams are
bit-identical across platforms, so x86 and aarch64 hosts build the same matrix
for the same seed. Normal variates are made from those uniforms by the
Box-Muller transform.
"""

from .matrices import (  # noqa: F401
    CSR,
    laplacian_2d,
    laplacian_3d_7pt,
    fd4_laplacian_3d,
    gaussian_wells_potential,
    powerlaw_graph_laplacian,
    parsec_like_hamiltonian,
    uneven_batch,
    random_normal_block,
    diagonal_csr,
    csr_checksum,
)
