"""Named benchmark workloads (parameters only; the matrices come from synth.matrices).

CONFIG2: 7-point Dirichlet Laplacian on a 100^3 grid (n = 1e6, nnz = 6.94e6)
plus a diagonal potential 0.5 * U(0,1) drawn from PCG64(2025); all eigenpairs
in [alpha, beta] at the low end of the spectrum. beta sits at the midpoint of
the widest spectral gap among eigenvalues 95..110 and `count` is the number of
eigenvalues in [alpha, beta]; both were computed by the CPU oracle with
tests/golden/make_config2_reference.py (tests/golden/config2_reference.json).

CONFIG3: real-space Hamiltonian stand-in: 4th-order 13-point FD -Laplacian on
a 120^3 grid (n = 1.728e6, nnz = 22,204,800) plus 64 negative Gaussian wells
(synth.matrices.gaussian_wells_potential, seed 3); the lowest eigenpairs up to
`beta` (the wells' bound states and the bottom of the box continuum). alpha
lies below the Gershgorin interval.

BATCH64: 64 independent 2D/3D Dirichlet Laplacians with U(0,1) diagonal
potentials (synth.matrices.uneven_batch, n log-uniform in [1e4, 2e5]), each
with the interval [0, beta_i] holding a target count drawn uniformly from
10..50. beta_i sits at the midpoint of the widest gap among the eigenvalues
around the target count; beta_i and the counts were computed by the CPU
oracle with tests/golden/make_batch64_reference.py
(tests/golden/batch64_reference.json).
"""

CONFIG2 = {
    "grid": 100,
    "seed": 2025,
    "potential_scale": 0.5,
    "alpha": 0.0,
    "beta": 0.28699178286577987,
    "count": 105,
    "degree": 60,
    "check_every": 10,
}

CONFIG3 = {
    "grid": 120,
    "wells": 64,
    "seed": 3,
    "alpha": -6.0,
    "degree": 200,
    "target": 200,
}

BATCH64 = {
    "count": 64,
    "seed": 4,
    "n_lo": 1e4,
    "n_hi": 2e5,
    "target_lo": 10,
    "target_hi": 50,
    "target_seed": 5,
}
