"""Named benchmark workloads (parameters only; the matrices come from synth.matrices).

CONFIG2: 7-point Dirichlet Laplacian on a 100^3 grid (n = 1e6, nnz = 6.94e6)
plus a diagonal potential 0.5 * U(0,1) drawn from PCG64(2025); all eigenpairs
in [alpha, beta] at the low end of the spectrum. beta sits at the midpoint of
the widest spectral gap among eigenvalues 95..110 and `count` is the number of
eigenvalues in [alpha, beta]; both were computed by the CPU oracle with
tests/golden/make_config2_reference.py (tests/golden/config2_reference.json).
`reference_iters` is the oracle run's block-step count at degree 60, r = 4.
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
    "reference_iters": 120,
}
