"""Writes tests/golden/config2_reference.json with the CPU oracle only.

Workload: 7-point Dirichlet Laplacian on a 100^3 grid plus a diagonal
potential 0.5 * U(0,1) (seed 2025), the lower end of the spectrum. The oracle
(block filtered Lanczos, FP64, r = 4) computes every eigenpair below a generous
upper end beta0; the script then places beta at the midpoint of the widest
spectral gap among eigenvalues 95..110 (so the count is about 100 and no
eigenvalue sits near an endpoint) and records the eigenvalues in [alpha, beta].

Run from the repository root:  python tests/golden/make_config2_reference.py

With --bench-degree M the script instead loads the stored reference and runs
the oracle once more on the stored [alpha, beta] at the benchmark's settings
(degree M, checks every 10 block steps), recording its block-step and check
counts under "oracle_at_bench_degree": the CPU timings of bench.py scale their
sampled per-step costs to that run.
"""

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import lanczos  # noqa: E402
from synth import csr_checksum, laplacian_3d_7pt, random_normal_block  # noqa: E402

SEED = 2025
ALPHA = 0.0
BETA0 = 0.2885


def main():
    rng = np.random.Generator(np.random.PCG64(SEED))
    Acsr = laplacian_3d_7pt(100, 100, 100, 0.5 * rng.random(100 ** 3))
    A = Acsr.to_scipy()
    t0 = time.time()
    res = lanczos.filtered_lanczos(A, ALPHA, BETA0, random_normal_block(Acsr.n, 4, 11),
                                   bounds_start=random_normal_block(Acsr.n, 1, 12)[:, 0],
                                   degree=60, tol=1e-10, max_blocks=400)
    wall = time.time() - t0
    lam = np.sort(res.eigenvalues)
    assert res.converged, "oracle did not converge"
    window = np.arange(95, min(111, lam.shape[0] - 1))
    gaps = lam[window + 1] - lam[window]
    k = int(window[np.argmax(gaps)])
    beta = 0.5 * (lam[k] + lam[k + 1])
    inside = lam[lam <= beta]
    out = {
        "_source": "written by tests/golden/make_config2_reference.py from the CPU oracle (oracle.lanczos.filtered_lanczos)",
        "grid": [100, 100, 100],
        "potential": "0.5 * PCG64(2025).random(1e6), added to the 7-point Laplacian diagonal",
        "matrix_checksum": csr_checksum(Acsr),
        "alpha": ALPHA,
        "beta": beta,
        "beta_gap": float(lam[k + 1] - lam[k]),
        "count": int(inside.shape[0]),
        "eigenvalues": [float(x) for x in inside],
        "oracle": {"degree": res.degree, "block_size": 4, "iters": res.iters, "bounds": [res.lmin, res.lmax],
                   "max_residual": float(np.max(res.residuals)), "wall_s": wall, "beta0": BETA0,
                   "count_below_beta0": int(lam.shape[0])},
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "config2_reference.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: v for k, v in out.items() if k != "eigenvalues"}, indent=1))


def bench_degree(m):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config2_reference.json")
    ref = json.load(open(path))
    rng = np.random.Generator(np.random.PCG64(SEED))
    Acsr = laplacian_3d_7pt(100, 100, 100, 0.5 * rng.random(100 ** 3))
    assert csr_checksum(Acsr) == ref["matrix_checksum"]
    t0 = time.time()
    res = lanczos.filtered_lanczos(Acsr.to_scipy(), ref["alpha"], ref["beta"], random_normal_block(Acsr.n, 4, 11),
                                   bounds_start=random_normal_block(Acsr.n, 1, 12)[:, 0],
                                   degree=m, tol=1e-10, check_every=10, max_blocks=400)
    wall = time.time() - t0
    assert res.converged and res.eigenvalues.shape[0] == ref["count"]
    ref["oracle_at_bench_degree"] = {
        "degree": m, "block_size": 4, "check_every": 10, "iters": res.iters, "checks": len(res.history),
        "count": int(res.eigenvalues.shape[0]), "max_residual": float(np.max(res.residuals)),
        "max_abs_diff_to_reference": float(np.max(np.abs(np.sort(res.eigenvalues) - np.array(ref["eigenvalues"])))),
        "wall_s": wall,
    }
    with open(path, "w") as f:
        json.dump(ref, f, indent=1)
    print(json.dumps(ref["oracle_at_bench_degree"], indent=1))


if __name__ == "__main__":
    if len(sys.argv) == 3 and sys.argv[1] == "--bench-degree":
        bench_degree(int(sys.argv[2]))
    else:
        main()
