"""Writes tests/golden/batch64_reference.json with the CPU oracle only.

Workload (BATCH64 in synth/workloads.py): 64 independent 2D/3D Dirichlet
Laplacians with U(0,1) diagonal potentials, n log-uniform in [1e4, 2e5]. For
each problem a target count k is drawn from 10..50. The oracle's spectrum
bounds give lambda_min; a first upper end beta0 = lambda_min + Delta is set
from a Weyl-law estimate of where about k + 15 eigenvalues end (count ~ C n
Delta^(d/2), C fitted once on a few problems) and widened until the oracle's
filtered Lanczos finds at least k + 4 eigenvalues in [0, beta0]. beta is then
the midpoint of the widest gap among the eigenvalues k-3..k+3 (1-based), so no
eigenvalue lies near an endpoint, and the script records the eigenvalues in
[0, beta]. All potentials are >= 0 and the Laplacians are positive definite,
so [0, beta] starts below the spectrum.

Run from the repository root:  python tests/golden/make_batch64_reference.py
(about 10 minutes on 8 cores; one process per problem).
"""

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import lanczos  # noqa: E402
from synth import csr_checksum, random_normal_block, uneven_batch  # noqa: E402
from synth.workloads import BATCH64  # noqa: E402

WEYL = {"2d": (0.0068, 1.0), "3d": (0.014, 1.5)}  # count ~ C n Delta^p


def targets():
    g = np.random.Generator(np.random.PCG64(BATCH64["target_seed"]))
    return [int(x) for x in g.integers(BATCH64["target_lo"], BATCH64["target_hi"] + 1, BATCH64["count"])]


def one(i):
    items = uneven_batch(BATCH64["count"], seed=BATCH64["seed"], n_lo=BATCH64["n_lo"], n_hi=BATCH64["n_hi"])
    csr, kind, dims = items[i]
    k = targets()[i]
    A = csr.to_scipy()
    t0 = time.time()
    lmin, lmax, _ = lanczos.lanczos_bounds(A, random_normal_block(csr.n, 1, 1000 + i)[:, 0], 60)
    C, p = WEYL[kind]
    delta = ((k + 15) / (C * csr.n)) ** (1.0 / p)
    for attempt in range(8):
        beta0 = lmin + delta
        res = lanczos.filtered_lanczos(A, 0.0, beta0, random_normal_block(csr.n, 4, 2000 + i),
                                       bounds=(lmin, lmax), tol=1e-10, max_blocks=600)
        lam = np.sort(res.eigenvalues)
        if res.converged and lam.shape[0] >= k + 4:
            break
        delta *= 1.6
    else:
        raise RuntimeError(f"problem {i}: could not bracket {k} eigenvalues")
    window = np.arange(max(k - 4, 1), min(k + 3, lam.shape[0] - 1))  # 0-based: gaps after eigenvalue k-3..k+3
    gaps = lam[window + 1] - lam[window]
    j = int(window[np.argmax(gaps)])
    beta = 0.5 * (lam[j] + lam[j + 1])
    inside = lam[lam <= beta]
    return {
        "index": i, "kind": kind, "dims": list(dims), "n": csr.n, "nnz": csr.nnz,
        "matrix_checksum": csr_checksum(csr), "target": k, "alpha": 0.0, "beta": float(beta),
        "beta_gap": float(lam[j + 1] - lam[j]), "count": int(inside.shape[0]),
        "eigenvalues": [float(x) for x in inside],
        "oracle": {"degree": res.degree, "iters": res.iters, "bounds": [res.lmin, res.lmax],
                   "max_residual": float(np.max(res.residuals)), "beta0": float(beta0),
                   "count_below_beta0": int(lam.shape[0]), "attempts": attempt + 1,
                   "wall_s": time.time() - t0},
    }


def main():
    n_proc = min(os.cpu_count() or 1, 8)
    ctx = mp.get_context("spawn")
    with ctx.Pool(n_proc) as pool:
        rows = pool.map(one, range(BATCH64["count"]), chunksize=1)
    out = {
        "_source": "written by tests/golden/make_batch64_reference.py from the CPU oracle "
                   "(oracle.lanczos.lanczos_bounds, oracle.lanczos.filtered_lanczos)",
        "workload": dict(BATCH64),
        "problems": rows,
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch64_reference.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("total count", sum(r["count"] for r in rows), "max oracle wall", max(r["oracle"]["wall_s"] for r in rows))


if __name__ == "__main__":
    main()
