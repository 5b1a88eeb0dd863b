"""Writes tests/golden/config3_reference.json with the CPU oracle only.

Workload (CONFIG3 in synth/workloads.py): 4th-order 13-point FD -Laplacian on
a 120^3 grid plus 64 negative Gaussian wells (seed 3). The oracle (block
filtered Lanczos, FP64, r = 4, degree 200) computes every eigenpair in
[alpha, beta0] for beta0 = 0.03, 0.05, 0.08, ... until at least 206 are found
(the wells bind a few states below 0; above 0 the spectrum is the box's
dense low continuum). beta is then the midpoint of the widest gap among
eigenvalues 195..205 (1-based), and the script records the eigenvalues in
[alpha, beta].

Run from the repository root:  python tests/golden/make_config3_reference.py
(about an hour on one core).
"""

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import lanczos  # noqa: E402
from synth import csr_checksum, fd4_laplacian_3d, gaussian_wells_potential, random_normal_block  # noqa: E402
from synth.workloads import CONFIG3  # noqa: E402


def main():
    N = CONFIG3["grid"]
    Acsr = fd4_laplacian_3d(N, gaussian_wells_potential(N, CONFIG3["wells"], seed=CONFIG3["seed"]))
    A = Acsr.to_scipy()
    t0 = time.time()
    lmin, lmax, _ = lanczos.lanczos_bounds(A, random_normal_block(Acsr.n, 1, 31)[:, 0], 60)
    k = CONFIG3["target"]
    for beta0 in (0.03, 0.05, 0.08, 0.12, 0.2):
        res = lanczos.filtered_lanczos(A, CONFIG3["alpha"], beta0, random_normal_block(Acsr.n, 4, 32),
                                       bounds=(lmin, lmax), degree=CONFIG3["degree"], tol=1e-10, max_blocks=600)
        lam = np.sort(res.eigenvalues)
        print("beta0", beta0, "count", lam.shape[0], "converged", res.converged, "iters", res.iters,
              "elapsed %.0f s" % (time.time() - t0), flush=True)
        if res.converged and lam.shape[0] >= k + 6:
            break
    else:
        raise RuntimeError("could not bracket the target count")
    window = np.arange(k - 6, k + 5)  # 0-based: gaps after eigenvalues 195..205 (1-based)
    gaps = lam[window + 1] - lam[window]
    j = int(window[np.argmax(gaps)])
    beta = 0.5 * (lam[j] + lam[j + 1])
    inside = lam[lam <= beta]
    out = {
        "_source": "written by tests/golden/make_config3_reference.py from the CPU oracle (oracle.lanczos)",
        "grid": [N, N, N],
        "potential": f"{CONFIG3['wells']} Gaussian wells, synth.matrices.gaussian_wells_potential(seed={CONFIG3['seed']})",
        "matrix_checksum": csr_checksum(Acsr),
        "alpha": CONFIG3["alpha"],
        "beta": float(beta),
        "beta_gap": float(lam[j + 1] - lam[j]),
        "count": int(inside.shape[0]),
        "eigenvalues": [float(x) for x in inside],
        "oracle": {"degree": res.degree, "block_size": 4, "iters": res.iters, "bounds": [res.lmin, res.lmax],
                   "max_residual": float(np.max(res.residuals)), "wall_s": time.time() - t0, "beta0": beta0,
                   "count_below_beta0": int(lam.shape[0])},
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "config3_reference.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({kk: v for kk, v in out.items() if kk != "eigenvalues"}, indent=1))


if __name__ == "__main__":
    main()
