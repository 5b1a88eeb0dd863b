"""Benchmark: eigenpairs/s of the GPU filtered Lanczos solver on a 3D Hamiltonian-like workload.

Workload (one GB300): the 7-point Dirichlet Laplacian on a 100^3 grid plus a
diagonal potential 0.5*U(0,1) (seed 2025), n = 1e6, nnz = 6.94e6, CSR FP64;
all eigenpairs in [alpha, beta] at the lower end of the spectrum (105),
block size 4, filter degree 100, residual tolerance 1e-10. The filter runs in
64-bit fixed point on the integer pipes (FP64-class: per degree one rounding
of 2^-62 of a column's norm per element); reorthogonalization, Rayleigh-Ritz
and residuals are FP64 (the plain FP64 filter is the "fp64_filter" variant).

One step = one flz_solve on the device-resident matrix: spectrum bounds,
filter construction, block Lanczos on p(A) with full reorthogonalization,
Rayleigh-Ritz checks and the Ritz vectors of the converged pairs (the time the
paper's Table 2 reports, bounds estimation included). L2 is flushed (a 512 MiB
write) before every timed step. `value` counts eigenpairs found with residual
<= 1e-8 per second of device time.

`e2e` is the same metric through the C ABI with host buffers: each step uploads
the CSR arrays from pinned host memory (flz_matrix_create_csr), solves, and
copies eigenvalues and eigenvectors back to the host.

`--impl reference` times the CPU oracle (numpy/scipy FP64) on the host cores on
a bounded sample of the same workload (see cpu_leg()).
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import (laplacian_3d_7pt, parsec_like_hamiltonian, powerlaw_graph_laplacian,  # noqa: E402
                   random_normal_block, uneven_batch)
from synth.matrices import fd4_laplacian_3d, gaussian_wells_potential  # noqa: E402
from synth.workloads import BATCH64, CONFIG2, CONFIG3  # noqa: E402

METRIC = "eigenpairs/s at residual 1e-8 (3D 7-point Laplacian 100^3 + potential, FP64)"
# Filter degree of the timed solve: among the degrees 40, 60, 100 and 150 on
# this workload, 100 gave the shortest time to solution (fewer block steps and
# reorthogonalizations at a moderate cost per step, as in Tables 2 and 3).
ORTHO = {"auto": 0, "cuda_cores": 1, "tensor": 2}
BENCH_DEGREE = 100
BATCH_DEGREE = 60


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def make_matrix():
    rng = np.random.Generator(np.random.PCG64(CONFIG2["seed"]))
    g = CONFIG2["grid"]
    return laplacian_3d_7pt(g, g, g, CONFIG2["potential_scale"] * rng.random(g ** 3))


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device=0):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate_ranks(seconds, pairs, dist=None, device="cpu"):
    """Whole-job totals over the ranks: the slowest rank's time (every rank's
    timed region starts after a barrier) and the eigenpairs all ranks found.
    Single process: the inputs."""
    if dist is None:
        return seconds, pairs
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    c = torch.tensor([pairs], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(c.item())


def filter_bytes_per_launch(n, nnz, r, s_val=8, s_vec=8, s_acc=8, recurrence="forward"):
    # CSR once (values + int32 columns + int32 row pointers) and the vector
    # streams. Forward: gather Y_k, read Y_{k-1}, write Y_{k+1}, read and
    # write the sum. Clenshaw: read V, gather B_{k+1}, read B_{k+2}, write B_k.
    csr = nnz * (s_val + 4) + 4 * (n + 1)
    if recurrence == "clenshaw":
        return csr + r * n * 4 * s_vec
    return csr + r * n * (3 * s_vec + 2 * s_acc)


def filter_flops_per_launch(n, nnz, r):
    # the degree step's arithmetic: a multiply-add per stored entry and column,
    # and per element the subtraction of Y_{k-1}, the shift and the running sum
    return 2 * nnz * r + 6 * n * r


# bytes per stored value, vector element and running-sum element of each filter arithmetic
PRECISION_NAMES = {0: "fp64", 1: "fp32", 2: "bf16", 3: "df64", 4: "fx64"}  # flz_precision values
ELEMENT_BYTES = {"fp64": (8, 8, 8), "fp32": (4, 4, 4), "bf16": (2, 2, 4), "df64": (8, 8, 8), "fx64": (8, 8, 8)}
KERNEL_NAMES = {
    ("fp64", "forward"): "cheb_sell_kernel<FP64> (fused Chebyshev degree step, SELL-32)",
    ("fp64", "clenshaw"): "clen_sell_kernel<FP64> (Clenshaw degree step, SELL-32)",
    ("fp32", "forward"): "cheb_sell_kernel<FP32>", ("fp32", "clenshaw"): "clen_sell_kernel<FP32>",
    ("bf16", "forward"): "cheb_sell_kernel<BF16>", ("bf16", "clenshaw"): "clen_sell_kernel<BF16>",
    ("df64", "forward"): "cheb_sell_kernel<double-FP32>", ("df64", "clenshaw"): "clen_sell_kernel<double-FP32>",
    ("fx64", "forward"): "fx_sell_kernel (64-bit fixed-point degree step, SELL-32 staged by bulk copies)",
}
# DRAM bytes (read + write) per launch from one ncu capture of the kernel as it
# is now, on this workload (profiles/); absent where no capture of the current
# kernel exists.
TRAFFIC = {("fx64", "forward"): 179.72e6 + 33.35e6}  # profiles/fx_sell_kernel_fx64_laplacian3d_100cubed_r4.md


def alu_fraction(flz, fprec, csr, r, ms_per_launch):
    """The degree step's arithmetic against the measured rate of its pipe: FP64
    FMAs for FP64; for the fixed-point step its 32-bit integer multiply-adds (7
    per product of a stored entry and a vector element, 2 ops each, and as many
    again per element for the running sum)."""
    try:
        if fprec == "fp64":
            peak = flz.flz_measure_alu_peak(0)
            work = filter_flops_per_launch(csr.n, csr.nnz, r)
            unit, what = "TFLOP/s", "FP64 flops (2 nnz r + 6 n r)"
        elif fprec == "fx64":
            peak = flz.flz_measure_alu_peak(1)
            work = 2 * 7 * (csr.nnz + csr.n) * r
            unit, what = "Tops/s", "32-bit integer multiply-add ops (2 x 7 per product)"
        else:
            return None
    except Exception as exc:  # the probe is a measurement aid; its failure is reported, not fatal
        return {"error": str(exc)}
    achieved = work / (ms_per_launch * 1e-3)
    return {"achieved": achieved / 1e12, "peak": peak / 1e12, "unit": unit, "frac": achieved / peak,
            "work_per_launch": work, "work": what, "peak_source": "measured (flz_measure_alu_peak)"}


def oracle_run_shape():
    """Block steps and convergence checks of the oracle's own solve of this workload at the benchmark's
    degree (tests/golden/config2_reference.json, written by tests/golden/make_config2_reference.py)."""
    ref = json.load(open(os.path.join(ROOT, "tests", "golden", "config2_reference.json")))
    o = ref["oracle_at_bench_degree"]
    return int(o["iters"]), int(o["checks"]), int(o["degree"]), int(ref["count"])


def cpu_leg(csr, alpha, beta, degree, r, budget_s=20.0):
    """Times the CPU oracle on a bounded sample and scales it to the oracle's whole solve.

    The oracle's own run of this workload at the benchmark's degree takes `iters`
    block steps with a convergence check every 10 (oracle_run_shape). Sample, in
    the oracle's own code: its bound estimation; block steps of its Clenshaw
    filter of the same degree until about `budget_s` seconds have passed (at
    least one); one full-reorthogonalization step as the oracle does it (basis
    concatenation, CGS2, Householder QR) against a basis of the run's average
    size r iters / 2; and the Ritz-pair work of a check (Ritz vector x = Q_k y,
    A x, Rayleigh quotient, residual) for a few pairs at that size. Scaled:
    the filter cost per step times `iters`; the reorthogonalization step (linear
    in the basis size) times `iters`; the two converged checks of the run (count
    stable over two checks) walking count + guard pairs each at the final basis
    size (earlier, partial walks are not counted, which favours the CPU).
    """
    from oracle import chebyshev, lanczos
    iters, checks, _, count = oracle_run_shape()
    A = csr.to_scipy()
    t0 = time.time()
    lmin, lmax, _ = lanczos.lanczos_bounds(A, random_normal_block(csr.n, 1, 12)[:, 0], 60)
    t_bounds = time.time() - t0
    c, e, am, bm = chebyshev.map_interval(alpha, beta, lmin, lmax)
    coeffs = chebyshev.filter_coefficients(max(am, -1.0), min(bm, 1.0), degree)
    Q, _ = np.linalg.qr(random_normal_block(csr.n, r, 11))
    t_filter, steps = 0.0, 0
    t_start = time.time()
    while (steps == 0 or time.time() - t_start < budget_s) and steps < 200:
        ta = time.time()
        W = chebyshev.clenshaw_apply(A, c, e, coeffs, Q)
        t_filter += time.time() - ta
        steps += 1
    # one reorthogonalization step against nb = iters / 2 blocks, as the oracle does it
    nb = max(1, iters // 2)
    rng = np.random.default_rng(5)
    blocks = [rng.standard_normal((csr.n, r)) / np.sqrt(csr.n) for _ in range(nb)]
    tb = time.time()
    Qall = np.hstack(blocks)
    C1 = Qall.T @ W
    W2 = W - Qall @ C1
    C2 = Qall.T @ W2
    W2 = W2 - Qall @ C2
    np.linalg.qr(W2)
    t_orth_mid = time.time() - tb
    # Ritz-pair work of a check at basis size nb r (one pair at a time, as the oracle)
    pairs = 4
    tp = time.time()
    for _ in range(pairs):
        y = rng.standard_normal(Qall.shape[1])
        x = Qall @ y
        x = x / np.linalg.norm(x)
        Ax = A @ x
        lam = float(x @ Ax)
        _ = float(np.linalg.norm(Ax - lam * x))
    t_pair_mid = (time.time() - tp) / pairs
    guard = max(r, 3)
    per_filter = t_filter / steps
    walk = 2 * (count + guard) * t_pair_mid * 2.0  # at the final basis size, twice the sampled one
    total = t_bounds + iters * (per_filter + t_orth_mid) + walk
    threads = os.environ.get("OPENBLAS_NUM_THREADS") or os.environ.get("OMP_NUM_THREADS")
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {
        "seconds_per_solve": total,
        "sample": (f"oracle bounds ({t_bounds:.1f} s), {steps} Clenshaw filters (degree {degree}, r = {r}) in "
                   f"{t_filter:.1f} s, one CGS2 + QR step and {pairs} Ritz pairs at basis size {nb * r}, scaled to "
                   f"the oracle's own run: {iters} block steps, {checks} checks, 2 converged walks of "
                   f"{count + guard} pairs"),
        "cores": int(threads) if threads else cores,
        "phases_s": {"bounds": t_bounds, "filter": iters * per_filter, "orth": iters * t_orth_mid, "checks": walk},
    }


def cpu_leg_threads(threads, degree, r, budget_s):
    """cpu_leg in a child process whose BLAS uses `threads` threads (set before numpy loads)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--mode", "cpu_leg", "--degree", str(degree),
                          "--block-size", str(r), "--cpu-budget", str(budget_s)],
                         capture_output=True, text=True, env=env, timeout=1200)
    if out.returncode != 0:
        raise RuntimeError(f"cpu leg failed: {out.stderr[-2000:]}")
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_reference(args):
    """The oracle on the host cores: every step a bounded sample (cpu_leg) scaled to the oracle's whole solve."""
    csr = make_matrix()
    alpha, beta = CONFIG2["alpha"], CONFIG2["beta"]
    vals = []
    for _ in range(args.warmup + args.steps):
        vals.append(cpu_leg(csr, alpha, beta, args.degree, args.block_size, budget_s=args.reference_budget))
    timed = vals[args.warmup:]
    per_solve = float(np.mean([v["seconds_per_solve"] for v in timed]))
    value = CONFIG2["count"] / per_solve
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_solve * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(csr, args),
        "cpu_baseline": {"value": value, "unit": "eigenpairs/s", "cores": timed[-1]["cores"], "kind": "oracle",
                         "sample": timed[-1]["sample"]},
        "e2e": {"value": value, "unit": "eigenpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def ortho_summary(st, n, r, hbm):
    """The reorthogonalization phase as a whole (CGS2 + block QR + the small
    kernels between them) against HBM: on the tensor cores each of the four
    passes of a step reads the digit copy of the K-column basis once (16 bytes
    per value), so the algorithmic bytes of a solve are 4 * 16 * n * sum_j K_j
    with K_j = r (j + 1) at block step j. On the CUDA cores the same passes read
    the FP64 basis (8 bytes per value) and are FP64-pipe bound (r / 4 flop/B)."""
    iters = int(st["iters"])
    cols = r * iters * (iters + 1) // 2
    tensor = st["ortho"] == 2
    nbytes = 4 * (16 if tensor else 8) * n * cols
    gbs = nbytes / (st["ms_orth"] * 1e-3) / 1e9 if st["ms_orth"] > 0 else None
    return {"path": "tensor" if tensor else "cuda_cores", "ms": st["ms_orth"],
            "basis_bytes_read": nbytes, "achieved_gbs": gbs, "hbm_frac": (gbs / hbm) if gbs else None,
            "flops": 4 * 2 * n * cols * r}


def config_dict(csr, args):
    return {"workload": "3D 7-point Dirichlet Laplacian 100^3 + 0.5*U(0,1) potential (seed 2025), "
                        "all eigenpairs in [alpha, beta] at the low end of the spectrum",
            "n": csr.n, "nnz": csr.nnz, "alpha": CONFIG2["alpha"], "beta": CONFIG2["beta"],
            "block_size": args.block_size, "degree": args.degree, "precision": args.precision, "tol": args.tol,
            "check_every": args.check_every, "recurrence": args.recurrence, "ortho": args.ortho,
            "l2": "flushed (512 MiB write) before each timed step", "parallelism": "single GPU"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--degree", type=int, default=BENCH_DEGREE)
    ap.add_argument("--block-size", type=int, default=4)
    ap.add_argument("--precision", default="fx64", choices=["fp64", "fp32", "bf16", "df64", "fx64"],
                    help="filter arithmetic (fx64: the 64-bit fixed-point filter, FP64-class; the rest of the "
                         "solver is FP64 in every mode)")
    ap.add_argument("--recurrence", default="forward", choices=["forward", "clenshaw"])
    ap.add_argument("--damping", default="none", choices=["none", "jackson", "sigma"],
                    help="filter damping (the paper uses none)")
    ap.add_argument("--ortho", default="auto", choices=["auto", "cuda_cores", "tensor"],
                    help="where the full reorthogonalization runs (auto: tensor cores for r <= 4)")
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--check-every", type=int, default=CONFIG2["check_every"])
    ap.add_argument("--table2-check", type=int, default=30,
                    help="--mode table2: block steps between convergence checks (Table 2's counts are multiples of 30)")
    ap.add_argument("--cpu-budget", type=float, default=12.0,
                    help="seconds of oracle block steps per CPU-baseline sample (each of 1 thread and all threads)")
    ap.add_argument("--reference-budget", type=float, default=3.0,
                    help="seconds of oracle block steps per --impl reference step")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the FP32/BF16-filter solves reported under 'variants'")
    ap.add_argument("--no-batch", action="store_true", help="skip the batch-of-64 leg")
    ap.add_argument("--batch-legs", default="fp32,fp64,df64,fx64,fx64_persistent,fp32_refined,sequential",
                    help="--mode batch: the legs to run (a single leg with --batch-once runs one solve, no warm-up)")
    ap.add_argument("--batch-once", action="store_true", help="--mode batch: one solve per leg, no warm-up (profiling)")
    ap.add_argument("--batch-check-every", type=int, default=5,
                    help="--mode batch: block steps between convergence checks of the batch legs")
    ap.add_argument("--batch-tile-rows", type=int, default=0,
                    help="--mode batch: rows per CTA of the fixed-point batch kernel (0: autotuned; 128 or 256)")
    ap.add_argument("--batch-block-size", type=int, default=0,
                    help="--mode batch: block width of the batch legs (0: autotuned, which timings under a profiler distort)")
    ap.add_argument("--ortho-n", type=int, default=1_000_000, help="rows of the --mode ortho basis")
    ap.add_argument("--ortho-basis", type=int, default=120, help="columns of the --mode ortho basis")
    ap.add_argument("--mode", default="solve", choices=["solve", "filter", "batch", "table2", "graph", "slices",
                                                        "ortho", "config3", "cpu_leg", "sequence"],
                    help="solve: whole flz_solve per step (default); filter: only flz_filter_apply at the "
                         "solver's shape, for the kernel roofline and profiling")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.mode == "cpu_leg":  # child process of cpu_leg_threads
        leg = cpu_leg(make_matrix(), CONFIG2["alpha"], CONFIG2["beta"], args.degree, args.block_size, args.cpu_budget)
        print(json.dumps(leg))
        return
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import __graft_entry__
    __graft_entry__.build()
    import paper_2409_15053_gb300 as flz

    prec = {"fp64": flz.FLZ_PREC_FP64, "fp32": flz.FLZ_PREC_FP32, "bf16": flz.FLZ_PREC_BF16,
            "df64": flz.FLZ_PREC_DF64, "fx64": flz.FLZ_PREC_FX64}[args.precision]
    if args.mode == "batch":
        print(json.dumps({"mode": "batch", **batch_leg(flz, torch, torch.cuda.current_stream(),
                                                        legs=args.batch_legs.split(","), once=args.batch_once,
                                                        block_size=args.batch_block_size,
                                                        tile_rows=args.batch_tile_rows,
                                                        check_every=args.batch_check_every)}))
        return
    if args.mode == "table2":
        return table2_mode(flz, torch, prec, args)
    if args.mode == "graph":
        return graph_mode(flz, torch, args)
    if args.mode == "slices":
        return slices_mode(flz, torch, prec, args)
    if args.mode == "ortho":
        return ortho_mode(flz, torch, args)
    if args.mode == "config3":
        return config3_mode(flz, torch, args)
    if args.mode == "sequence":
        return sequence_mode(flz, torch, prec, args)
    csr = make_matrix()
    if args.mode == "filter":
        return filter_mode(flz, torch, csr, prec, args)
    alpha, beta = CONFIG2["alpha"], CONFIG2["beta"]
    # Replicas: every rank solves the same workload on its own GPU (the
    # solver does not shard; no data-path collective).
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
    p = flz.flz_params_default()
    p.block_size = args.block_size
    p.degree = args.degree
    p.tol = args.tol
    p.check_every = args.check_every
    p.precision = prec
    p.recurrence = {"forward": flz.FLZ_REC_FORWARD, "clenshaw": flz.FLZ_REC_CLENSHAW}[args.recurrence]
    p.damping = {"none": 0, "jackson": 1, "sigma": 2}[args.damping]
    p.ortho = ORTHO[args.ortho]
    p.seed = 1 + rank
    s = flz.flz_solver_create(h, p)
    flz.flz_solver_set_interval(s, alpha, beta)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")

    def one_solve():
        st = flz.flz_solve(s, stream)
        return st

    for _ in range(args.warmup):
        one_solve()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    times, found, stats_list = [], [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = one_solve()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        res = flz.flz_get_residuals(s)
        found.append(int(np.sum(res <= 1e-8)))
        stats_list.append(flz.flz_get_stats(s))
        check_history = flz.flz_get_checks(s)
        assert st == flz.FLZ_OK, flz.flz_status_string(st)
    clocks = sampler.stop()
    total_time, total_pairs = aggregate_ranks(float(np.sum(times)), int(sum(found)), dist, "cuda")
    value = total_pairs / total_time
    st = stats_list[-1]

    # Roofline of the dominant kernel (the fused Chebyshev degree step), from
    # the solver's own CUDA-event timing of its filter applications: the roof is
    # HBM (algorithmic bytes per launch / launch time, against the measured copy
    # rate); the arithmetic fraction is reported beside it against the rate of
    # the pipe the kernel computes on, measured on this GPU (flz_measure_alu_peak).
    launches_filter = st["iters"] * st["degree"]
    ms_per_launch = st["ms_filter"] / max(launches_filter, 1)
    fprec = {0: "fp64", 1: "fp32", 2: "bf16", 3: "df64", 4: "fx64"}[st["filter_precision"]]
    nbytes = filter_bytes_per_launch(csr.n, csr.nnz, args.block_size, *ELEMENT_BYTES[fprec],
                                     recurrence=args.recurrence)
    hbm, hbm_src = peaks()
    achieved_gbs = nbytes / (ms_per_launch * 1e-3) / 1e9
    roofline = {
        "kernel": KERNEL_NAMES[(fprec, args.recurrence)],
        "bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s", "frac": achieved_gbs / hbm,
        "peak_source": hbm_src, "traffic": TRAFFIC.get((fprec, args.recurrence)),
        "algorithmic_bytes_per_launch": nbytes, "ms_per_launch": ms_per_launch,
        "alu": alu_fraction(flz, fprec, csr, args.block_size, ms_per_launch),
    }

    fp64_vals = flz.flz_get_eigenvalues(s).copy()
    variants = None
    if not args.no_variants and args.precision == "fx64":
        variants = variant_leg(flz, torch, h, p, alpha, beta, stream, flush, fp64_vals, args)

    batch = None
    if not args.no_batch and rank == 0:
        batch = batch_leg(flz, torch, stream)

    e2e = None
    if not args.no_e2e:
        e2e = e2e_leg(flz, torch, csr, p, alpha, beta, stream, args)

    cpu = None
    if not args.no_cpu and rank == 0:
        legs = {t: cpu_leg_threads(t, args.degree, args.block_size, args.cpu_budget)
                for t in (len(os.sched_getaffinity(0)), 1)}
        allt, one = legs[max(legs)], legs[1]
        cpu = {"value": CONFIG2["count"] / allt["seconds_per_solve"], "unit": "eigenpairs/s",
               "cores": allt["cores"], "kind": "oracle", "sample": allt["sample"], "phases_s": allt["phases_s"],
               "one_thread": {"value": CONFIG2["count"] / one["seconds_per_solve"], "cores": 1,
                              "phases_s": one["phases_s"]},
               "gpu_speedup": {"vs_all_threads": value / (CONFIG2["count"] / allt["seconds_per_solve"]),
                               "vs_one_thread": value / (CONFIG2["count"] / one["seconds_per_solve"])}}

    flz.flz_solver_destroy(s)
    flz.flz_matrix_destroy(h)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_time / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "bf16": "bf16", "df64": "f32x2", "fx64": "i64"}[args.precision],
            "data": "synthetic", "config": config_dict(csr, args), "roofline": roofline, "cpu_baseline": cpu,
            "e2e": e2e, "variants": variants, "batch64": batch, "gpu_launches": int(sum(x["kernel_launches"] for x in stats_list)), "clocks": clocks,
            "solver": {k: st[k] for k in ("iters", "matvecs", "count", "degree", "checks", "lmin", "lmax",
                                          "max_residual", "ms_bounds", "ms_filter", "ms_orth", "ms_check",
                                          "ms_total", "basis_vectors", "kernel_launches", "ortho")},
            "ortho": ortho_summary(st, csr.n, args.block_size, hbm),
            # the timed solve's convergence checks: [block steps, pairs inside, walked, outside, all passed, ended]
            "check_history": [[c["block_steps"], c["inside"], c["walked"], c["outside"], c["all_small"], c["converged"]]
                              for c in check_history],
            "found_per_step": found,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def variant_leg(flz, torch, h, p, alpha, beta, stream, flush, ref_vals, args):
    """Filter variants versus the headline (fixed-point) run on the same workload
    (everything but the filter stays FP64): plain FP64 (tensor-core or CUDA-core
    reorthogonalization), double-FP32 (hi + lo FP32 pairs) and the Clenshaw
    recurrence at the FP64 tolerance, FP32 / BF16 storage at the residual those
    reach alone (1e-6, 1e-3), and the same refined to 1e-8 (params.refine: the
    mixed-precision form), each with its eigenvalue
    difference to the headline run. Times 2 solves after 1 warm-up, device time per
    solve. `value` counts pairs with residual <= 1e-8."""
    out = {}
    # the reduced-precision filters at the residual they can reach, double-FP32 at the FP64 tolerance
    F, C = flz.FLZ_REC_FORWARD, flz.FLZ_REC_CLENSHAW
    T, CC = flz.FLZ_ORTHO_AUTO, flz.FLZ_ORTHO_CUDA_CORES
    for name, prec, tol, rec, ortho, refine in (("fp64_filter", flz.FLZ_PREC_FP64, p.tol, F, T, 0),
                                                ("fp64_cuda_core_ortho", flz.FLZ_PREC_FP64, p.tol, F, CC, 0),
                                                ("fp64_clenshaw", flz.FLZ_PREC_FP64, p.tol, C, T, 0),
                                                ("df64_filter", flz.FLZ_PREC_DF64, p.tol, F, T, 0),
                                                ("df64_clenshaw", flz.FLZ_PREC_DF64, p.tol, C, T, 0),
                                                ("fp32_filter", flz.FLZ_PREC_FP32, 1e-6, F, T, 0),
                                                ("bf16_filter", flz.FLZ_PREC_BF16, 1e-3, F, T, 0),
                                                ("fp32_filter_refined", flz.FLZ_PREC_FP32, 1e-8, F, T, 1),
                                                ("bf16_filter_refined", flz.FLZ_PREC_BF16, 1e-8, F, T, 1)):
        q = flz.flz_params_default()
        for f, _ in q._fields_:
            setattr(q, f, getattr(p, f))
        q.precision = prec
        q.recurrence = rec
        q.ortho = ortho
        q.refine = refine
        q.tol = tol if refine else max(tol, p.tol)
        sv = flz.flz_solver_create(h, q)
        flz.flz_solver_set_interval(sv, alpha, beta)
        flz.flz_solve(sv, stream)
        times, st = [], None
        for _ in range(2):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = flz.flz_solve(sv, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        vals = flz.flz_get_eigenvalues(sv)
        res = flz.flz_get_residuals(sv)
        stats = flz.flz_get_stats(sv)
        flz.flz_solver_destroy(sv)
        same = vals.shape == ref_vals.shape
        out[name] = {
            "status": flz.flz_status_string(st), "value": float(np.sum(res <= 1e-8)) / float(np.mean(times)),
            "unit": "eigenpairs/s", "ms_per_solve": 1e3 * float(np.mean(times)), "count": int(vals.shape[0]),
            "tol": q.tol, "solves_per_s": 1.0 / float(np.mean(times)),
            "max_abs_eig_diff_vs_headline": float(np.max(np.abs(vals - ref_vals))) if same and vals.size else None,
            "max_residual": float(np.max(res)) if res.size else None,
            "ms_filter": stats["ms_filter"], "ms_orth": stats["ms_orth"], "ms_check": stats["ms_check"],
            "iters": stats["iters"], "ortho": ["auto", "cuda_cores", "tensor"][stats["ortho"]],
            "refine_sweeps": stats["refine_sweeps"], "refine_degree": stats["refine_degree"],
            "ms_refine": stats["ms_refine"],
        }
    return out


def batch_leg(flz, torch, stream, legs=("fp32", "fp64", "df64", "fx64", "fx64_persistent", "fp32_refined", "sequential"),
              once=False,
              block_size=0, tile_rows=0, check_every=5):
    """The batched form against one-at-a-time FP64 solves on the same GPU.

    Workload: 64 independent 2D/3D Laplacians with U(0,1) potentials, n
    log-uniform in [1e4, 2e5], each with the interval [0, beta_i] and the
    eigenvalue counts the CPU oracle computed (tests/golden/batch64_reference.json).
    Times (CUDA events, after one warm-up solve each): the batch with the FP32
    filter (tol 1e-6, its attainable residual), the batch with the FP64 and
    with the double-FP32 filter (tol 1e-10), and the 64 problems solved one
    after another with the FP64
    filter (r = 4); filter degree 60 throughout (the eps-rule's degrees of
    17-23 would need up to 480 block steps). Each result is checked against
    the oracle's counts and eigenvalues."""
    ref = json.load(open(os.path.join(ROOT, "tests", "golden", "batch64_reference.json")))["problems"]
    items = uneven_batch(BATCH64["count"], seed=BATCH64["seed"], n_lo=BATCH64["n_lo"], n_hi=BATCH64["n_hi"])
    hs = [flz.flz_matrix_create_csr(c.n, c.nnz, c.rowptr, c.col, c.val) for c, _, _ in items]
    alphas = [p["alpha"] for p in ref]
    betas = [p["beta"] for p in ref]
    want = [np.array(p["eigenvalues"]) for p in ref]
    total = int(sum(w.shape[0] for w in want))

    def timed(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / 1e3

    def score(vals_list, res_list, norms, tol):
        counts_ok = all(v.shape == w.shape for v, w in zip(vals_list, want))
        err = max((float(np.max(np.abs(v - w)) / nrm) if v.shape == w.shape and v.size else 0.0)
                  for v, w, nrm in zip(vals_list, want, norms))
        good = int(sum(np.sum(r <= tol) for r in res_list))
        return counts_ok, err, good

    out = {"problems": len(items), "sum_n": int(sum(c.n for c, _, _ in items)), "eigenpairs": total}
    for name, prec, tol in (("batch_fp32", flz.FLZ_PREC_FP32, 1e-6), ("batch_fp64", flz.FLZ_PREC_FP64, 1e-10),
                            ("batch_df64", flz.FLZ_PREC_DF64, 1e-10), ("batch_fx64", flz.FLZ_PREC_FX64, 1e-10),
                            ("batch_fx64_persistent", flz.FLZ_PREC_FX64, 1e-10),
                            ("batch_fp32_refined", flz.FLZ_PREC_FP32, 1e-8)):
        if name[6:] not in legs:
            continue
        p = flz.flz_params_default()
        p.block_size = block_size
        p.degree = BATCH_DEGREE
        p.precision = prec
        p.tol = tol
        p.check_every = check_every
        p.persistent = 1 if name.endswith("persistent") else 0
        p.refine = 1 if name.endswith("refined") else 0
        p.tile_rows = tile_rows
        bt = flz.flz_batch_create(hs, alphas, betas, p)
        if not once:
            flz.flz_batch_solve(bt, stream)
        st, sec = timed(lambda: flz.flz_batch_solve(bt, stream))
        vals = [flz.flz_batch_get_eigenvalues(bt, i) for i in range(len(items))]
        res = [flz.flz_batch_get_residuals(bt, i) for i in range(len(items))]
        stats = [flz.flz_batch_get_stats(bt, i) for i in range(len(items))]
        norms = [max(abs(x["lmin"]), abs(x["lmax"])) for x in stats]
        ok, err, good = score(vals, res, norms, tol)
        out[name] = {"status": flz.flz_status_string(st), "seconds": sec, "eigenpairs_per_s": good / sec,
                     "tol": tol, "counts_match_oracle": ok, "max_rel_eig_err_vs_oracle": err,
                     "block_size": stats[0]["block_size"], "max_iters": max(x["iters"] for x in stats),
                     "filter_precision": PRECISION_NAMES.get(stats[0]["filter_precision"]),
                     "refine_ms_sum": sum(x["ms_refine"] for x in stats),
                     "tile_rows": stats[0]["tile_rows"],
                     "ms_bounds": stats[0]["ms_bounds"], "ms_steps": stats[0]["ms_filter"],
                     "ms_check": stats[0]["ms_check"], "max_checks": max(x["checks"] for x in stats),
                     # rows and stored entries times block steps, summed over the problems (filter traffic)
                     "row_steps": int(sum(x["iters"] * c.n for x, (c, _, _) in zip(stats, items))),
                     "nnz_steps": int(sum(x["iters"] * c.nnz for x, (c, _, _) in zip(stats, items)))}
        flz.flz_batch_destroy(bt)
    if "sequential" in legs:
        p = flz.flz_params_default()
        p.block_size = 4
        p.degree = BATCH_DEGREE
        p.check_every = check_every
        solvers = []
        for h, a, z in zip(hs, alphas, betas):
            sv = flz.flz_solver_create(h, p)
            flz.flz_solver_set_interval(sv, a, z)
            flz.flz_solve(sv, stream)
            solvers.append(sv)

        def all_solves():
            return [flz.flz_solve(sv, stream) for sv in solvers]

        sts, sec = timed(all_solves)
        vals = [flz.flz_get_eigenvalues(sv) for sv in solvers]
        res = [flz.flz_get_residuals(sv) for sv in solvers]
        norms = []
        for sv in solvers:
            x = flz.flz_get_stats(sv)
            norms.append(max(abs(x["lmin"]), abs(x["lmax"])))
        ok, err, good = score(vals, res, norms, 1e-10)
        out["sequential_fp64"] = {"status": "FLZ_OK" if all(x == flz.FLZ_OK for x in sts) else "some not converged",
                                  "seconds": sec, "eigenpairs_per_s": good / sec, "tol": 1e-10,
                                  "counts_match_oracle": ok, "max_rel_eig_err_vs_oracle": err, "block_size": 4}
        for sv in solvers:
            flz.flz_solver_destroy(sv)
    for h in hs:
        flz.flz_matrix_destroy(h)
    return out


# Table 2's Ge87H76 rows (K40, Cucheb, r = 3): degree -> (iters, MV, seconds, max residual)
TABLE2_GE87H76 = {50: (210, 31500, 31, 1.7e-14), 100: (180, 54000, 40, 4.0e-13), 150: (150, 67500, 44, 7.4e-14),
                  200: (150, 90000, 56, 6.3e-14), "auto (49)": (210, 30870, 31, 9.0e-14)}


def table2_mode(flz, torch, prec, args):
    """Table 2's sweep on a synthetic stand-in shaped like Ge87H76.

    The PARSEC matrices are not available; parsec_like_hamiltonian() builds a
    real-space Hamiltonian of the same size, density and spectral interval
    (12th-order finite differences on a sphere, Gaussian local potentials,
    dense non-local projector blocks). Interval [-0.645, -0.0053] as in
    Table 2, block size 3, degrees 50, 100, 150, 200 and automatic, checks every
    30 block steps (--table2-check); one warm-up solve per degree, then one timed solve (CUDA
    events). The paper's K40 numbers for Ge87H76 are printed beside each row
    for context (a different matrix of the same shape, on other hardware)."""
    csr = parsec_like_hamiltonian()
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
    stream = torch.cuda.current_stream()
    rows = []
    for m in (50, 100, 150, 200, 0):
        p = flz.flz_params_default()
        p.block_size = 3
        p.degree = m
        p.precision = prec
        p.tol = args.tol
        p.check_every = args.table2_check
        p.recurrence = {"forward": flz.FLZ_REC_FORWARD, "clenshaw": flz.FLZ_REC_CLENSHAW}[args.recurrence]
        p.damping = {"none": 0, "jackson": 1, "sigma": 2}[args.damping]
        s = flz.flz_solver_create(h, p)
        flz.flz_solver_set_interval(s, -0.645, -0.0053)
        flz.flz_solve(s, stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = flz.flz_solve(s, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        x = flz.flz_get_stats(s)
        res = flz.flz_get_residuals(s)
        key = m if m else "auto (%d)" % x["degree"]
        paper = TABLE2_GE87H76.get(m if m else "auto (49)")
        rows.append({"m": key, "status": flz.flz_status_string(st), "eigs": int(x["count"]), "iters": int(x["iters"]),
                     "MV": int(x["matvecs"]), "seconds": e0.elapsed_time(e1) / 1e3,
                     "residual": float(res.max()) if res.size else None,
                     "PREPROC_ORTH_MV_percent": [round(100 * x["ms_bounds"] / x["ms_total"]),
                                                 round(100 * x["ms_orth"] / x["ms_total"]),
                                                 round(100 * x["ms_filter"] / x["ms_total"])],
                     "paper_K40": {"iters": paper[0], "MV": paper[1], "seconds": paper[2], "residual": paper[3]},
                     "checks": [[c["block_steps"], c["inside"], c["walked"], c["outside"], c["all_small"]]
                                for c in flz.flz_get_checks(s)]})
        flz.flz_solver_destroy(s)
    flz.flz_matrix_destroy(h)
    print(json.dumps({"mode": "table2", "matrix": "synthetic Ge87H76-shaped stand-in", "n": csr.n, "nnz": csr.nnz,
                      "interval": [-0.645, -0.0053], "block_size": 3, "precision": args.precision,
                      "check_every": args.table2_check,
                      "checks_format": "[block steps, pairs in the window, pairs walked, guard pairs met, all passed]",
                      "recurrence": args.recurrence, "damping": args.damping,
                      "tol": args.tol, "rows": rows}))


def slices_mode(flz, torch, prec, args):
    """Spectrum slicing on the benchmark workload: the same [alpha, beta] solved
    as 1, 2, 3 and 4 equal-width slices (one timed flz_solve_sliced after a
    warm-up each); count, residual, summed block steps and phase times."""
    csr = make_matrix()
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
    stream = torch.cuda.current_stream()
    rows = []
    for k in (1, 2, 3, 4):
        p = flz.flz_params_default()
        p.block_size = args.block_size
        p.degree = args.degree
        p.precision = prec
        p.tol = args.tol
        p.check_every = args.check_every
        p.recurrence = {"forward": flz.FLZ_REC_FORWARD, "clenshaw": flz.FLZ_REC_CLENSHAW}[args.recurrence]
        s = flz.flz_solver_create(h, p)
        flz.flz_solver_set_interval(s, CONFIG2["alpha"], CONFIG2["beta"])
        flz.flz_solve_sliced(s, k, stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = flz.flz_solve_sliced(s, k, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        x = flz.flz_get_stats(s)
        res = flz.flz_get_residuals(s)
        rows.append({"slices": k, "status": flz.flz_status_string(st), "count": int(x["count"]),
                     "seconds": e0.elapsed_time(e1) / 1e3, "max_residual": float(res.max()) if res.size else None,
                     "block_steps": int(x["iters"]), "ms_filter": x["ms_filter"], "ms_orth": x["ms_orth"],
                     "ms_check": x["ms_check"], "largest_basis": int(x["basis_vectors"])})
        flz.flz_solver_destroy(s)
    flz.flz_matrix_destroy(h)
    print(json.dumps({"mode": "slices", "workload": config_dict(csr, args)["workload"], "expected_count": CONFIG2["count"],
                      "precision": args.precision, "degree": args.degree, "rows": rows}))


def graph_mode(flz, torch, args):
    """The irregular workload: a power-law graph Laplacian, n = 4e6.

    Chung-Lu expected degrees (exponent 2.5, mean 15), weights U(0.1, 1), plus
    a ring (seed 5): about 64e6 stored entries, rows from 3 to ~8200 entries.
    Interval [alpha, beta] at the top of the spectrum holding about 500
    eigenpairs (the modes localized on the heaviest hubs): alpha is the
    520th-largest weighted degree, beta lies above the spectrum. Block size
    16. The FP32-storage filter (tol 1e-5) and the double-FP32 mode (tol 1e-9),
    each above its rounding floor for this ||A||, against plain FP64 (tol
    1e-10), one timed solve each after a warm-up; eigenvalue differences to
    the FP64 run."""
    t0 = time.time()
    csr = powerlaw_graph_laplacian(4_000_000, seed=5)
    gen_s = time.time() - t0
    deg = np.diff(csr.rowptr)
    S_diag = np.zeros(csr.n)
    rows = np.repeat(np.arange(csr.n), deg)
    on = rows == csr.col
    S_diag[rows[on]] = csr.val[on]
    alpha = float(np.sort(S_diag)[-520])
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
    stream = torch.cuda.current_stream()
    out = {"mode": "graph", "n": csr.n, "nnz": csr.nnz, "max_row": int(deg.max()), "generate_s": gen_s,
           "alpha": alpha, "block_size": 16, "degree": args.degree}
    ref = None
    # tolerances above each arithmetic's floor for ||A|| ~ 4.8e3
    for name, prec, tol in (("fp64", flz.FLZ_PREC_FP64, 1e-10), ("fp32_filter", flz.FLZ_PREC_FP32, 1e-5),
                            ("df64", flz.FLZ_PREC_DF64, 1e-9)):
        p = flz.flz_params_default()
        p.block_size = 16
        p.degree = args.degree
        p.precision = prec
        p.tol = tol
        p.check_every = 10
        # 110 block steps of 16: room for the ~100 the solve takes, and for the
        # basis's digit copy (24 bytes per value with the FP64 basis) in HBM
        p.max_basis = 1760
        s = flz.flz_solver_create(h, p)
        flz.flz_solver_set_interval(s, alpha, 1e9)
        flz.flz_solve(s, stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = flz.flz_solve(s, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        x = flz.flz_get_stats(s)
        vals = flz.flz_get_eigenvalues(s)
        res = flz.flz_get_residuals(s)
        if name == "fp64":
            ref = vals.copy()
        out[name] = {"status": flz.flz_status_string(st), "seconds": e0.elapsed_time(e1) / 1e3,
                     "count": int(vals.shape[0]), "iters": int(x["iters"]), "degree": int(x["degree"]),
                     "max_residual": float(res.max()) if res.size else None,
                     "eigenpairs_per_s_at_1e-8": float(np.sum(res <= 1e-8)) / (e0.elapsed_time(e1) / 1e3),
                     "ms_filter": x["ms_filter"], "ms_orth": x["ms_orth"], "ms_check": x["ms_check"],
                     "ortho": ["auto", "cuda_cores", "tensor"][x["ortho"]], "lmin": x["lmin"], "lmax": x["lmax"],
                     "max_abs_eig_diff_vs_headline": (float(np.max(np.abs(vals - ref)))
                                                  if ref is not None and vals.shape == ref.shape and vals.size else None)}
        flz.flz_solver_destroy(s)
    flz.flz_matrix_destroy(h)
    print(json.dumps(out))


def config3_mode(flz, torch, args):
    """The 4th-order finite-difference Hamiltonian at full size (120^3 grid,
    64 Gaussian wells, n = 1.728e6, 22.2e6 entries), r = 4, checks every 10
    block steps, one warm-up then one timed solve per row: the bound states
    [-6, -0.2] (m = 200), [-6, 0] (m = 300) and [-6, 0.03] reaching into the
    box continuum (m = 400) with the fixed-point filter; the bound states and
    the widest window also with the plain FP64 filter, the FP32 filter refined
    to 1e-8 (params.refine) and the double-FP32 filter and basis."""
    N = CONFIG3["grid"]
    csr = fd4_laplacian_3d(N, gaussian_wells_potential(N, CONFIG3["wells"], seed=CONFIG3["seed"]))
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
    stream = torch.cuda.current_stream()
    F, C = flz.FLZ_REC_FORWARD, flz.FLZ_REC_CLENSHAW
    rows = []
    O = ORTHO[args.ortho]
    X, D, S, H = flz.FLZ_PREC_FX64, flz.FLZ_PREC_DF64, flz.FLZ_PREC_FP64, flz.FLZ_PREC_FP32
    for beta, m, prec, rec, ortho, refine in ((-0.2, 200, X, F, O, 0), (-0.2, 200, S, F, O, 0),
                                              (-0.2, 200, H, F, O, 1), (-0.2, 200, D, C, O, 0),
                                              (0.0, 300, X, F, O, 0),
                                              (0.03, 400, X, F, O, 0), (0.03, 400, S, F, O, 0),
                                              (0.03, 400, H, F, O, 1), (0.03, 400, D, F, O, 0)):
        p = flz.flz_params_default()
        p.block_size = 4
        p.degree = m
        p.precision = prec
        p.recurrence = rec
        p.ortho = ortho
        p.check_every = 10
        p.refine = refine
        p.tol = 1e-8 if refine else args.tol
        s = flz.flz_solver_create(h, p)
        flz.flz_solver_set_interval(s, CONFIG3["alpha"], beta)
        flz.flz_solve(s, stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = flz.flz_solve(s, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        x = flz.flz_get_stats(s)
        res = flz.flz_get_residuals(s)
        rows.append({"interval": [CONFIG3["alpha"], beta], "m": m,
                     "precision": {0: "fp64", 1: "fp32 refined to 1e-8", 3: "df64", 4: "fx64"}[prec],
                     "recurrence": ["forward", "clenshaw"][rec], "ms_refine": x["ms_refine"],
                     "refine_sweeps": x["refine_sweeps"],
                     "ortho": ["auto", "cuda_cores", "tensor"][x["ortho"]], "status": flz.flz_status_string(st),
                     "count": int(x["count"]), "block_steps": int(x["iters"]), "seconds": e0.elapsed_time(e1) / 1e3,
                     "max_residual": float(res.max()) if res.size else None,
                     "eigenvalues_head": [float(v) for v in flz.flz_get_eigenvalues(s)[:3]],
                     "ms_filter": x["ms_filter"], "ms_orth": x["ms_orth"], "ms_check": x["ms_check"]})
        flz.flz_solver_destroy(s)
    flz.flz_matrix_destroy(h)
    print(json.dumps({"mode": "config3", "n": csr.n, "nnz": csr.nnz, "tol": args.tol, "rows": rows}))


def sequence_mode(flz, torch, prec, args):
    """A sequence of related problems (the self-consistent-field setting of
    the paper's Section 1): config 2's matrix with the potential moved by
    0.02 t (U(0,1) - 1/2) at steps t = 0..3, all eigenpairs in [0, beta] with
    the headline's beta. Each step is solved from a random start block (cold),
    by filtered Lanczos from combinations of the previous step's eigenvectors
    (krylov, flz_solver_set_start_vectors), and by filtered subspace iteration
    on them (subspace, params.start_mode SUBSPACE); each arm carries its own
    eigenvectors to its next step. All are timed (one solve each, CUDA events)
    and must return the same eigenvalues."""
    rng = np.random.Generator(np.random.PCG64(CONFIG2["seed"]))
    g = CONFIG2["grid"]
    v0 = CONFIG2["potential_scale"] * rng.random(g ** 3)
    dv = np.random.Generator(np.random.PCG64(CONFIG2["seed"] + 1)).random(g ** 3) - 0.5
    stream = torch.cuda.current_stream()
    arms = ("cold", "krylov", "subspace")
    rows, prev = [], {}
    for t in range(4):
        csr = laplacian_3d_7pt(g, g, g, v0 + 0.02 * t * dv)
        h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
        row, vals = {"step": t}, {}
        for mode in arms:
            if mode != "cold" and t == 0:
                continue
            p = flz.flz_params_default()
            p.block_size = args.block_size
            p.degree = args.degree
            p.check_every = args.check_every
            p.precision = prec
            p.tol = args.tol
            p.start_mode = flz.FLZ_START_SUBSPACE if mode == "subspace" else flz.FLZ_START_KRYLOV
            s = flz.flz_solver_create(h, p)
            flz.flz_solver_set_interval(s, CONFIG2["alpha"], CONFIG2["beta"])
            if mode != "cold":
                flz.flz_solver_set_start_vectors(s, prev[mode].T, ld=csr.n)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = flz.flz_solve(s, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            x = flz.flz_get_stats(s)
            vals[mode] = flz.flz_get_eigenvalues(s)
            row[mode] = {"status": flz.flz_status_string(st), "count": int(x["count"]), "block_steps": int(x["iters"]),
                         "matvecs": int(x["matvecs"] + x["sweep_matvecs"]), "sweeps": int(x["refine_sweeps"]),
                         "start_used": int(x["start_used"]), "seconds": e0.elapsed_time(e1) / 1e3,
                         "max_residual": float(flz.flz_get_residuals(s).max())}
            nxt = torch.empty((int(x["count"]), csr.n), dtype=torch.float64, device="cuda")
            flz.lib().flz_get_eigenvectors(s, nxt.data_ptr(), csr.n, int(x["count"]), flz.FLZ_DEVICE)
            if t == 0:
                for a in arms:
                    prev[a] = nxt
            else:
                prev[mode] = nxt
            flz.flz_solver_destroy(s)
        for mode in arms[1:]:
            if mode in vals:
                a, b = vals["cold"], vals[mode]
                row["max_abs_eig_diff_%s_vs_cold" % mode] = float(np.max(np.abs(a - b))) if a.shape == b.shape else None
        flz.flz_matrix_destroy(h)
        rows.append(row)
    out = {"mode": "sequence", "workload": config_dict(make_matrix(), args)["workload"],
           "potential_step": "0.02 t (U(0,1) - 1/2), t = 0..3", "rows": rows}
    for mode in arms:
        out["block_steps_%s_steps_1_3" % mode] = sum(r[mode]["block_steps"] for r in rows[1:])
        out["matvecs_%s_steps_1_3" % mode] = sum(r[mode]["matvecs"] for r in rows[1:])
        out["seconds_%s_steps_1_3" % mode] = sum(r[mode]["seconds"] for r in rows[1:])
    print(json.dumps(out))


def ortho_mode(flz, torch, args):
    """Full reorthogonalization alone: classical Gram-Schmidt twice of an n x r
    block against a K-column orthonormal basis (on the 2^-62 grid), on the
    tensor cores and on the CUDA cores, each call checked for orthogonality and
    against the other path. The small case the kernel profiles are taken on
    (about 3 GB on the device for the defaults). Each flz_basis_orthogonalize
    call also builds the digit copy of the caller's basis, so its wall time is
    not the solver's per-step cost; the kernels' own times come from ncu."""
    n, K, r = args.ortho_n, args.ortho_basis, args.block_size
    nb = K // r
    g = torch.Generator(device="cuda").manual_seed(9)
    Q = torch.randn(n, nb * r, dtype=torch.float64, device="cuda", generator=g)
    for _ in range(2):  # CholeskyQR2 (matrix products on the GPU, the small Cholesky on the host)
        R = np.linalg.cholesky((Q.T @ Q).cpu().numpy()).T
        Q = Q @ torch.from_numpy(np.linalg.inv(R)).cuda()
    Q = torch.round(Q * 2.0**62) * 2.0**-62
    blocks = Q.reshape(n, nb, r).permute(1, 0, 2).contiguous()
    W0 = torch.randn(n, r, dtype=torch.float64, device="cuda", generator=g) + 30.0 * Q[:, :r]
    out = {}
    for name, method in (("tensor", flz.FLZ_ORTHO_TENSOR), ("cuda_cores", flz.FLZ_ORTHO_CUDA_CORES)):
        for _ in range(max(args.steps, 2)):
            W = W0.clone()
            C = torch.zeros(nb * r, r, dtype=torch.float64, device="cuda")
            flz.flz_basis_orthogonalize(n, nb, r, blocks, W, C, method)
        torch.cuda.synchronize()
        proj = (Q.T @ W) / torch.linalg.norm(W, dim=0)
        out[name] = {"max_rel_projection_after": float(proj.abs().max()), "W": W}
    diff = float((out["tensor"]["W"] - out["cuda_cores"]["W"]).abs().max() / W0.abs().max())
    print(json.dumps({"mode": "ortho", "n": n, "basis": nb * r, "r": r,
                      "digit_bytes_per_pass": 16 * n * nb * r, "fp64_bytes_per_pass": 8 * n * nb * r,
                      "tensor_max_rel_projection_after": out["tensor"]["max_rel_projection_after"],
                      "cuda_cores_max_rel_projection_after": out["cuda_cores"]["max_rel_projection_after"],
                      "max_rel_diff_tensor_vs_cuda_cores": diff}))


def filter_mode(flz, torch, csr, prec, args):
    """Times flz_filter_apply alone (p_m(Ahat) on an n x r block) with CUDA events per call."""
    r, m = args.block_size, args.degree
    h = flz.flz_matrix_create_csr(csr.n, csr.nnz, csr.rowptr, csr.col, csr.val)
    lmin, lmax = 0.0, 12.5
    c, e = 0.5 * (lmin + lmax), 0.5 * (lmax - lmin)
    coeffs = flz.flz_filter_coefficients(-1.0, (CONFIG2["beta"] - c) / e, m)
    rec = {"forward": flz.FLZ_REC_FORWARD, "clenshaw": flz.FLZ_REC_CLENSHAW}[args.recurrence]
    V = torch.from_numpy(random_normal_block(csr.n, r, 5)).cuda()
    W = torch.empty_like(V)
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        flz.flz_filter_apply(h, c, e, coeffs, m, r, V, W, prec, stream, rec)
    torch.cuda.synchronize()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    sampler.start()
    times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        flz.flz_filter_apply(h, c, e, coeffs, m, r, V, W, prec, stream, rec)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    flz.flz_matrix_destroy(h)
    launches = m + (0 if prec == flz.FLZ_PREC_FP64 else 1)
    ms = float(np.mean(times)) / m
    sizes = ELEMENT_BYTES[args.precision]
    nbytes = filter_bytes_per_launch(csr.n, csr.nnz, r, *sizes, recurrence=args.recurrence)
    hbm, src = peaks()
    print(json.dumps({"mode": "filter", "precision": args.precision, "recurrence": args.recurrence,
                      "n": csr.n, "nnz": csr.nnz, "r": r,
                      "degree": m, "launches_per_apply": launches, "ms_per_apply": float(np.mean(times)),
                      "ms_per_degree": ms, "algorithmic_bytes_per_degree": nbytes,
                      "gbs": nbytes / (ms * 1e-3) / 1e9, "hbm_peak_gbs": hbm, "hbm_frac": nbytes / (ms * 1e-3) / 1e9 / hbm,
                      "fp64_tflops": filter_flops_per_launch(csr.n, csr.nnz, r) / (ms * 1e-3) / 1e12,
                      "clocks": clocks}))


def e2e_leg(flz, torch, csr, p, alpha, beta, stream, args):
    """Same metric through the C ABI from pinned host buffers, copies included."""
    rp = torch.from_numpy(csr.rowptr).pin_memory()
    cl = torch.from_numpy(csr.col).pin_memory()
    vl = torch.from_numpy(csr.val).pin_memory()
    total, pairs, h2d, d2h = 0.0, 0, 0, 0
    out = None
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = flz.flz_matrix_create_csr(csr.n, csr.nnz, rp.data_ptr(), cl.data_ptr(), vl.data_ptr())
        s = flz.flz_solver_create(h, p)
        flz.flz_solver_set_interval(s, alpha, beta)
        flz.flz_solve(s, stream)
        cnt = flz.flz_get_count(s)
        vals = flz.flz_get_eigenvalues(s)
        res = flz.flz_get_residuals(s)
        if out is None or out.shape[0] < cnt:
            out = torch.empty((max(cnt, 1), csr.n), dtype=torch.float64).pin_memory()
        flz.flz_get_eigenvectors(s, out.data_ptr(), csr.n, out.shape[0], flz.FLZ_HOST)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        flz.flz_solver_destroy(s)
        flz.flz_matrix_destroy(h)
        if it >= args.warmup:
            total += dt
            pairs += int(np.sum(res <= 1e-8))
            h2d = 4 * (csr.n + 1) + 12 * csr.nnz
            d2h = 8 * cnt * csr.n + 16 * cnt
            del vals
    return {"value": pairs / total, "unit": "eigenpairs/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}


if __name__ == "__main__":
    main()
