"""Benchmark: the Chebyshev filter of ChASE (Alg. 4) in mixed precision on
one GB300, against the FP64 filter on the same GPU.

Workload (default, ``--workload filter``): N = 30000 complex128 Hermitian H
with a DFT-like spectrum (N/4 eigenvalues in [-2, 0], the rest 50 u^2 up to
50; FFT construction of Q diag(lambda) Q^H), block of nev + nex = 1200 + 300
columns.  One step = one ``chase_filter`` call of degree 20 on the whole
block with the split-BF16 tensor-core product (Eq. 7 recurrence, FP64
epilogue).  Beside the timed steps the line carries: the FP64 filter of the
same block (degree 2, timed, and extrapolated by FLOPs), one cold solve of
the same problem to residual <= 1e-10 ||H|| with the split filter and FP64
QR, Rayleigh-Ritz and residuals, the end-to-end rate through host buffers,
the roofline of the product kernel and the CPU oracle on a column subset.

``--workload sequence`` gives the correlated-sequence solves (N = 8000,
nev 400, nex 80, warm starts) with the FP64 solve of the same problem; the
other workloads are listed under ``--workload``.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead (a
bounded sample of the same workload on the host cores).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Filter TFLOP/s and s per solve at resid≤1e-10, mixed vs FP64; serve p50/p99"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 has no entry in the measured peaks: the measured bf16 figure times the
# nominal FP64 / BF16 dense ratio of GB300 (1.25 / 2250 TFLOP/s).
NOMINAL_FP64_OVER_BF16 = 1.25 / 2250.0
# The FP64 kernels form a complex product with three real products (the 3M /
# Gauss form): 6 executed real FLOPs per 8 algorithmic ones.
FP64_EXECUTED_PER_ALGORITHMIC = 6.0 / 8.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--n", type=int, default=None,
                   help="matrix order (default 30000 for filter/solve, 8000 otherwise)")
    p.add_argument("--nev", type=int, default=None)
    p.add_argument("--nex", type=int, default=None)
    p.add_argument("--tol", type=float, default=1e-10)
    p.add_argument("--seed", type=int, default=2024)
    p.add_argument("--precision", default="split",
                   choices=["split", "split_rr", "split_adapt", "fp64"],
                   help="split: split-BF16 filter; split_rr: also Rayleigh-Ritz's H Q on the "
                        "split product; fp64: FP64 throughout")
    p.add_argument("--workload", default="filter",
                   choices=["filter", "sequence", "serve", "batched", "batched-solve",
                            "degree-sweep", "side", "variants", "solve"],
                   help="filter: timed degree-m filter calls on one N = 30000 problem, split "
                        "vs FP64, plus one cold solve (default); sequence: timed solves of the "
                        "correlated N = 8000 sequence")
    p.add_argument("--filter-degree", type=int, default=20)
    p.add_argument("--deg-extra", type=int, default=None,
                   help="DEGEXTRA of Alg. 5 for the sequence workload (default: 6 with a "
                        "split filter, Table 1's 2 with --precision fp64)")
    p.add_argument("--sweep-degrees", default="6,10,14,18,22,26,30,34,40")
    p.add_argument("--batch-problems", type=int, default=512)
    p.add_argument("--batch-degrees", default="const", choices=["const", "mixed"],
                   help="const: every column at --filter-degree; mixed: seeded even degrees "
                        "in [2, 36] per column")
    p.add_argument("--batch-tile", type=int, default=-1)
    p.add_argument("--serve-requests", type=int, default=10)
    p.add_argument("--serve-rate", type=float, default=20.0)
    p.add_argument("--serve-slots", type=int, default=4)
    p.add_argument("--serve-cap-gb", type=float, default=150.0)
    p.add_argument("--serve-sizes", default="2048,4096,8192,16384")
    p.add_argument("--serve-policy", default="sjf", choices=["fifo", "sjf"],
                   help="admission order of waiting requests: arrival, or shortest job first "
                        "(default; on the serving trace p50 55 s against 125 s, p99 and "
                        "throughput unchanged)")
    p.add_argument("--serve-max-wait", type=float, default=None,
                   help="sjf: seconds after which a waiting request goes ahead of newer ones")
    p.add_argument("--no-fp64-compare", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample-seconds", type=float, default=20.0)
    p.add_argument("--no-solve", action="store_true",
                   help="filter workload: skip the cold solve")
    p.add_argument("--solve-deg-extra", type=int, default=None,
                   help="filter workload: DEGEXTRA of the cold solve")
    p.add_argument("--deg-max", type=int, default=None,
                   help="DEGMAX of Alg. 5 for the sequence, serve and batched-solve workloads "
                        "(default: 64 with a split filter, Table 1's 36 with FP64)")
    p.add_argument("--solve-deg-max", type=int, default=None,
                   help="filter workload: DEGMAX of the cold solve (default 64)")
    args = p.parse_args()
    big = args.workload in ("filter", "solve")
    if args.n is None:
        args.n = 30000 if big else 8000
    if args.nev is None:
        args.nev = 1200 if big else 400
    if args.nex is None:
        args.nex = 300 if big else 80
    return args


def build_library():
    """Build (or find current) libchase.so; returns what the build did, for
    the JSON line: whether nvcc compiled anything in this process and the
    digest of the sources the library was built from."""
    from paper_1805_10121_gb300 import build
    build.build()
    info = dict(build.last_build)
    prov = build.library_provenance()
    return {"nvcc_ran_in_this_process": bool(info["compiled"]) or bool(info["linked"]),
            "sources_sha256": info["sources_sha256"][:16],
            "library_built_on": prov.get("machine"), "library_built_at": prov.get("built_at"),
            "library_matches_sources": bool(prov.get("matches_tree"))}


BUILD_INFO = None


def emit(line):
    """Print the JSON line (with the build record of this process)."""
    if BUILD_INFO is not None:
        line["build"] = BUILD_INFO
    print(json.dumps(line), flush=True)


def combine_over_ranks(elapsed, flops, device):
    """Whole-job figures of replicas: the slowest rank's time and the FLOPs of
    all ranks (the identity without a process group)."""
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    f = torch.tensor([float(flops)], dtype=torch.float64, device=device)
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(f, op=dist.ReduceOp.SUM)
    return float(t.item()), float(f.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            pk = json.load(f)
        return pk, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def warm_eigensolver(dev, widths):
    from paper_1805_10121_gb300 import serve
    serve.warm_eigensolver(dev, widths)


class ClockSampler:
    """nvidia-smi sampling during the timed region (clocks and throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        out.update(sm_mhz=statistics.median(sm) if sm else None,
                   sm_max_mhz=max(mx) if mx else None, reasons=reasons, samples=len(rows))
        return out


def make_sequence(n, count, seed, device):
    """H_1 .. H_count on the device (column-major complex128)."""
    from paper_1805_10121_gb300 import synth
    lam = synth.spectrum_dft(n, seed, device=device)
    q = synth.unitary_dft(n, seed + 1, device=device)
    H = synth.hermitian_from(q, lam)
    del q
    hnorm = float(lam.abs().max())
    seq = [H]
    for k in range(1, count):
        E = synth.hermitian_noise(n, seed + 100 + k, device=device)
        Hn = (seq[-1] + (1e-3 * hnorm) * E).t().contiguous().t()
        del E
        seq.append(Hn)
    return seq, lam, hnorm


def prec_code(name):
    from paper_1805_10121_gb300 import chase
    return {"split": chase.CHASE_SPLIT_BF16, "split_rr": chase.CHASE_SPLIT_BF16_RR,
            "split_adapt": chase.CHASE_SPLIT_BF16_ADAPT, "fp64": chase.CHASE_FP64}[name]


# Slice-pair products the split-BF16 kernel executes per FP64-equivalent
# product: pairs (s, t) of 7 slices with s + t <= 6.
SPLIT_PAIRS = 28


# DRAM traffic of single launches of other shapes, measured with ncu: the
# sequence workload's own launches (N = 8000, 480 columns; the FP64 H Q on
# its 64 x 16 tile) have no capture, so its "traffic" stays null and these
# figures ride along as context.
NCU_TRAFFIC = {
    "zgemm_split_kernel": {"case": "N=8000, 1500 complex columns, full-width degree step of the "
                                   "persistent kernel (the sequence workload's blocks are narrower)",
                           "dram_bytes": 12.25e9 + 0.191e9, "algorithmic_bytes": 2.656e9},
    "zgemm_tma_kernel": {"case": "N=4000, 64 columns, first product of a degree-2 FP64 filter on "
                                 "the 64 x 32 tile that the host picks there (the N=8000 "
                                 "Rayleigh-Ritz H Q of 480 columns takes 64 x 16)",
                         "dram_bytes": 263.4e6 + 3.4e6, "algorithmic_bytes": 264e6},
}


def _split_filter_roofline(stats_list, pk, src):
    flops = sum(s["flops_filter"] for s in stats_list)
    secs = sum(s["t_filter"] for s in stats_list)
    fp64_equiv = flops / secs / 1e12 if secs > 0 else 0.0
    # BF16 tensor work the algorithm executes: 28 slice products, each a real
    # GEMM of 8 N^2 b FLOPs per b complex columns.  The kernel runs inside a
    # multi-second solve: sustained bf16 peak.
    achieved = SPLIT_PAIRS * fp64_equiv
    peak = pk.get("bf16_tflops_sustained", 1700.0)
    return {
        "bound": "tensor",
        "kernel": "zgemm_split_kernel (tcgen05 BF16 slice products, exact level sums, "
                  "fused recurrence epilogue): the filter steps",
        "achieved": round(achieved, 2),
        "peak": round(peak, 1),
        "unit": "TFLOP/s",
        "frac": round(achieved / peak, 4),
        "traffic": None,
        "peak_source": f"{src} bf16_tflops_sustained",
        "fp64_equivalent_tflops": round(fp64_equiv, 3),
        "timing": "filter phase (product launches and the slicing of the block), CUDA events "
                  "on the solve's stream",
        "traffic_ncu_small_case": NCU_TRAFFIC["zgemm_split_kernel"],
    }


def _fp64_roofline(flops, secs, pk, src, what):
    # The FP64 products draw little power and run at the maximum SM clock
    # (sampled below), so the burst figure is the applicable one.
    alg = flops / secs / 1e12 if secs > 0 else 0.0
    peak = pk.get("bf16_tflops", 1900.0) * NOMINAL_FP64_OVER_BF16
    executed = FP64_EXECUTED_PER_ALGORITHMIC * alg
    return {
        "bound": "tensor",
        "kernel": f"zgemm_tma_kernel (FP64 DMMA, 3M complex form): {what}",
        "achieved": round(executed, 4),
        "peak": round(peak, 4),
        "unit": "TFLOP/s",
        "frac": round(executed / peak, 4),
        "traffic": None,
        "peak_source": f"{src} bf16_tflops (burst) x nominal FP64/BF16 ratio (1.25/2250); "
                       "a DMMA-only probe kernel measured 1.05 TFLOP/s on GB300",
        "achieved_counts": "executed DMMA FLOPs (3M form: 6 per 8 algorithmic)",
        "algorithmic_tflops": round(alg, 4),
        "traffic_ncu_small_case": NCU_TRAFFIC["zgemm_tma_kernel"],
    }


def roofline_entry(stats_list, pk, src, precision):
    """(dominant kernel's roofline, the other hot kernel's) for a solve."""
    if precision == "fp64":
        flops = sum(s["flops_filter"] for s in stats_list)
        secs = sum(s["t_filter"] for s in stats_list)
        return _fp64_roofline(flops, secs, pk, src, "the filter steps"), None
    filt = _split_filter_roofline(stats_list, pk, src)
    rr_fl = sum(s["flops_rr_product"] for s in stats_list)
    rr_t = sum(s["t_rr_product"] for s in stats_list)
    if precision == "split_rr":
        rr = {"kernel": "zgemm_split_kernel: Rayleigh-Ritz H Q",
              "fp64_equivalent_tflops": round(rr_fl / rr_t / 1e12, 3) if rr_t > 0 else None,
              "seconds": round(rr_t, 3)}
        return filt, rr
    # split: Rayleigh-Ritz's H Q stays FP64 and takes more device time than
    # the filter (ncu launch list), so it is the dominant kernel
    rr = _fp64_roofline(rr_fl, rr_t, pk, src, "Rayleigh-Ritz H Q (FP64 by specification)")
    rr["timing"] = "H Q products, CUDA events on the solve's stream"
    if rr_t >= sum(s["t_filter"] for s in stats_list):
        return rr, filt
    return filt, rr


def lanczos_entry(stats_list, n, pk, src):
    """Rate of the Lanczos phase (Alg. 6): its matvecs run on the few-column
    product (one vector per step after a warm start), which reads H once per
    step and is bound by the FP64 FMA pipe (2 FLOP/byte against a machine
    balance of 0.15)."""
    mv = sum(s.get("lanczos_matvecs", 0) for s in stats_list)
    t = sum(s["t_lanczos"] for s in stats_list)
    if mv <= 0 or t <= 0:
        return None
    flops = 8.0 * n * n * mv
    hbm_bytes = 16.0 * n * n * mv  # warm-started solves: one vector per step
    peak = pk.get("bf16_tflops", 1900.0) * NOMINAL_FP64_OVER_BF16
    tf = flops / t / 1e12
    return {
        "kernel": "fewcol_kernel (FP64 FMA on the CUDA cores): the Lanczos matvecs",
        "bound": "fp64",
        "matvecs": int(mv),
        "seconds": round(t, 4),
        "achieved": round(tf, 4),
        "peak": round(peak, 4),
        "unit": "TFLOP/s",
        "frac": round(tf / peak, 4),
        "hbm_gbs": round(hbm_bytes / t / 1e9, 1),
        "hbm_frac": round(hbm_bytes / t / 1e9 / pk.get("hbm_gbs", 6800.0), 4),
        "timing": "whole Lanczos phase (matvecs, three-term steps, host tridiagonal "
                  "eigensolves), CUDA events on the solve's stream",
        "peak_source": f"{src} bf16_tflops x nominal FP64/BF16 ratio (1.25/2250)",
    }


# DEGEXTRA of Alg. 5 (Table 1: 2).  With the split filter a column product
# costs about 1/36 of the FP64 work per FLOP that Rayleigh-Ritz and QR do, so
# slightly higher degrees, which lock columns sooner and leave smaller
# blocks for the FP64 steps, pay off: N = 8000 sequence, 2.60 s per solve
# with 2, 2.47 s with 6, 2.49 s with 12 (measured).  The FP64 path keeps 2.
SPLIT_DEG_EXTRA = 6
# The cold N = 30000 solve of the filter workload (nev 1200, nex 300): 195 s
# and 18 iterations with DEGEXTRA 2, 165 s / 14 with 6, 155 s / 13 with 10
# (measured; Rayleigh-Ritz's FP64 H Q, about 5.6 s per iteration there,
# is what fewer iterations save).
COLD_SOLVE_DEG_EXTRA = 10
# DEGMAX of Alg. 5 (Table 1: 36) for solves with the split filter.  Higher
# caps let far-from-converged columns take the degree that converges them in
# one more iteration; each saved iteration saves an FP64 Rayleigh-Ritz and QR
# (measured: N = 8000 sequence 2.47 s / 9 iterations per warm solve with 36,
# 1.94 s / 6 with 64, 1.71 s / 4-5 with 96; cold N = 30000 solve 160 s / 13
# with 36, 139 s / 10 with 48, 135 s / 9 with 64, 129 s / 7 with 96; the
# 512-problem batched solve 10.1 s with 36, 9.9 s with 64).  The cap also
# guards rank deficiency of the filtered block (Sec. 4.1.3): at 96 the
# batched solve's Cholesky QR needed its shifted retries (QR 6.5 s against
# 1.1 s) and at 128 it broke down, so the split path takes 64 and the FP64
# path keeps Table 1's 36.
SPLIT_DEG_MAX = 64


def deg_max_for(args, precision_code):
    """DEGMAX of Alg. 5 for a workload's solves: --deg-max, else SPLIT_DEG_MAX
    with a split filter and the library's default (Table 1) with FP64."""
    from paper_1805_10121_gb300 import chase
    if getattr(args, "deg_max", None) is not None:
        return int(args.deg_max)
    if precision_code == chase.CHASE_FP64:
        return int(chase.chase_opts_default().deg_max)
    return SPLIT_DEG_MAX


def deg_extra_for(args, precision_code):
    from paper_1805_10121_gb300 import chase
    if getattr(args, "deg_extra", None) is not None:
        return args.deg_extra
    return 2 if precision_code == chase.CHASE_FP64 else SPLIT_DEG_EXTRA


def workload_config(args, world):
    n, nev, nex, tol = args.n, args.nev, args.nex, args.tol
    return {
        "workload": f"sequence of correlated problems, N={n} complex128, nev={nev}, "
                    f"nex={nex}, tol={tol} x ||H||, warm start; step = one solve",
        "n": n, "nev": nev, "nex": nex, "tol": tol, "precision": args.precision,
        "l2": f"inputs larger than L2 (H = {n * n * 16 / 1e9:.2f} GB per problem)",
        "parallelism": "replicas" if world > 1 else "single GPU",
    }


class OracleSample:
    """A bounded sample of the workload for the CPU oracle: one degree-2
    filter of the full N x (nev+nex) block of problem 1, its Householder QR
    and the Rayleigh quotient (the dense products that dominate a solve).
    Inputs come from the same seeded generators on the host (the host and
    device random streams differ, the shapes and distributions do not)."""

    def __init__(self, n, nev, nex, seed):
        import oracle
        from paper_1805_10121_gb300 import synth
        self.oracle = oracle
        nx = nev + nex
        lam = synth.spectrum_dft(n, seed)
        q = synth.unitary_dft(n, seed + 1)
        self.H = synth.hermitian_from(q, lam).numpy()
        del q
        self.V = synth.gaussian_block(n, nx, seed + 7).numpy()
        self.l = lam.numpy()
        self.n, self.nx = n, nx
        self.flops = 2 * 8.0 * n * n * nx + 8.0 * n * n * nx + 8.0 * n * nx * nx + 16.0 * n * nx * nx

    def step(self):
        o = self.oracle
        W = o.cheb_filter(self.H, self.V, [2] * self.nx, 50.5, float(self.l[0]),
                          float(self.l[self.nx]))
        Q, _ = o.householder_qr(W)
        G = Q.conj().T @ (self.H @ Q)
        return G

    def describe(self, reps):
        return (f"{reps} x [degree-2 filter + Householder QR + Rayleigh quotient] on the "
                f"N={self.n} x {self.nx} block of problem 1, NumPy (BLAS threads = all host cores)")


def cpu_baseline_sample(n, nev, nex, seed, budget_s):
    smp = OracleSample(n, nev, nex, seed)
    t0 = time.perf_counter()
    reps = 0
    while True:
        smp.step()
        reps += 1
        if time.perf_counter() - t0 > budget_s or reps >= 3:
            break
    dt = time.perf_counter() - t0
    return {
        "value": round(smp.flops * reps / dt / 1e12, 6),
        "unit": "TFLOP/s",
        "cores": os.cpu_count(),
        "kind": "oracle",
        "sample": smp.describe(reps),
        "seconds": round(dt, 2),
    }


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle as it stands, W untimed and K timed
    bounded samples of the workload (rank 0 only).  Filter workload: each
    step is the oracle's Alg. 4 of the workload's degree on 8 columns of the
    N x (nev + nex) block (inputs from the same seeded generators on the
    host).  Sequence workload: a degree-2 filter of the whole block, its
    Householder QR and the Rayleigh quotient."""
    if rank != 0:
        return
    if args.workload == "filter":
        from paper_1805_10121_gb300 import synth
        lam = synth.spectrum_dft(args.n, args.seed)
        H = synth.hermitian_dft(lam, args.seed + 1).numpy()
        V = synth.gaussian_block(args.n, 8, args.seed + 7).numpy()
        smp = OracleFilterSample(H, V, lam.numpy(), args.nev + args.nex, args.filter_degree)
        step, flops, describe = smp.step, smp.flops(), smp.describe
        cfg = filter_workload_config(args, world)
        cfg["precision"] = "fp64 (CPU oracle)"
    else:
        smp = OracleSample(args.n, args.nev, args.nex, args.seed)
        step, flops, describe = smp.step, smp.flops, smp.describe
        cfg = workload_config(args, world)
        cfg["precision"] = "fp64 (CPU oracle)"
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = flops * args.steps / dt / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * dt / args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": round(value, 6), "unit": "TFLOP/s", "cores": os.cpu_count(),
                         "kind": "oracle", "sample": describe(args.steps)},
        "e2e": {"value": round(value, 6), "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


class BlasThreads:
    """Set the BLAS thread count of NumPy's bundled OpenBLAS for a region
    (for the one-thread oracle figure).  ``ok`` is False when the library or
    its thread call cannot be found; the region then runs unchanged."""

    def __init__(self, n):
        self.n = n
        self.ok = False
        self.prev = None
        self.set_fn = self.get_fn = None
        import ctypes
        try:
            with open("/proc/self/maps") as f:
                paths = sorted({ln.split()[-1] for ln in f
                                if "openblas" in ln.lower() and ".so" in ln})
        except OSError:
            paths = []
        for path in paths:
            try:
                lib = ctypes.CDLL(path)
            except OSError:
                continue
            for suffix in ("scipy_openblas_set_num_threads64_", "openblas_set_num_threads64_",
                           "openblas_set_num_threads"):
                if hasattr(lib, suffix):
                    self.set_fn = getattr(lib, suffix)
                    get = suffix.replace("set_num", "get_num")
                    self.get_fn = getattr(lib, get) if hasattr(lib, get) else None
                    self.ok = True
                    return

    def __enter__(self):
        if self.ok:
            self.prev = int(self.get_fn()) if self.get_fn else os.cpu_count()
            self.set_fn(int(self.n))
        return self

    def __exit__(self, *exc):
        if self.ok:
            self.set_fn(int(self.prev))
        return False


class OracleFilterSample:
    """A bounded sample of the filter workload for the CPU oracle: Alg. 4 of
    the given degree on a subset of the block's columns (the oracle's
    ``cheb_filter``, NumPy BLAS products with H).  ``H`` is a host array
    (column-major complex128) of the workload's matrix."""

    def __init__(self, H, V, l, nx, degree):
        import oracle
        self.oracle = oracle
        self.H, self.V = H, V
        self.n = H.shape[0]
        self.cols = V.shape[1]
        self.degree = degree
        self.b_sup, self.mu1, self.mu_nn = 1.01 * float(l[-1]), float(l[0]), float(l[nx])

    def flops(self, degree=None):
        return 8.0 * self.n * self.n * self.cols * (degree or self.degree)

    def step(self, degree=None):
        d = degree or self.degree
        return self.oracle.cheb_filter(self.H, self.V, [d] * self.cols, self.b_sup, self.mu1,
                                       self.mu_nn)

    def describe(self, reps, threads="all host cores", degree=None):
        return (f"{reps} x oracle Alg. 4 filter of degree {degree or self.degree} on {self.cols} "
                f"of the columns of the N={self.n} block (NumPy, BLAS threads = {threads})")


def filter_cpu_baseline(smp, budget_s):
    """The oracle sample timed on the host cores: repeated until budget_s is
    spent (at least once), then a short one-thread figure."""
    t0 = time.perf_counter()
    reps = 0
    while True:
        smp.step()
        reps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    out = {"value": round(smp.flops() * reps / dt / 1e12, 6), "unit": "TFLOP/s",
           "cores": os.cpu_count(), "kind": "oracle", "sample": smp.describe(reps),
           "seconds": round(dt, 2)}
    one = {"value": None, "note": "BLAS thread control not found"}
    bt = BlasThreads(1)
    if bt.ok:
        with bt:
            t1 = time.perf_counter()
            smp.step(degree=2)
            d1 = time.perf_counter() - t1
        one = {"value": round(smp.flops(degree=2) / d1 / 1e12, 6), "unit": "TFLOP/s",
               "cores": 1, "sample": smp.describe(1, threads="1", degree=2),
               "seconds": round(d1, 2)}
    out["one_thread"] = one
    return out


def filter_workload_config(args, world):
    n, nx, m = args.n, args.nev + args.nex, args.filter_degree
    return {
        "workload": (f"mixed-precision Chebyshev filter, N={n} complex128 (FFT construction of "
                     f"Q diag(lambda) Q^H, DFT-like spectrum), block of nev+nex={args.nev}+"
                     f"{args.nex} columns, degree {m} for every column; step = one chase_filter "
                     f"call (Alg. 4) with the split-BF16 tensor-core product"),
        "n": n, "nev": args.nev, "nex": args.nex, "degree": m, "precision": "split",
        "l2": (f"inputs larger than L2 (H {16 * n * n / 1e9:.1f} GB, its BF16 slices "
               f"{28 * n * n / 1e9:.1f} GB, block {16 * n * nx / 1e9:.2f} GB)"),
        "parallelism": "replicas" if world > 1 else "single GPU",
    }


# DRAM traffic of one zgemm_split_kernel launch of the default filter
# workload (one of its four K segments: 30000 rows of H, 1500 complex
# columns, K = 15000), measured with ncu on the persistent-CTA kernel
# (dram__bytes_read.sum 58.80 GB + dram__bytes_write.sum 0.72 GB, one
# pass, --clock-control none; the command is in the profile of this
# kernel).  Set back to None whenever the kernel or its launch shape
# changes.
SPLIT_N30000_TRAFFIC = 58.80e9 + 0.72087e9


def split_algorithmic_bytes(n, ncols, k_per_launch):
    """Bytes one split product launch must move at least: the 7 slice planes
    of H and of the block over its K range, once, and the FP64 result
    (a K-segment partial product, N x ncols complex)."""
    return 7 * 2.0 * (n + 2 * ncols) * k_per_launch + 16.0 * n * ncols


def run_filter_workload(args, rank, world, local):
    """The mixed-precision filter configuration (default)."""
    from paper_1805_10121_gb300 import build, chase, synth
    build.build()
    chase.lib()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    n, nev, nex, m = args.n, args.nev, args.nex, args.filter_degree
    nx = nev + nex
    W, K = args.warmup, args.steps
    seed = args.seed + 1000 * rank
    lam = synth.spectrum_dft(n, seed, device=dev)
    H = synth.hermitian_dft(lam, seed + 1)
    V0 = synth.gaussian_block(n, nx, seed + 7, device=dev)
    l = lam.cpu().numpy()
    hnorm = float(np.abs(l).max())
    b_sup, mu1, mu_nn = 1.01 * float(l[-1]), float(l[0]), float(l[nx])
    degs = torch.full((nx,), m, dtype=torch.int32)
    stream = torch.cuda.current_stream(dev)
    split = chase.CHASE_SPLIT_BF16

    V = V0.clone()
    for _ in range(W):
        chase.chase_filter(H, V, degs, b_sup, mu1, mu_nn, precision=split)
    torch.cuda.synchronize()
    # ---------------- timed region ----------------
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = chase.chase_kernel_launches()
    chase.chase_kernel_timing(True)
    clocks.start()
    e0.record(stream)
    for _ in range(K):
        chase.chase_filter(H, V, degs, b_sup, mu1, mu_nn, precision=split)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    chase.chase_kernel_timing(False)
    if world > 1:
        torch.distributed.barrier()
    launches = chase.chase_kernel_launches() - launches0
    kt = chase.chase_kernel_timing_read(chase.CHASE_TIMED_SPLIT_PRODUCT)
    elapsed = e0.elapsed_time(e1) / 1e3
    flops_step = 8.0 * n * n * nx * m
    t_max, total_flops = combine_over_ranks(elapsed, flops_step * K, dev)
    value = total_flops / t_max / 1e12
    pk, src = peaks()

    # roofline of the product kernel, from its own launches in the timed region
    peak = pk.get("bf16_tflops_sustained", 1700.0)
    per_launch_s = kt["seconds"] / max(kt["launches"], 1)
    tensor_per_launch = kt["tensor_flops"] / max(kt["launches"], 1)
    achieved = tensor_per_launch / per_launch_s / 1e12 if per_launch_s > 0 else 0.0
    launches_per_product = kt["launches"] / max(K * m, 1)
    k_per_launch = 2.0 * n / launches_per_product
    alg_bytes = split_algorithmic_bytes(n, nx, k_per_launch)
    roof = {
        "bound": "tensor",
        "kernel": "zgemm_split_kernel (tcgen05 BF16 slice products, exact int32 level sums, "
                  "FP64 recurrence epilogue)",
        "achieved": round(achieved, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
        "frac": round(achieved / peak, 4),
        "traffic": SPLIT_N30000_TRAFFIC if (n == 30000 and nx == 1500) else None,
        "peak_source": f"{src} bf16_tflops_sustained (a kernel inside a multi-second loop)",
        "achieved_counts": "BF16 tensor FLOPs the kernel executes: 28 slice-pair products of "
                           "8 N^2 per complex column",
        "fp64_equivalent_tflops": round(kt["flops"] / kt["seconds"] / 1e12, 3)
        if kt["seconds"] > 0 else None,
        "launches": kt["launches"], "avg_launch_ms": round(1e3 * per_launch_s, 3),
        "algorithmic_bytes_per_launch": alg_bytes,
        "traffic_over_algorithmic": round(SPLIT_N30000_TRAFFIC / alg_bytes, 2)
        if SPLIT_N30000_TRAFFIC and n == 30000 and nx == 1500 else None,
        "timing": "CUDA events recorded by the library on the launching stream around the "
                  "product launches of the timed steps (chase_kernel_timing)",
    }

    # ---------------- FP64 filter of the same block ----------------
    fp64 = None
    if not args.no_fp64_compare:
        Vw = V0[:, :64].clone()
        chase.chase_filter(H, Vw, torch.full((64,), 2, dtype=torch.int32), b_sup, mu1, mu_nn,
                           precision=chase.CHASE_FP64)  # warm-up of the FP64 kernels
        del Vw
        V64 = V0.clone()
        torch.cuda.synchronize()
        chase.chase_kernel_timing(True)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        chase.chase_filter(H, V64, torch.full((nx,), 2, dtype=torch.int32), b_sup, mu1, mu_nn,
                           precision=chase.CHASE_FP64)
        c1.record(stream)
        torch.cuda.synchronize()
        chase.chase_kernel_timing(False)
        k64 = chase.chase_kernel_timing_read(chase.CHASE_TIMED_FP64_PRODUCT)
        t64 = c0.elapsed_time(c1) / 1e3
        fl64 = 8.0 * n * n * nx * 2
        fp64_peak = pk.get("bf16_tflops", 1900.0) * NOMINAL_FP64_OVER_BF16
        ex = k64["tensor_flops"] / k64["seconds"] / 1e12 if k64["seconds"] > 0 else 0.0
        fp64 = {"filter_tflops": round(fl64 / t64 / 1e12, 4),
                "seconds_degree2": round(t64, 3),
                "seconds_same_filter_extrapolated": round(t64 * m / 2.0, 1),
                "speedup_split_vs_fp64_filter": round((flops_step * K / elapsed) / (fl64 / t64), 2),
                "roofline": {"bound": "tensor",
                             "kernel": "zgemm_tma_kernel (FP64 DMMA, 3M complex form)",
                             "achieved": round(ex, 4), "peak": round(fp64_peak, 4),
                             "unit": "TFLOP/s", "frac": round(ex / fp64_peak, 4),
                             "achieved_counts": "executed DMMA FLOPs (6 of 8 algorithmic)",
                             "peak_source": f"{src} bf16_tflops (burst) x nominal FP64/BF16 "
                                            "ratio (1.25/2250)"}}
        del V64

    # ---------------- end to end through host buffers ----------------
    e2e = None
    Hh = None
    if not args.no_e2e:
        Hh = torch.empty((n, n), dtype=torch.complex128, pin_memory=True).t()
        Hh.copy_(H)
        Vh = torch.empty((nx, n), dtype=torch.complex128, pin_memory=True).t()
        reps = max(1, min(K, 3))
        chase.chase_filter(Hh, Vh.copy_(V0), degs, b_sup, mu1, mu_nn, precision=split)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            chase.chase_filter(Hh, Vh, degs, b_sup, mu1, mu_nn, precision=split)
        torch.cuda.synchronize()
        te = (time.perf_counter() - t0) / reps
        e2e = {"value": round(flops_step / te / 1e12, 4), "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(16 * n * n + 16 * n * nx),
               "d2h_bytes_per_step": int(16 * n * nx), "seconds": round(te, 3),
               "steps": reps,
               "how": "chase_filter with pinned host H and V: the library copies both in, "
                      "filters, and copies V out, all inside the timed call"}
        del Vh

    # ---------------- one cold solve of the same problem ----------------
    solve = None
    if not args.no_solve:
        de = args.solve_deg_extra if args.solve_deg_extra is not None else COLD_SOLVE_DEG_EXTRA
        warm_eigensolver(dev, [nx])
        Vs = synth.gaussian_block(n, nx, seed + 11, device=dev)
        S = synth.gaussian_block(n, 5, seed + 8, device=dev)
        o = chase.chase_opts_default(precision=split, deg_extra=de)
        o.deg_max = int(args.solve_deg_max) if args.solve_deg_max is not None else SPLIT_DEG_MAX
        chase.chase_kernel_timing(True)
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        st, ritz, res, ss = chase.chase_solve(H, nev, nex, args.tol, Vs, S, opts=o)
        s1.record(stream)
        torch.cuda.synchronize()
        chase.chase_kernel_timing(False)
        ts = s0.elapsed_time(s1) / 1e3
        k64s = chase.chase_kernel_timing_read(chase.CHASE_TIMED_FP64_PRODUCT)
        # The FP64 solve takes the same iterations (every step but the filter
        # product is the same FP64 code); its time is this solve's time with
        # the filter replaced by the same FLOPs at the measured FP64 filter rate.
        fp64_model = None
        if fp64 is not None:
            t_f64 = ss["flops_filter"] / (fp64["filter_tflops"] * 1e12)
            fp64_model = {"seconds": round(ts - ss["t_filter"] + t_f64, 1),
                          "speedup_split_vs_fp64": round((ts - ss["t_filter"] + t_f64) / ts, 2),
                          "how": "split solve time - its filter time + its filter FLOPs at the "
                                 "FP64 filter rate measured above (same iterations: every other "
                                 "step is the same FP64 code)"}
        solve = {"status": st, "seconds": round(ts, 2), "iterations": ss["iterations"],
                 "deg_extra": de, "deg_max": int(o.deg_max),
                 "resid_max_over_norm": float(np.max(res[:nev])) / hnorm,
                 "eig_err_max_over_norm": float(np.max(np.abs(ritz[:nev] - l[:nev]))) / hnorm,
                 "phase_seconds": {k2: round(ss[k2], 2) for k2 in
                                   ("t_lanczos", "t_filter", "t_qr", "t_rr", "t_eigh",
                                    "t_rr_product")},
                 "filter_tflops": round(ss["flops_filter"] / max(ss["t_filter"], 1e-12) / 1e12, 2),
                 "rr_columns_total": int(round(ss["flops_rr_product"] / (8.0 * n * n))),
                 "rr_fp64_product_tflops": round(k64s["flops"] / k64s["seconds"] / 1e12, 4)
                 if k64s["seconds"] > 0 else None,
                 "fp64_solve_modelled": fp64_model}
        del Vs, S

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    cb = None
    if not args.no_cpu_baseline and world == 1:
        if Hh is None:
            Hh = H.cpu()
        smp = OracleFilterSample(Hh.numpy(), V0[:, :8].cpu().numpy(), l, nx, m)
        cb = filter_cpu_baseline(smp, args.cpu_sample_seconds)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "TFLOP/s", "n_gpus": world,
        "steps": K, "warmup": W, "ms_per_step": round(1e3 * t_max / K, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16-split+f64", "data": "synthetic",
        "config": filter_workload_config(args, world),
        "roofline": roof,
        "fp64_filter": fp64,
        "solve": solve,
        "cpu_baseline": cb,
        "e2e": e2e,
        "gpu_launches": int(launches), "clocks": clk,
    }
    emit(line)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batched_workload(args, rank, world, local):
    """Many independent problems (N uniform in [256, 2048], nev = 5% N,
    nex = 2% N, eigenvalues uniform in [-1, 1]): one step = one grouped
    filter call over the whole batch (one launch per degree step, captured
    in a CUDA graph).  Both precisions are timed on the same batch."""
    from paper_1805_10121_gb300 import build, chase, synth
    build.build()
    chase.lib()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P = args.batch_problems
    seed = args.seed + 1000 * rank
    shapes = synth.batched_shapes(P, seed)
    rng = np.random.default_rng(seed + 5)
    Hs, V0s, degs, bs, m1, mn = [], [], [], [], [], []
    for k, (n, nev, nex) in enumerate(shapes):
        nx = nev + nex
        lam = synth.spectrum_uniform(n, seed + 10 * k, device=dev)
        Hs.append(synth.hermitian_dft(lam, seed + 10 * k + 1))
        V0s.append(synth.gaussian_block(n, nx, seed + 10 * k + 2, device=dev))
        if args.batch_degrees == "const":
            degs.append(np.full(nx, args.filter_degree, dtype=np.int32))
        else:
            degs.append((2 * rng.integers(1, 19, size=nx)).astype(np.int32))
        l = lam.cpu().numpy()
        bs.append(1.01)
        m1.append(float(l[0]))
        mn.append(float(l[nx]))
    stream = torch.cuda.current_stream(dev)
    h_bytes = sum(16 * n * n for n, _, _ in shapes)
    v_bytes = sum(16 * n * (nev + nex) for n, nev, nex in shapes)

    def timed(prec, reps, warm):
        Vs = [v.clone() for v in V0s]
        for _ in range(warm):
            chase.chase_filter_batched(Hs, Vs, degs, bs, m1, mn, precision=prec,
                                       tile=args.batch_tile)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        clocks = ClockSampler(local)
        clocks.start()
        launches0 = chase.chase_kernel_launches()
        st = []
        a.record(stream)
        for _ in range(reps):
            st.append(chase.chase_filter_batched(Hs, Vs, degs, bs, m1, mn, precision=prec,
                                                 tile=args.batch_tile))
        b.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        return (a.elapsed_time(b) / 1e3 / reps, st, clk,
                chase.chase_kernel_launches() - launches0)

    split = args.precision != "fp64"
    prec = chase.CHASE_SPLIT_BF16 if split else chase.CHASE_FP64
    t_main, st_main, clk, launches = timed(prec, args.steps, args.warmup)
    flops = st_main[0]["flops"]
    value = flops / t_main / 1e12
    t_steps = statistics.mean(s["t_steps"] for s in st_main)
    # product launches timed by events inside the graph; the whole graph if
    # the driver gave no time for them
    t_prod = statistics.mean(s["t_product"] for s in st_main) or t_steps
    pk, src = peaks()
    other = None
    if not args.no_fp64_compare:
        t_o, st_o, _, _ = timed(chase.CHASE_FP64 if split else chase.CHASE_SPLIT_BF16, 1, 1)
        other = {"precision": "fp64" if split else "split",
                 "tflops": round(flops / t_o / 1e12, 4), "seconds": round(t_o, 3),
                 "product_seconds": round(st_o[0]["t_product"], 3),
                 "tile_config": st_o[0]["tile_config"]}
    if split:
        achieved = SPLIT_PAIRS * flops / t_prod / 1e12
        peak = pk.get("bf16_tflops_sustained", 1700.0)
        roof = {"bound": "tensor",
                "kernel": "zgemm_split_grouped_kernel (tcgen05 BF16 slice products over all "
                          "problems of a degree step)",
                "achieved": round(achieved, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "peak_source": f"{src} bf16_tflops_sustained",
                "fp64_equivalent_tflops": round(flops / t_prod / 1e12, 3)}
        # slice planes of H (28 N^2 bytes) stream from HBM once per degree step
        hbm = sum(28.0 * n * n for n, _, _ in shapes) * st_main[0]["steps"] / t_prod / 1e9
        roof["hbm_gbs_slices_of_h"] = round(hbm, 1)
        roof["hbm_frac"] = round(hbm / pk.get("hbm_gbs", 6800.0), 4)
    else:
        peak = pk.get("bf16_tflops", 1900.0) * NOMINAL_FP64_OVER_BF16
        achieved = FP64_EXECUTED_PER_ALGORITHMIC * flops / t_prod / 1e12
        roof = {"bound": "tensor",
                "kernel": "zgemm_grouped_kernel (FP64 DMMA 3M form, all problems of a degree "
                          "step)",
                "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "peak_source": f"{src} bf16_tflops (burst) x nominal FP64/BF16 ratio",
                "achieved_counts": "executed DMMA FLOPs (3M form: 6 per 8 algorithmic)",
                "algorithmic_tflops": round(flops / t_prod / 1e12, 4)}
    e2e = None
    if not args.no_e2e:
        # host buffers in pinned memory; copies in and out inside the timed region
        Hh = [h.cpu().pin_memory() for h in Hs]
        Vh = [v.cpu().pin_memory() for v in V0s]
        Hd = [torch.empty_like(h) for h in Hs]
        Vd = [torch.empty_like(v) for v in V0s]
        Vo = [torch.empty_like(v).pin_memory() for v in Vh]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(P):
            Hd[k].copy_(Hh[k], non_blocking=True)
            Vd[k].copy_(Vh[k], non_blocking=True)
        chase.chase_filter_batched(Hd, Vd, degs, bs, m1, mn, precision=prec,
                                   tile=args.batch_tile)
        for k in range(P):
            Vo[k].copy_(Vd[k], non_blocking=True)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        e2e = {"value": round(flops / te / 1e12, 4), "unit": "TFLOP/s",
               "h2d_bytes_per_step": int(h_bytes + v_bytes), "d2h_bytes_per_step": int(v_bytes),
               "seconds": round(te, 3)}
        del Hh, Vh, Hd, Vd, Vo
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        cpu = batched_cpu_baseline(shapes, degs, args.seed, args.cpu_sample_seconds)
    ns = [n for n, _, _ in shapes]
    cfg = {
        "workload": (f"batch of {P} independent problems, N uniform in [256, 2048] "
                     f"(sum N = {sum(ns)}), nev = 5% N, nex = 2% N, eigenvalues uniform in "
                     f"[-1, 1], degrees {args.batch_degrees}"
                     + (f" {args.filter_degree}" if args.batch_degrees == "const" else " in [2, 36]")
                     + "; step = one grouped filter call"),
        "problems": P, "precision": args.precision,
        "l2": f"inputs larger than L2 (H of the batch = {h_bytes / 1e9:.1f} GB)",
        "parallelism": "replicas" if world > 1 else "single GPU",
    }
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t_main, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16-split+f64" if split else "f64", "data": "synthetic", "config": cfg,
        "batched": {"tile_config": st_main[0]["tile_config"], "steps": st_main[0]["steps"],
                    "graph_seconds": round(t_steps, 4), "product_seconds": round(t_prod, 4),
                    "graph_build_seconds": round(st_main[0]["t_graph_build"], 4),
                    "launches_per_call": st_main[0]["launches"]},
        "other_precision": other, "roofline": roof, "e2e": e2e, "cpu_baseline": cpu,
        "gpu_launches": int(launches), "clocks": clk,
    }
    if rank == 0:
        emit(line)


def run_batched_solve_workload(args, rank, world, local):
    """Many independent problems solved by chase_solve_batched: every
    iteration's filters of all problems still iterating run as one grouped
    launch per degree step.  Also times the first 32 problems solved one by
    one with chase_solve against the batched solve of the same 32."""
    from paper_1805_10121_gb300 import build, chase, synth
    build.build()
    chase.lib()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P = args.batch_problems
    seed = args.seed + 1000 * rank
    shapes = synth.batched_shapes(P, seed)
    Hs, lams, V0s, Ss = [], [], [], []
    for k, (n, nev, nex) in enumerate(shapes):
        lam = synth.spectrum_uniform(n, seed + 10 * k, device=dev)
        Hs.append(synth.hermitian_dft(lam, seed + 10 * k + 1))
        lams.append(lam.cpu().numpy())
        V0s.append(synth.gaussian_block(n, nev + nex, seed + 10 * k + 2, device=dev))
        Ss.append(synth.gaussian_block(n, 5, seed + 10 * k + 3, device=dev))
    nevs = [s[1] for s in shapes]
    nexs = [s[2] for s in shapes]
    prec = prec_code(args.precision)
    o = chase.chase_opts_default(precision=prec, deg_extra=deg_extra_for(args, prec),
                                 deg_max=deg_max_for(args, prec))

    def batched(idx):
        Vs = [V0s[i].clone() for i in idx]
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = chase.chase_solve_batched([Hs[i] for i in idx], [nevs[i] for i in idx],
                                        [nexs[i] for i in idx], args.tol, Vs,
                                        [Ss[i] for i in idx], opts=o)
        torch.cuda.synchronize()
        return time.perf_counter() - t, out

    sub = list(range(min(32, P)))
    # warm-up: library, handles, kernels, and one problem per size bucket of
    # the batched eigensolver (its first use per size costs seconds)
    cover = {}
    for i in range(P):
        cover.setdefault((nevs[i] + nexs[i] + 15) // 16, i)
    warm = sorted(cover.values())
    batched(warm)
    for _ in range(max(0, args.warmup - 1)):
        batched(sub[:4])
    clocks = ClockSampler(local)
    launches0 = chase.chase_kernel_launches()
    clocks.start()
    wall, (st, sts, ritz, res, stats, bst) = batched(list(range(P)))
    clk = clocks.stop()
    launches = chase.chase_kernel_launches() - launches0
    flops = sum(s["flops_total"] for s in stats)
    ok = all(x == 0 for x in sts)
    err = max(float(np.max(np.abs(ritz[k][:nevs[k]] - lams[k][:nevs[k]]))) /
              float(np.abs(lams[k]).max()) for k in range(P))
    # the same 32 problems one by one
    t_seq = 0.0
    for i in sub:
        V = V0s[i].clone()
        torch.cuda.synchronize()
        t = time.perf_counter()
        chase.chase_solve(Hs[i], nevs[i], nexs[i], args.tol, V, Ss[i], opts=o)
        torch.cuda.synchronize()
        t_seq += time.perf_counter() - t
    t_b32, _ = batched(sub)
    pk, src = peaks()
    cfg = {
        "workload": (f"batched solve of {P} independent problems, N uniform in [256, 2048], "
                     f"nev = 5% N, nex = 2% N, eigenvalues uniform in [-1, 1], tol {args.tol}; "
                     f"step = one chase_solve_batched call"),
        "problems": P, "precision": args.precision, "deg_extra": o.deg_extra,
        "l2": "inputs larger than L2",
        "parallelism": "replicas" if world > 1 else "single GPU",
    }
    its = [s["iterations"] for s in stats]
    line = {
        "metric": METRIC, "value": round(flops / wall / 1e12, 4), "unit": "TFLOP/s",
        "n_gpus": world, "steps": 1, "warmup": args.warmup, "ms_per_step": round(1e3 * wall, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16-split+f64" if prec != chase.CHASE_FP64 else "f64", "data": "synthetic",
        "config": cfg,
        "batched_solve": {"all_converged": ok, "max_eig_err_over_norm": err,
                          "iterations_min_mean_max": [min(its), round(float(np.mean(its)), 2),
                                                      max(its)],
                          "grouped_filter_seconds": round(bst["t_steps"], 3),
                          "grouped_product_seconds": round(bst["t_product"], 3),
                          "grouped_steps": bst["steps"],
                          "qr_seconds": round(bst["t_qr"], 3),
                          "rr_seconds": round(bst["t_rr"], 3),
                          "eigh_seconds": round(bst["t_eigh"], 3),
                          "lock_reorder_seconds": round(bst["t_lock"], 3),
                          "lanczos_seconds_sum": round(sum(s["t_lanczos"] for s in stats), 3),
                          "phases_note": "QR, Rayleigh-Ritz (with the batched eigensolves) and "
                                         "the reordering run for all problems at once (device "
                                         "seconds of the whole batch); Lanczos runs per problem "
                                         "on eight worker threads (sum over problems)",
                          "first32_one_by_one_seconds": round(t_seq, 3),
                          "first32_batched_seconds": round(t_b32, 3),
                          "first32_speedup": round(t_seq / t_b32, 2)},
        "gpu_launches": int(launches), "clocks": clk,
    }
    if rank == 0:
        emit(line)


def batched_cpu_baseline(shapes, degs, seed, budget_s):
    """The oracle's filter on the first problems of the same batch (inputs
    from the host generators), until the time budget is spent; only the
    filter calls are timed."""
    import oracle
    from paper_1805_10121_gb300 import synth
    spent, fl, k = 0.0, 0.0, 0
    while k < len(shapes) and spent < budget_s:
        n, nev, nex = shapes[k]
        nx = nev + nex
        lam = synth.spectrum_uniform(n, seed + 10 * k)
        H = synth.hermitian_dft(lam, seed + 10 * k + 1).numpy()
        V = synth.gaussian_block(n, nx, seed + 10 * k + 2).numpy()
        l = lam.numpy()
        ts = time.perf_counter()
        oracle.cheb_filter(H, V, np.sort(degs[k]), 1.01, float(l[0]), float(l[nx]))
        spent += time.perf_counter() - ts
        fl += 8.0 * n * n * float(np.sum(degs[k]))
        k += 1
    return {"value": round(fl / spent / 1e12, 6), "unit": "TFLOP/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"oracle Alg. 4 filter of the first {k} problems of the batch (NumPy, "
                      f"BLAS threads = all host cores)",
            "seconds": round(spent, 2)}


def run_degree_sweep(args, rank, world, local):
    """Fig. 1a/2 on synthetic data: total and filter FLOPs and time of one
    cold solve against the (initial) degree, with the per-column degree
    optimisation (Alg. 5) off and on.  The problem is problem 1 of the
    sequence workload (--n, --nev, --nex)."""
    from paper_1805_10121_gb300 import build, chase, synth
    build.build()
    chase.lib()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, nev, nex, tol = args.n, args.nev, args.nex, args.tol
    seed = args.seed + 1000 * rank
    seq, lam, hnorm = make_sequence(n, 1, seed, dev)
    H = seq[0]
    V0 = synth.gaussian_block(n, nev + nex, seed + 7, device=dev)
    S = synth.gaussian_block(n, 5, seed + 8, device=dev)
    prec = prec_code(args.precision)
    degs = [int(x) for x in args.sweep_degrees.split(",")]
    rows = []
    # warm-up: one solve (library load, cuSOLVER handle)
    chase.chase_solve(H, nev, nex, tol, V0.clone(), S,
                      opts=chase.chase_opts_default(precision=prec, deg=degs[0]))
    torch.cuda.synchronize()
    launches0 = chase.chase_kernel_launches()
    clocks = ClockSampler(local)
    clocks.start()
    t_all = time.perf_counter()
    for optim in (0, 1):
        for deg in degs:
            V = V0.clone()
            o = chase.chase_opts_default(precision=prec, deg=deg, optim=optim)
            t0 = time.perf_counter()
            st, ritz, res, stt = chase.chase_solve(H, nev, nex, tol, V, S, opts=o)
            dt = time.perf_counter() - t0
            rows.append({"optim": optim, "deg": deg, "status": int(st),
                         "iterations": stt["iterations"],
                         "gflops_total": round(stt["flops_total"] / 1e9, 1),
                         "gflops_filter": round(stt["flops_filter"] / 1e9, 1),
                         "filter_matvecs": stt["filter_matvecs"], "seconds": round(dt, 3),
                         "max_resid_over_norm": float(np.max(res[:nev])) / hnorm})
    wall = time.perf_counter() - t_all
    clk = clocks.stop()
    fl = sum(r["gflops_total"] for r in rows) * 1e9
    spread = {}
    for optim in (0, 1):
        g = [r["gflops_total"] for r in rows if r["optim"] == optim and r["status"] == 0]
        spread[f"optim{optim}"] = round(max(g) / min(g), 3) if g else None
    cfg = workload_config(args, world)
    cfg["workload"] = (f"degree sweep (Fig. 1a/2 on synthetic data): one cold solve of problem 1 "
                       f"of the sequence workload, N={n}, nev={nev}, nex={nex}, tol={tol}, "
                       f"deg in {degs}, optim off and on; step = the whole sweep")
    line = {
        "metric": METRIC, "value": round(fl / wall / 1e12, 4), "unit": "TFLOP/s", "n_gpus": world,
        "steps": 1, "warmup": 1, "ms_per_step": round(1e3 * wall, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16-split+f64" if prec == chase.CHASE_SPLIT_BF16 else "f64",
        "data": "synthetic", "config": cfg,
        "sweep": rows, "gflops_max_over_min": spread,
        "gpu_launches": int(chase.chase_kernel_launches() - launches0), "clocks": clk,
    }
    if rank == 0:
        emit(line)


def run_side_workload(args, rank, world, local):
    """The steps beside the filter, one C-ABI call each on problem 1 of the
    sequence workload: the Lanczos bound estimate of a warm start (Alg. 6,
    one vector, k = 25 matvecs), the full Lanczos of a cold start (1 + n_vec
    = 5 vectors as one block) and the residual norms of the nev + nex block
    (one product with H plus the fused norm kernel).  All are FP64; on this
    GPU the FP64 pipe, not HBM, bounds each of them (the one-vector matvec
    has 2 FLOP/byte against a machine balance of 0.15), so each line gives
    the FP64 rate and the HBM rate the pass over H achieved."""
    from paper_1805_10121_gb300 import build, chase, synth
    build.build()
    chase.lib()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, nev, nex = args.n, args.nev, args.nex
    nx = nev + nex
    seed = args.seed + 1000 * rank
    seq, lam, hnorm = make_sequence(n, 1, seed, dev)
    H = seq[0]
    S = synth.gaussian_block(n, 5, seed + 8, device=dev)
    V = synth.gaussian_block(n, nx, seed + 7, device=dev)
    w = np.linspace(float(lam.min()), float(lam.max()), nx)
    stream = torch.cuda.current_stream(dev)
    k = 25

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3 / args.steps

    launches0 = chase.chase_kernel_launches()
    clocks = ClockSampler(local)
    clocks.start()
    t_warm = timed(lambda: chase.chase_lanczos(H, k, 4, 1, nev, nex, S[:, :1]))
    t_cold = timed(lambda: chase.chase_lanczos(H, k, 4, 0, nev, nex, S))
    t_res = timed(lambda: chase.chase_residuals(H, V, w))
    clk = clocks.stop()
    launches = chase.chase_kernel_launches() - launches0
    pk, src = peaks()
    fp64_peak = pk.get("bf16_tflops", 1900.0) * NOMINAL_FP64_OVER_BF16
    hbm = pk.get("hbm_gbs", 6800.0)

    def entry(what, secs, flops, hbm_bytes, kernel):
        tf = flops / secs / 1e12
        gbs = hbm_bytes / secs / 1e9
        return {"step": what, "kernel": kernel, "seconds": round(secs, 5),
                "tflops": round(tf, 4), "fp64_frac": round(tf / fp64_peak, 4),
                "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4)}

    h_bytes = 16.0 * n * n
    rows = [
        entry("Lanczos bound, warm start (1 vector, 25 steps)", t_warm, 8.0 * n * n * k,
              h_bytes * k, "fewcol_kernel<1> + lanczos_step_kernel"),
        entry("Lanczos with DoS, cold start (5 vectors, 25 steps)", t_cold, 8.0 * n * n * k * 5,
              h_bytes * k, "fewcol_kernel<5> + lanczos_step_kernel"),
        entry(f"residual norms of {nx} columns", t_res, 8.0 * n * n * nx,
              h_bytes + 3 * 16.0 * n * nx, "zgemm_tma_kernel + resid_norms_kernel"),
    ]
    cfg = workload_config(args, world)
    cfg["workload"] = (f"steps beside the filter on problem 1 of the sequence workload, N={n}, "
                       f"nev={nev}, nex={nex}: Lanczos (warm and cold) and residual norms; "
                       f"step = one call of each")
    line = {
        "metric": METRIC, "value": rows[0]["tflops"], "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * (t_warm + t_cold + t_res), 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg, "side_steps": rows,
        "roofline": {"bound": "tensor", "kernel": "fewcol_kernel (FP64 FMA): Lanczos matvec",
                     "achieved": rows[0]["tflops"], "peak": round(fp64_peak, 4),
                     "unit": "TFLOP/s", "frac": rows[0]["fp64_frac"], "traffic": None,
                     "peak_source": f"{src} bf16_tflops x nominal FP64/BF16 ratio (1.25/2250)"},
        "gpu_launches": int(launches), "clocks": clk,
    }
    if rank == 0:
        emit(line)


def run_variants_workload(args, rank, world, local):
    """The real symmetric and single-precision solvers on the sequence law:
    a correlated sequence H_{k+1} = H_k + 1e-3 ||H_1|| E_k with the
    spectrum of the sequence workload, built as a real symmetric matrix
    (Q orthogonal, E symmetric) for float64 and float32 and as a Hermitian
    one for complex64; warm-started solves as in the default workload.
    Single precision uses tol = max(--tol, 1e-5) (Table 1's single-precision
    column).  Each variant's line gives seconds per solve, iterations, the
    largest residual and its algorithmic TFLOP/s."""
    from paper_1805_10121_gb300 import build, chase, synth
    build.build()
    chase.lib()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, nev, nex = args.n, args.nev, args.nex
    nx = nev + nex
    W, K = args.warmup, args.steps
    seed = args.seed + 1000 * rank
    prec = prec_code(args.precision)
    stream = torch.cuda.current_stream(dev)

    def sequence(real, dtype):
        lam = synth.spectrum_dft(n, seed, device=dev)
        hnorm = float(lam.abs().max())
        if real:
            H = synth.symmetric_from(synth.orthogonal_qr(n, seed + 1, device=dev), lam)
        else:
            H = synth.hermitian_from(synth.unitary_dft(n, seed + 1, device=dev), lam)
        seq = []
        for k in range(W + K):
            if k > 0:
                E = (synth.symmetric_noise if real else synth.hermitian_noise)(
                    n, seed + 100 + k, device=dev)
                H = (H + (1e-3 * hnorm) * E).t().contiguous().t()
                del E
            seq.append(H.to(dtype).t().contiguous().t())
        del H
        return seq, hnorm

    rows = []
    launches0 = chase.chase_kernel_launches()
    clocks = ClockSampler(local)
    clocks.start()
    stol = max(args.tol, 1e-5)
    split = chase.CHASE_SPLIT_BF16
    for name, real, dtype, entry, precision, tol in (
            ("float64 real symmetric", True, torch.float64, chase.chase_solve_real, prec, args.tol),
            ("complex64", False, torch.complex64, chase.chase_solve_c32, None, stol),
            ("complex64, filter on the 4-slice split product", False, torch.complex64,
             chase.chase_solve_c32, split, stol),
            ("float32 real symmetric", True, torch.float32, chase.chase_solve_f32, None, stol),
            ("float32 real symmetric, filter on the 4-slice split product", True, torch.float32,
             chase.chase_solve_f32, split, stol)):
        seq, hnorm = sequence(real, dtype)
        blk = synth.gaussian_block_real if real else synth.gaussian_block
        V = blk(n, nx, seed + 7, device=dev).to(dtype)
        S = blk(n, 5, seed + 8, device=dev).to(dtype).t().contiguous().t()
        Lam = None
        times, its, res_max, flops, t_filt = [], [], 0.0, 0.0, 0.0
        for k in range(W + K):
            kw = {} if precision is None else {"precision": precision}
            o = chase.chase_opts_default(approx=0 if k == 0 else 1, **kw)
            Sk = S if k == 0 else S[:, :1].contiguous()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st, Lam, res, s = entry(seq[k], nev, nex, tol, V, Sk, Lambda=Lam, opts=o)
            b.record(stream)
            torch.cuda.synchronize()
            if k >= W:
                times.append(a.elapsed_time(b) / 1e3)
                its.append(s["iterations"])
                res_max = max(res_max, float(np.max(res[:nev])) / hnorm)
                flops += s["flops_total"]
                t_filt += s["t_filter"]
                if st != 0:
                    raise RuntimeError(f"{name}: solve {k} returned status {st}")
        label = "fp32" if precision is None else (
            "split4" if dtype in (torch.complex64, torch.float32) else args.precision)
        rows.append({"variant": name, "tol": tol, "precision": label,
                     "s_per_solve": round(float(np.mean(times)), 3), "iterations": its,
                     "filter_s_per_solve": round(t_filt / len(times), 3),
                     "resid_max_over_norm": res_max,
                     "tflops": round(flops / sum(times) / 1e12, 3)})
        del seq, V, S
        torch.cuda.empty_cache()
    clk = clocks.stop()
    cfg = workload_config(args, world)
    cfg["workload"] = (f"real symmetric and single-precision solves of the sequence law, N={n}, "
                       f"nev={nev}, nex={nex}, warm start; step = one solve of each variant")
    line = {
        "metric": METRIC, "value": rows[0]["tflops"], "unit": "TFLOP/s", "n_gpus": world,
        "steps": K, "warmup": W, "ms_per_step": round(1e3 * sum(r["s_per_solve"] for r in rows), 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64/c32/f32", "data": "synthetic", "config": cfg, "variants": rows,
        "gpu_launches": int(chase.chase_kernel_launches() - launches0), "clocks": clk,
    }
    if rank == 0:
        emit(line)


def run_solve_workload(args, rank, world, local):
    """One cold solve of a problem with the sequence law's spectrum, built
    by the FFT construction (``synth.hermitian_dft``, O(N^2 log N), so that
    N = 30000 builds in seconds): approx = 0, so Lanczos with the density of
    states, the constant initial degree, then per-column degrees; the
    mixed-precision configuration's solve.  --warmup solves of an
    N = min(N, 2000) problem load the library and handles first; --steps
    cold solves at the full size are timed.  The spectrum is known, so the
    line gives the eigenvalue error against it."""
    from paper_1805_10121_gb300 import build, chase, synth
    build.build()
    chase.lib()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, nev, nex, tol = args.n, args.nev, args.nex, args.tol
    nx = nev + nex
    seed = args.seed + 1000 * rank
    prec = prec_code(args.precision)
    de = args.deg_extra if args.deg_extra is not None else (
        2 if prec == chase.CHASE_FP64 else COLD_SOLVE_DEG_EXTRA)
    stream = torch.cuda.current_stream(dev)

    def problem(nn, sd):
        lam = synth.spectrum_dft(nn, sd, device=dev)
        return synth.hermitian_dft(lam, sd + 1), lam.cpu().numpy()

    nw = min(n, 2000)
    Hw, _ = problem(nw, seed + 50)
    for _ in range(args.warmup):
        ns = max(1, nw * nev // n)
        nxw = max(ns + 1, nw * nx // n)
        chase.chase_solve(Hw, ns, nxw - ns, tol, synth.gaussian_block(nw, nxw, seed + 51, device=dev),
                          synth.gaussian_block(nw, 5, seed + 52, device=dev),
                          opts=chase.chase_opts_default(precision=prec, deg_extra=de,
                                                        deg_max=deg_max_for(args, prec)))
    del Hw
    warm_eigensolver(dev, [nx])
    H, lam = problem(n, seed)
    hnorm = float(np.abs(lam).max())
    S = synth.gaussian_block(n, 5, seed + 8, device=dev)
    launches0 = chase.chase_kernel_launches()
    clocks = ClockSampler(local)
    clocks.start()
    rows = []
    total_t, total_f = 0.0, 0.0
    for k in range(args.steps):
        V = synth.gaussian_block(n, nx, seed + 7 + k, device=dev)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st, ritz, res, s = chase.chase_solve(H, nev, nex, tol, V, S,
                                             opts=chase.chase_opts_default(
                                                 precision=prec, deg_extra=de,
                                                 deg_max=deg_max_for(args, prec)))
        b.record(stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / 1e3
        total_t += t
        total_f += s["flops_total"]
        rows.append({"status": st, "seconds": round(t, 2), "iterations": s["iterations"],
                     "resid_max_over_norm": float(np.max(res[:nev])) / hnorm,
                     "eig_err_max_over_norm": float(np.max(np.abs(ritz[:nev] - lam[:nev]))) / hnorm,
                     "phase_seconds": {k2: round(s[k2], 2) for k2 in
                                       ("t_lanczos", "t_filter", "t_qr", "t_rr", "t_eigh")},
                     "filter_matvecs": s["filter_matvecs"],
                     "filter_matvecs_low_precision": s["filter_matvecs_low"],
                     "filter_tflops": round(s["flops_filter"] / max(s["t_filter"], 1e-12) / 1e12, 2)})
        del V
    clk = clocks.stop()
    cfg = workload_config(args, world)
    cfg["deg_extra"] = de
    cfg["workload"] = (f"cold solve of one problem, N={n} complex128 (FFT construction of "
                       f"Q diag(lambda) Q^H, the sequence law's spectrum), nev={nev}, nex={nex}, "
                       f"tol={tol} x ||H||; step = one solve")
    line = {
        "metric": METRIC, "value": round(total_f / total_t / 1e12, 4), "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * total_t / args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16-split+f64" if args.precision != "fp64" else "f64", "data": "synthetic",
        "config": cfg, "solves": rows,
        "gpu_launches": int(chase.chase_kernel_launches() - launches0), "clocks": clk,
    }
    if rank == 0:
        emit(line)


def run_serve_workload(args, rank, world, local):
    """Replay a seeded Poisson trace of sequence-solve requests through the
    continuous-batching server; report throughput and p50/p99 latency."""
    from paper_1805_10121_gb300 import build, chase, serve
    build.build()
    chase.lib()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    split = args.precision != "fp64"
    prec = prec_code(args.precision)
    sizes = tuple(int(x) for x in args.serve_sizes.split(","))
    weights = (4, 3, 2, 1)[:len(sizes)]
    trace = serve.poisson_trace(args.serve_requests, args.serve_rate, args.seed + 1000 * rank,
                                sizes=sizes, weights=weights)
    fp = lambda r: serve.footprint_bytes(r.n, r.nev, r.nex, split)
    solver = serve.gpu_sequence_solver(dev, prec, tol=args.tol, deg_extra=deg_extra_for(args, prec),
                                       deg_max=deg_max_for(args, prec))
    # warm-up: one small request (library load, handles, kernels)
    small = serve.Request(-1, min(sizes), int(np.ceil(0.04 * min(sizes))),
                          int(np.ceil(0.008 * min(sizes))), 2, 99, 0.0)
    serve.Server(solver, args.serve_cap_gb * 1e9, 1, fp).run([small])
    warm_eigensolver(dev, sorted({r.nev + r.nex for r in trace}))
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    launches0 = chase.chase_kernel_launches()
    clocks.start()
    t0 = time.perf_counter()
    srv = serve.Server(solver, args.serve_cap_gb * 1e9, args.serve_slots, fp,
                       policy=args.serve_policy, max_wait_s=args.serve_max_wait)
    res = srv.run(trace)
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    lat = [r.latency for r in res]
    flops = sum(r.flops for r in res)
    nprob = sum(r.nprob for r in res)
    ok = all(st == 0 for r in res for st in r.statuses)
    cfg = workload_config(args, world)
    cfg["workload"] = (f"serving: {len(trace)} sequence-solve requests, Poisson {args.serve_rate}/s, "
                       f"N in {sizes} weighted {weights}, 5-10 problems each, nev = 4% N, "
                       f"nex = 20% nev, admission cap {args.serve_cap_gb} GB, "
                       f"{args.serve_slots} slots, admission {args.serve_policy}; "
                       f"step = the whole trace")
    cfg["deg_extra"] = deg_extra_for(args, prec)
    cfg["deg_max"] = deg_max_for(args, prec)
    line = {
        "metric": METRIC, "value": round(flops / wall / 1e12, 3), "unit": "TFLOP/s",
        "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": round(1e3 * wall, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16-split+f64" if split else "f64", "data": "synthetic", "config": cfg,
        "serve": {"p50_latency_s": round(serve.percentile(lat, 50), 3),
                  "p99_latency_s": round(serve.percentile(lat, 99), 3),
                  "mean_queueing_s": round(float(np.mean([r.queueing for r in res])), 3),
                  "requests_per_s": round(len(res) / wall, 4),
                  "problems_per_s": round(nprob / wall, 4),
                  "all_converged": ok, "peak_concurrency": srv.peak_concurrency,
                  "peak_admitted_gb": round(srv.peak_mem / 1e9, 2),
                  "max_resid_over_norm": max(max(r.resid_max_over_norm) for r in res),
                  "per_request": [{"rid": r.rid, "n": r.n, "problems": r.nprob,
                                   "arrival": round(r.arrival, 3),
                                   "queueing": round(r.queueing, 3),
                                   "latency": round(r.latency, 3),
                                   "iterations": r.iterations} for r in res]},
        "gpu_launches": int(chase.chase_kernel_launches() - launches0), "clocks": clk,
    }
    if rank == 0:
        emit(line)


def main():
    global BUILD_INFO
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    BUILD_INFO = build_library()
    if args.workload == "filter":
        run_filter_workload(args, rank, world, local)
        return
    if args.workload == "serve":
        run_serve_workload(args, rank, world, local)
        return
    if args.workload == "batched":
        run_batched_workload(args, rank, world, local)
        return
    if args.workload == "batched-solve":
        run_batched_solve_workload(args, rank, world, local)
        return
    if args.workload == "solve":
        run_solve_workload(args, rank, world, local)
        return
    if args.workload == "variants":
        run_variants_workload(args, rank, world, local)
        return
    if args.workload == "side":
        run_side_workload(args, rank, world, local)
        return
    if args.workload == "degree-sweep":
        run_degree_sweep(args, rank, world, local)
        return
    from paper_1805_10121_gb300 import build, chase, synth
    build.build()
    chase.lib()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    n, nev, nex, tol = args.n, args.nev, args.nex, args.tol
    nx = nev + nex
    W, K = args.warmup, args.steps
    seed = args.seed + 1000 * rank
    seq, lam, hnorm = make_sequence(n, W + K, seed, dev)
    V = synth.gaussian_block(n, nx, seed + 7, device=dev)
    starts = synth.gaussian_block(n, 5, seed + 8, device=dev).t().contiguous().t()
    Lam = None

    prec = prec_code(args.precision)

    def solve(k, Vb, Lamb, precision=None):
        p = prec if precision is None else precision
        o = chase.chase_opts_default(approx=0 if k == 0 else 1, precision=p,
                                     deg_extra=deg_extra_for(args, p), deg_max=deg_max_for(args, p))
        S = starts if k == 0 else starts[:, :1].contiguous()
        return chase.chase_solve(seq[k], nev, nex, tol, Vb, S, Lambda=Lamb, opts=o)

    stats_w = []
    for k in range(W):
        st, Lam, res, s = solve(k, V, Lam)
        stats_w.append((st, s))
    torch.cuda.synchronize()
    V_before = V.clone()
    Lam_before = Lam.copy()
    # ---------------- timed region ----------------
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    launches0 = chase.chase_kernel_launches()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    stats_t = []
    statuses = []
    resid_max = 0.0
    first_lam = None
    for k in range(W, W + K):
        st, Lam, res, s = solve(k, V, Lam)
        if first_lam is None:
            first_lam = Lam.copy()
            first_time = s["t_total"]
        stats_t.append(s)
        statuses.append(st)
        resid_max = max(resid_max, float(np.max(res[:nev])) / hnorm)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    launches = chase.chase_kernel_launches() - launches0
    elapsed = e0.elapsed_time(e1) / 1e3
    t_max, total_flops = combine_over_ranks(elapsed, sum(s["flops_total"] for s in stats_t), dev)
    value = total_flops / t_max / 1e12

    # ---------------- the same problem on the FP64 path ----------------
    fp64 = None
    if args.precision != "fp64" and not args.no_fp64_compare:
        Vc = V_before.clone()
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        st_c, lam_c, res_c, s_c = solve(W, Vc, Lam_before.copy(), precision=chase.CHASE_FP64)
        c1.record(stream)
        torch.cuda.synchronize()
        t_c = c0.elapsed_time(c1) / 1e3
        fp64 = {"s_per_solve": round(t_c, 3), "iterations": s_c["iterations"], "status": st_c,
                "filter_tflops": round(s_c["flops_filter"] / s_c["t_filter"] / 1e12, 4),
                "resid_max_over_norm": float(np.max(res_c[:nev])) / hnorm,
                "max_abs_eig_diff_vs_split_over_norm":
                    float(np.max(np.abs(lam_c[:nev] - first_lam[:nev]))) / hnorm,
                "speedup_split_vs_fp64": round(t_c / first_time, 2)}
        del Vc

    # ------- the same problem with Rayleigh-Ritz's H Q on the split product -------
    split_rr = None
    if args.precision == "split" and not args.no_fp64_compare:
        Vc = V_before.clone()
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        st_c, lam_c, res_c, s_c = solve(W, Vc, Lam_before.copy(),
                                        precision=chase.CHASE_SPLIT_BF16_RR)
        c1.record(stream)
        torch.cuda.synchronize()
        t_c = c0.elapsed_time(c1) / 1e3
        split_rr = {"s_per_solve": round(t_c, 3), "iterations": s_c["iterations"], "status": st_c,
                    "t_rr": round(s_c["t_rr"], 3),
                    "resid_max_over_norm": float(np.max(res_c[:nev])) / hnorm,
                    "max_abs_eig_diff_vs_split_over_norm":
                        float(np.max(np.abs(lam_c[:nev] - first_lam[:nev]))) / hnorm,
                    "speedup_vs_split": round(first_time / t_c, 3)}
        del Vc

    # ---------------- end-to-end through host buffers ----------------
    e2e = None
    if not args.no_e2e:
        k = W
        Hh = torch.empty((n, n), dtype=torch.complex128, pin_memory=True).t()
        Hh.copy_(seq[k])
        Vh = torch.empty((nx, n), dtype=torch.complex128, pin_memory=True).t()
        Vh.copy_(V_before)
        Sh = torch.empty((1, n), dtype=torch.complex128, pin_memory=True).t()
        Sh.copy_(starts[:, :1])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        o = chase.chase_opts_default(approx=1, precision=prec,
                                     deg_extra=deg_extra_for(args, prec),
                                     deg_max=deg_max_for(args, prec))
        st_e, lam_e, res_e, s_e = chase.chase_solve(Hh, nev, nex, tol, Vh, Sh,
                                                    Lambda=Lam_before, opts=o)
        t_e2e = time.perf_counter() - t0
        h2d = (Hh.numel() + Vh.numel() + Sh.numel()) * 16
        d2h = Vh.numel() * 16 + 2 * nx * 8
        e2e = {"value": round(s_e["flops_total"] / t_e2e / 1e12, 4), "unit": "TFLOP/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "seconds": round(t_e2e, 3), "status": st_e}
        del Hh, Vh, Sh

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    pk, src = peaks()
    roof_main, roof_other = roofline_entry(stats_t, pk, src, args.precision)
    cb = None
    if not args.no_cpu_baseline and world == 1:
        cb = cpu_baseline_sample(n, nev, nex, args.seed, args.cpu_sample_seconds)
    filt_fl = sum(s["flops_filter"] for s in stats_t)
    filt_t = sum(s["t_filter"] for s in stats_t)
    line = {
        "metric": METRIC,
        "value": round(value, 4),
        "unit": "TFLOP/s",
        "n_gpus": world,
        "steps": K,
        "warmup": W,
        "ms_per_step": round(1e3 * t_max / K, 1),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "bf16-split+f64" if args.precision != "fp64" else "f64",
        "data": "synthetic",
        "config": dict(workload_config(args, world), deg_extra=deg_extra_for(args, prec),
                       deg_max=deg_max_for(args, prec)),
        "s_per_solve": round(t_max / K, 3),
        "filter_tflops": round(filt_fl / filt_t / 1e12, 4) if filt_t > 0 else None,
        "filter_share_of_time": round(filt_t / max(elapsed, 1e-12), 4),
        "iterations": [s["iterations"] for s in stats_t],
        "matvecs": [s["matvecs"] for s in stats_t],
        "filter_matvecs_low_precision": [s["filter_matvecs_low"] for s in stats_t],
        "status": statuses,
        "resid_max_over_norm": resid_max,
        "phase_seconds": {k2: round(sum(s[k2] for s in stats_t), 3)
                          for k2 in ("t_lanczos", "t_filter", "t_qr", "t_rr", "t_eigh", "t_host")},
        "warmup_iterations": [s["iterations"] for _, s in stats_w],
        "roofline": roof_main,
        "roofline_other_kernel": roof_other,
        "lanczos": lanczos_entry(stats_t, n, pk, src),
        "fp64_same_problem": fp64,
        "split_rr_same_problem": split_rr,
        "cpu_baseline": cb,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    emit(line)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
