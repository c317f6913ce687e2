#!/usr/bin/env python3
"""Benchmark: solved nodes/s of the RBF-FD Poisson pipeline on GB300.

Workload (default): the unit-disk problem with N ~ 4.0e6 scattered nodes,
m = 6 (s = 28 monomials), n = 56 nearest neighbours, manufactured solution
u = sin(pi x) sin(pi y), solved to a relative residual of 1e-10.

One step = the whole hot path on inputs already resident in HBM:
stencils -> weights -> assembly (pattern, f64 + f32 values) -> rhs ->
multigrid hierarchy (coarse node sets, rediscretised operators, transfer
operators) -> BiCGSTAB solve right-preconditioned by a V-cycle.  The
headline `value` uses the mixed solve (float32 V-cycle inside the FP64
BiCGSTAB); the same steps with an FP64 V-cycle are timed beside it ("fp64").
`--precond jacobi` runs the Jacobi-scaled solvers instead (mixed: float32
inner BiCGSTAB in FP64 refinement).  `e2e` repeats the step through the
public API from pinned host buffers, host<->device copies inside the timed
region.

Multi-GPU: the problem is solved independently on every rank (replicas:
the path has no cross-GPU exchange here), value = nodes of all ranks /
max-over-ranks time, scaling "weak".

`--impl reference` times the CPU oracle (the plain FP64 numpy/scipy
implementation the tests check against) on a bounded sample of the same
workload: the same disk recipe, m and n, at a spacing sized for seconds of
single-core work per step.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (h, m, n) -- grid spacing fixed so N is reproducible
    "disk_4M_m6_n56": (8.862e-4, 6, 56),
    "disk_1M_m4_n30": (1.7725e-3, 4, 30),
    "disk_h0.04_m2_n12": (0.04, 2, 12),
    # profiling case: the 1M-node set at the highest degree (m = 6 weights and
    # solve at a quarter of the headline size, for ncu captures)
    "disk_1M_m6_n56": (1.7725e-3, 6, 56),
}
METRIC = "solved nodes/s (weights+solve) at m=6, 4M nodes; mixed vs FP64; % roofline"
# The batched workload (a separate measurement, not the headline line): 256
# disks with N log-uniform in [1e4, 2e5] and m uniform in {2, 4, 6} (n = 2s),
# 64 random Fourier right-hand sides each, g = 0, mixed solve to 1e-10.
BATCH_WORKLOAD = "disk_batch256_rhs64"
BATCH_METRIC = "solved node-rhs/s, 256 disks (N log-uniform 1e4..2e5, m in {2,4,6}) x 64 rhs, mixed, tol 1e-10"
# The paper's own GPU workload (Sec. IV Eq. 4, Sec. V): the explicit Euler
# loop, dt = 1e-6; measured on the 1M-node disk (m = 4, n = 30) and swept over
# N and n for the L2 data-size model of Table 1.
EXPLICIT_WORKLOAD = "explicit_1M_m4_n30"
EXPLICIT_METRIC = "explicit Euler node-steps/s (Eq. 4), 1M-node disk, m=4, n=30, dt=1e-6"
EXPLICIT_SWEEP_N = (1e4, 3e4, 1e5, 3e5, 1e6, 3e6)
EXPLICIT_SWEEP_n = (12, 15, 20, 30, 45, 60)
# The differentiable solve: forward solve and the adjoint gradient of
# L = sum_interior (u - u*)^2 with respect to f and g, on the 1M-node disk
# (m = 4, n = 30); u* solves the problem with a seeded Fourier source.
ADJOINT_WORKLOAD = "adjoint_1M_m4_n30"
ADJOINT_METRIC = ("differentiable solve nodes/s (forward + adjoint gradient dL/df, dL/dg), 1M-node disk, m=4, "
                  "n=30, tol 1e-10")
# The support-size sweep of the implicit path: n in {12, 15, 20, 30, 45, 60}
# x m in {2, 4, 6} (n >= s) on the 1M-node disk.
SWEEP_WORKLOAD = "support_sweep_1M"
SWEEP_METRIC = ("weights+solve nodes/s over the support sweep n x m on the 1M-node disk (the m = 4, n = 30 point; "
                "every point in 'sweep')")
SWEEP_N = (12, 15, 20, 30, 45, 60)
SWEEP_M = (2, 4, 6)
BATCH_RHS = 64
BATCH_SAMPLE_RHS = 8  # oracle sample: right-hand sides of the smallest instance per step
SEED = 2107
CPU_SAMPLE_H = 0.012  # oracle sample: same recipe, ~22k nodes, ~10-30 s of one core


# ------------------------------------------------------------------ helpers --
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(dist, v: float, device=None) -> float:
    """Largest value of v over all ranks (the slowest rank's time); v itself on one rank."""
    if dist is None:
        return float(v)
    import torch

    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(dist, ws: int, units_per_rank: int, steps: int, ms_local: float, device=None):
    """Whole-job throughput of independent replicas: the units all ranks processed / the slowest rank's time.

    Returns (value in units/s, max-over-ranks ms)."""
    ms = max_over_ranks(dist, ms_local, device)
    return ws * units_per_rank * steps / (ms * 1e-3), ms


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# DRAM traffic of the inner-solve SpMV from one ncu capture of
# spmv_df_kernel at 1M nodes (m = 4, n = 30): dram read + write per launch
# divided by the kernel's algorithmic bytes at that size.  The ratio scales
# the capture to a full-size launch (traffic grows with the matrix) and is
# valid only while the kernel's source is the one captured.
SPMV_DF_TRAFFIC = {"source_sha256_16": "ea63d4b54b1529b9", "traffic_over_algorithmic": (271.693312e6 + 8.42624e6)
                   / 279652728.0}


# DRAM traffic of the FP64 weight solve from one ncu capture of
# weights_ns_kernel<128, NsF64> (four warps per stencil) at 1M nodes, m = 6,
# n = 56: dram read + write per stencil (idx read, w written; the gathered
# coordinates come from L2).  Valid only at that (n, m) and while the
# kernel's sources are the ones captured.
WEIGHTS_F64_TRAFFIC = {"source_sha256_16": "5a541d3a57e1eb7e", "n": 56, "m": 6,
                       "bytes_per_node": (259.903744e6 + 406.790144e6) / 1001697.0}


def weights_source_hash():
    import hashlib

    d = os.path.join(ROOT, "paper_2107_03632_gb300", "csrc")
    seg = "".join(open(os.path.join(d, f)).read() for f in ("weights.cu", "common.cuh", "checked.cuh"))
    return hashlib.sha256(seg.encode()).hexdigest()[:16]


def spmv_df_source_hash():
    import hashlib

    src = open(os.path.join(ROOT, "paper_2107_03632_gb300", "csrc", "krylov.cu")).read()
    a = src.index("// ============================================================ double-float ==")
    b = src.index("__global__ void __launch_bounds__(kThreads) update_s_df_kernel")
    seg = src[a:b] + open(os.path.join(ROOT, "paper_2107_03632_gb300", "csrc", "df32.cuh")).read()
    return hashlib.sha256(seg.encode()).hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def weights_flops(n: int, m: int) -> float:
    """FP64 flops per node of the null-space weight solve (division and square
    root counted as one flop each): scaling 2n, monomials ~n s, Gauss-Jordan
    on P (2s - 1)(n s - s(s-1)/2), kernel matrix 4 n(n-1) + 5n, T = 2 s^2 q,
    u = 2 n s, S (lower) 2 s q (q+1), t = 2 q s, Cholesky q^3/3 + q^2/2 + 2q,
    substitutions 2 q^2 + 2q, w = 2 s q, output n."""
    s = (m + 1) * (m + 2) // 2
    q = n - s
    return (2 * n + n * s + (2 * s - 1) * (n * s - s * (s - 1) / 2) + 4 * n * (n - 1) + 5 * n + 2 * s * s * q
            + 2 * n * s + 2 * s * q * (q + 1) + 2 * q * s + q ** 3 / 3 + q * q / 2 + 2 * q + 2 * q * q + 2 * q
            + 2 * s * q + n)


# FP64 (non-tensor and tensor alike on this chip) peak from unit counts and the
# maximum clock: 152 SMs x 2 FP64 FMA per clock x 2 flops x 2070 MHz.
FP64_PEAK_TFLOPS_UNITS = 152 * 2 * 2 * 2070e6 / 1e12
# FP32 pipe: 152 SMs x 128 lanes x 2070 MHz, in tera lane-instructions per second.
FP32_PEAK_TINSTR_UNITS = 152 * 128 * 2070e6 / 1e12

# FP32 instructions of one double-float operation of the weight kernel, as
# written (df32.cuh and the NsDF policy): c - a b 15, a b 7, a + b 20,
# a^-1/2 20 (plus one MUFU op), 1/a 10.
DF_INSTR = {"nfma": 15, "mul": 7, "add": 20, "rsqrt": 20, "rcp": 10}


def weights_df_ops(n: int, m: int) -> dict:
    """Double-float operations per node of the null-space weight solve (the
    same steps as weights_flops): Gauss-Jordan on P, the r^3 matrix and
    f = 9|x|, T, u, S, t, Cholesky, the two substitutions and w = w0 + Z z."""
    s = (m + 1) * (m + 2) // 2
    q = n - s
    pairs = n * (n - 1) // 2
    gj_rows = s * n - s * (s - 1) // 2
    chol_tr = sum((q - c - 1) * (q - c) // 2 for c in range(q))
    return {
        "nfma": (s - 1) * gj_rows + s * q * s + n * s + (q * (q + 1) // 2) * 2 * s + q * s + chol_tr
                + q * (q - 1) + s * q,
        "mul": gj_rows + 4 * pairs + 4 * n + q * (q - 1) // 2 + q + 2 * q + n * 2 * m,
        "add": 3 * pairs + 2 * n + s * q + n + q * (q + 1) // 2 + q + s,
        "rsqrt": pairs + n + q,
        "rcp": s,
    }


def weights_df_instr(n: int, m: int) -> float:
    ops = weights_df_ops(n, m)
    return float(sum(DF_INSTR[k] * v for k, v in ops.items()))


def weights_roofline(kernel_name: str, n: int, m: int, N: int, ms: float, extra: dict) -> dict:
    """Roofline of the weight solve: FP64 kernels against the FP64 units'
    peak (counted flops); double-float kernels against the FP32 pipe's peak
    (FP32 instructions of the df operations), with the FP64-equivalent rate
    beside it."""
    fl = weights_flops(n, m)
    f64_equiv = fl * N / (ms * 1e-3) / 1e12
    if "df" in kernel_name:
        ins = weights_df_instr(n, m)
        ach = ins * N / (ms * 1e-3) / 1e12
        out = {"kernel": f"weights_ns_kernel, double-float ({kernel_name}), m={m}, n={n}", "bound": "alu",
               "achieved": ach, "peak": FP32_PEAK_TINSTR_UNITS, "unit": "T FP32 lane-instr/s",
               "frac": ach / FP32_PEAK_TINSTR_UNITS,
               "peak_kind": "FP32 lanes x max clock (152 SMs x 128 lanes x 2070 MHz)",
               "instr_per_node": ins, "df_ops_per_node": weights_df_ops(n, m),
               "fp64_equivalent_tflops": f64_equiv, "fp64_equivalent_frac_of_fp64_units": f64_equiv / FP64_PEAK_TFLOPS_UNITS}
    else:
        out = {"kernel": f"weights_ns_kernel, FP64 ({kernel_name}), m={m}, n={n}", "bound": "alu",
               "achieved": f64_equiv, "peak": FP64_PEAK_TFLOPS_UNITS, "unit": "TFLOP/s",
               "frac": f64_equiv / FP64_PEAK_TFLOPS_UNITS,
               "peak_kind": "FP64 units x max clock (152 SMs x 2 FMA/clk x 2070 MHz)"}
    traffic = None
    t = WEIGHTS_F64_TRAFFIC
    if "df" not in kernel_name and (n, m) == (t["n"], t["m"]) and weights_source_hash() == t["source_sha256_16"]:
        traffic = t["bytes_per_node"] * N
    out.update({"traffic": traffic, "traffic_unit": "bytes per launch (ncu dram read + write, scaled by N)",
                "flops_per_node": fl, "ms_per_launch": ms, "launches": 1})
    out.update(extra)
    return out


def fp64_peak_tflops(torch, dev):
    """cuBLAS DGEMM throughput on this GPU (the FP64 denominator), best of 5."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    for _ in range(2):
        a @ b
    torch.cuda.synchronize(dev)
    best = 1e30
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        a @ b
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


# ------------------------------------------------------------ CPU oracle ------
def oracle_sample_step(h: float, m: int, n: int):
    """One pass of the oracle pipeline on the sample disk; returns (nodes, seconds)."""
    import oracle
    from fixtures import disk_nodes, manufactured

    d = disk_nodes(h, SEED)
    u, f, g = manufactured(d.xy)
    t0 = time.perf_counter()
    oracle.poisson_solve(d.xy, d.is_dirichlet, f, g, m, n)
    return d.N, time.perf_counter() - t0


def oracle_batch_sample_step(seed: int, h: float, m: int, n: int, n_rhs: int):
    """The oracle on one instance of the batched workload with all its right-hand
    sides (stencils and weights once, one sparse solve per rhs); returns
    (node-rhs pairs, seconds)."""
    import oracle
    from fixtures import disk_nodes, fourier_sources

    d = disk_nodes(h, seed)
    F = fourier_sources(d.xy, n_rhs, seed)
    zero = np.zeros(d.N)
    t0 = time.perf_counter()
    idx = oracle.knn(d.xy, n)
    w, _ = oracle.weights(d.xy, idx, m)
    rp, col, val = oracle.assemble(idx, w, d.is_dirichlet)
    for k in range(n_rhs):
        oracle.solve_direct(rp, col, val, oracle.rhs(F[k], zero, d.is_dirichlet))
    return d.N * n_rhs, time.perf_counter() - t0


def batch_sample_spec():
    """The smallest instance of the batched workload (the CPU sample)."""
    from fixtures import disk_nodes

    specs = batch_specs()
    return min(specs, key=lambda sp: disk_nodes(sp[1], sp[0]).N)


def cpu_baseline_subprocess(h: float, m: int, n: int, steps: int = 1, batch: bool = False):
    """Run the oracle in a single-threaded child process (BLAS pinned to one
    thread, the paper's single-core convention)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    env.pop("CUDA_VISIBLE_DEVICES", None)
    if batch:
        code = ("import sys, json; sys.path.insert(0, %r); import bench; sp = bench.batch_sample_spec(); "
                "r = [bench.oracle_batch_sample_step(*sp, %d) for _ in range(%d)]; print(json.dumps(r))"
                % (ROOT, BATCH_SAMPLE_RHS, steps))
    else:
        code = ("import sys, json; sys.path.insert(0, %r); import bench; "
                "r = [bench.oracle_sample_step(%r, %d, %d) for _ in range(%d)]; print(json.dumps(r))"
                % (ROOT, h, m, n, steps))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def _oracle_knn_chunk(a):
    import oracle

    xy, n, q = a
    return oracle.knn_query(xy, n, q)


def _oracle_weights_chunk(a):
    import oracle

    xy, idx, m, nodes = a
    return oracle.weights(xy, idx, m, nodes=nodes)


def oracle_sample_step_parallel(h: float, m: int, n: int, procs: int):
    """The oracle pipeline of oracle_sample_step with its loops over nodes (the
    brute-force kNN and the per-stencil solves) split into contiguous chunks
    over `procs` worker processes; assembly and the sparse solve sequential.
    Returns (nodes, seconds, per-stage seconds); the pool is started before
    the clock."""
    import multiprocessing as mp

    import oracle
    from fixtures import disk_nodes, manufactured

    d = disk_nodes(h, SEED)
    u, f, g = manufactured(d.xy)
    chunks = np.array_split(np.arange(d.N), procs * 4)
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_oracle_knn_chunk, [(d.xy[:64], 4, np.arange(4))] * procs)  # start the workers
        t0 = time.perf_counter()
        idx = np.concatenate(pool.map(_oracle_knn_chunk, [(d.xy, n, c) for c in chunks]))
        t1 = time.perf_counter()
        res = pool.map(_oracle_weights_chunk, [(d.xy, idx, m, c) for c in chunks])
        t2 = time.perf_counter()
    w = np.concatenate([r[0] for r in res])
    if np.concatenate([r[1] for r in res]).any():
        raise RuntimeError("singular stencil in the CPU sample")
    rp, col, val = oracle.assemble(idx, w, d.is_dirichlet)
    oracle.solve_direct(rp, col, val, oracle.rhs(f, g, d.is_dirichlet))
    t3 = time.perf_counter()
    return d.N, t3 - t0, {"knn": t1 - t0, "weights": t2 - t1, "assemble_solve": t3 - t2}


def cpu_baseline_parallel_subprocess(h: float, m: int, n: int, procs: int):
    """oracle_sample_step_parallel in a child interpreter without the GPU, BLAS
    at one thread per worker."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_sample_step_parallel(%r, %d, %d, %d)))" % (ROOT, h, m, n, procs))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800,
                         cwd=ROOT)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload == BATCH_WORKLOAD:
        return run_reference_batched(args)
    if args.workload == EXPLICIT_WORKLOAD:
        return run_reference_explicit(args)
    if args.workload == ADJOINT_WORKLOAD:
        return run_reference_adjoint(args)
    # the sweep's reference point is m = 4, n = 30
    h, m, n = WORKLOADS[args.workload] if args.workload != SWEEP_WORKLOAD else (None, 4, 30)
    metric = SWEEP_METRIC if args.workload == SWEEP_WORKLOAD else METRIC
    res = cpu_baseline_subprocess(CPU_SAMPLE_H, m, n, steps=args.warmup + args.steps)
    timed = res[args.warmup:]
    nodes = timed[0][0]
    secs = sum(t for _, t in timed)
    value = nodes * len(timed) / secs
    sample = (f"oracle pipeline (brute-force kNN, per-stencil LU, CSR assembly, SuperLU solve) on the same "
              f"disk recipe at h={CPU_SAMPLE_H} ({nodes} nodes, m={m}, n={n}) per step")
    line = {
        "impl": "reference", "metric": metric, "value": value, "unit": "nodes/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / len(timed),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample_h": CPU_SAMPLE_H, "sample_nodes": nodes, "m": m, "n": n},
        "cpu_baseline": {"value": value, "unit": "nodes/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "nodes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def oracle_explicit_sample(h: float, m: int, n: int, steps: int):
    """The oracle's explicit step (Eq. 4) repeated on the sample disk; returns
    (node-steps, seconds of the steps alone)."""
    import oracle
    from fixtures import disk_nodes, manufactured

    d = disk_nodes(h, SEED)
    u, f, g = manufactured(d.xy)
    idx = oracle.knn(d.xy, n)
    w, _ = oracle.weights(d.xy, idx, m)
    t0 = time.perf_counter()
    for _ in range(steps):
        u = oracle.explicit_step(idx, w, d.is_dirichlet, f, u, 1e-6)
    return d.N * steps, time.perf_counter() - t0


def oracle_subprocess(call: str):
    """Runs `call` (an expression over the module bench) in a fresh one-thread
    interpreter with no GPU and returns its JSON result."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    env.pop("CUDA_VISIBLE_DEVICES", None)
    code = "import sys, json; sys.path.insert(0, %r); import bench; print(json.dumps(%s))" % (ROOT, call)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


EXPLICIT_SAMPLE_STEPS = 100


def cpu_explicit(warmup: int, steps: int):
    """(value node-steps/s, seconds per sample, sample text) of the oracle's explicit step."""
    res = oracle_subprocess("[bench.oracle_explicit_sample(%r, 4, 30, %d) for _ in range(%d)]"
                            % (CPU_SAMPLE_H, EXPLICIT_SAMPLE_STEPS, warmup + steps))[warmup:]
    units = sum(u for u, _ in res)
    secs = sum(t for _, t in res)
    sample = (f"oracle explicit step (numpy gather + einsum) on the same disk recipe at h={CPU_SAMPLE_H}, m=4, "
              f"n=30, {EXPLICIT_SAMPLE_STEPS} steps per sample, one core")
    return units / secs, secs / len(res), sample


def run_reference_explicit(args):
    value, secs, sample = cpu_explicit(args.warmup, args.steps)
    line = {
        "impl": "reference", "metric": EXPLICIT_METRIC, "value": value, "unit": "node-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample_h": CPU_SAMPLE_H, "m": 4, "n": 30, "dt": 1e-6},
        "cpu_baseline": {"value": value, "unit": "node-steps/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "node-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_batched(warmup: int, steps: int):
    """(value node-rhs/s, seconds per step, pairs per step, sample text) of the oracle on the batched sample."""
    sp = batch_sample_spec()
    timed = cpu_baseline_subprocess(0.0, 0, 0, steps=warmup + steps, batch=True)[warmup:]
    pairs = timed[0][0]
    secs = sum(t for _, t in timed)
    sample = (f"oracle (brute-force kNN, per-stencil LU, CSR assembly, one SuperLU solve per rhs) on the "
              f"smallest instance of the batched recipe ({pairs // BATCH_SAMPLE_RHS} nodes, m={sp[2]}, n={sp[3]}) "
              f"x its first {BATCH_SAMPLE_RHS} rhs per step, one core")
    return pairs * len(timed) / secs, secs / len(timed), pairs, sample


def run_reference_batched(args):
    sp = batch_sample_spec()
    value, secs, pairs, sample = cpu_batched(args.warmup, args.steps)
    line = {
        "impl": "reference", "metric": BATCH_METRIC, "value": value, "unit": "node-rhs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample_nodes": pairs // BATCH_SAMPLE_RHS, "m": sp[2], "n": sp[3],
                   "sample_rhs": BATCH_SAMPLE_RHS},
        "cpu_baseline": {"value": value, "unit": "node-rhs/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "node-rhs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------- batched workload ----
def batch_specs(count: int = 256):
    """(seed_i, h_i, m_i, n_i) of the batched workload's instances."""
    from fixtures import batched_instances

    return [(s, h, m, (m + 1) * (m + 2)) for s, h, m in batched_instances(SEED, count)]


def batch_sources_gpu(torch, xy, n_rhs: int, seed: int):
    """The fixture's Fourier sources (same draws), evaluated on the device: N x n_rhs."""
    from fixtures import fourier_params

    kx, ky, a = (torch.from_numpy(v).to(xy.device) for v in fourier_params(n_rhs, seed))
    arg = xy[:, 0, None, None] * kx[None] + xy[:, 1, None, None] * ky[None]  # N x R x waves
    return (torch.sin(arg) * a[None]).sum(dim=2).contiguous()


def run_gpu_batched(args):
    import numpy as np
    import torch

    from fixtures import disk_nodes
    from paper_2107_03632_gb300 import rbffd

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    rbffd.load()
    specs = batch_specs()
    R = BATCH_RHS
    nodes = [disk_nodes(h, s) for s, h, m, n in specs]
    sizes = [(d.N, m, n) for d, (s, h, m, n) in zip(nodes, specs)]
    N = sum(d.N for d in nodes)
    h_xy = torch.from_numpy(np.concatenate([d.xy for d in nodes])).pin_memory()
    h_mask = torch.from_numpy(np.concatenate([d.is_dirichlet for d in nodes])).pin_memory()
    xy, mask = h_xy.to(dev), h_mask.to(dev)
    F = torch.empty((N, R), dtype=torch.float64, device=dev)
    off = 0
    for d, (s, h, m, n) in zip(nodes, specs):
        F[off:off + d.N] = batch_sources_gpu(torch, xy[off:off + d.N], R, s)
        off += d.N
    G = torch.zeros_like(F)
    U = torch.zeros_like(F)
    h_F = torch.empty((N, R), dtype=torch.float64).pin_memory()
    h_F.copy_(F)
    h_U = torch.empty((N, R), dtype=torch.float64).pin_memory()
    # one-time tuning of the weight solve per (n, m), on the first instance of each
    wcfg = {}
    off = 0
    for d, (s, h, m, n) in zip(nodes, specs):
        if (n, m) not in wcfg:
            xi = xy[off:off + d.N]
            wcfg[(n, m)] = rbffd.rbffd_weights_autotune(xi, rbffd.rbffd_stencils(xi, n), m)
        off += d.N
    use_mg = args.precond == "mg"
    if use_mg:
        # per-instance multigrid; FP64 BiCGSTAB per (instance, rhs), one pass
        opts = rbffd.make_opts(tol=1e-10, precision="mixed", inner_tol=args.mg_pass_tol)
        opts.precond = 1
    else:
        opts = rbffd.make_opts(tol=1e-10, precision="mixed", inner_tol=args.inner_tol)
    wsb = rbffd.batched_workspace(sizes, R, dev, opts)

    def step():
        U.zero_()
        _, infos, st = rbffd.rbffd_solve_batched(sizes, xy, mask, F, G, U, opts, raise_on_error=False, ws=wsb)
        if st != 0:
            raise rbffd.RbffdError(st, "rbffd_solve_batched")
        return infos

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    rbffd.rbffd_profile_read(reset=True)
    rbffd.rbffd_profile_enable(True)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        infos = step()
    t1.record()
    barrier()
    clk = clocks.stop()
    prof = rbffd.rbffd_profile_read(reset=True)
    rbffd.rbffd_profile_enable(False)
    value, ms = replica_value(dist, ws, N * R, args.steps, t0.elapsed_time(t1), dev)

    e2e_value = None
    h2d = h_xy.numel() * 8 + h_mask.numel() + h_F.numel() * 8
    d2h = N * R * 8
    if args.e2e_steps > 0:
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.e2e_steps):
            xy.copy_(h_xy, non_blocking=True)
            mask.copy_(h_mask, non_blocking=True)
            F.copy_(h_F, non_blocking=True)
            step()
            h_U.copy_(U, non_blocking=True)
        e1.record()
        barrier()
        e2e_value, _ = replica_value(dist, ws, N * R, args.e2e_steps, e0.elapsed_time(e1), dev)

    status = [i["status"] for i in infos]
    line = {
        "metric": BATCH_METRIC, "value": value, "unit": "node-rhs/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "instances": len(sizes), "N_total": N, "rhs": R,
                   "m_counts": {m: sum(1 for x in sizes if x[1] == m) for m in (2, 4, 6)},
                   "tol": 1e-10, "inner_tol": args.mg_pass_tol if use_mg else args.inner_tol,
                   "precond": ("per-instance multigrid V(2,2), float32 V-cycle over all rhs, FP64 BiCGSTAB per pair"
                               if use_mg else "jacobi (float32 inner BiCGSTAB, FP64 refinement)"),
                   "parallelism": f"replicas x{ws}",
                   "weights_config": {f"n{k[0]}_m{k[1]}": v for k, v in wcfg.items()},
                   "l2": "inputs larger than L2 (vectors ~%.0f GB)" % (N * R * 8 * 8 / 1e9)},
        "solve": {"iters_max": max(i["iters"] for i in infos), "iters_mean": float(np.mean([i["iters"] for i in infos])),
                  "rounds_max": max(i["outer_sweeps"] for i in infos),
                  "worst_rel_residual": max(i["rel_residual"] for i in infos),
                  "failed_instances": sum(1 for x in status if x != 0)},
        "e2e": ({"value": e2e_value, "unit": "node-rhs/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                 "steps": args.e2e_steps} if e2e_value is not None else None),
        "gpu_launches": prof["launches"],
        "clocks": clk,
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cv, csecs, _, csample = cpu_batched(0, 1)
        line["cpu_baseline"] = {"value": cv, "unit": "node-rhs/s", "cores": 1, "kind": "oracle",
                                "sample": csample + f", {csecs:.1f} s"}
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    if prof["batch_iter_launches"]:
        it_ms = prof["batch_iter_ms"] / prof["batch_iter_launches"]
        it_by = prof["batch_iter_bytes"] / prof["batch_iter_launches"]
        gbs = it_by / (it_ms * 1e-3) / 1e9
        line["roofline"] = {"kernel": "one batched multigrid iteration (graph replay: outer FP64 kernels and every "
                                      "instance's two float32 V-cycles)", "bound": "hbm", "achieved": gbs,
                            "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "traffic": None, "peak_kind": peak_kind,
                            "bytes_per_launch": it_by, "ms_per_launch": it_ms,
                            "launches": prof["batch_iter_launches"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------ explicit workload ----
def explicit_bytes_per_step(N: int, Ni: int, n: int) -> int:
    """Algorithmic bytes of one step: the packed interior rows (n weights +
    n indices + the row id), f, u read and u written per interior row, u read
    once per node for the gathers."""
    return Ni * (n * 12 + 4 + 8 + 8 + 8) + N * 8


def run_gpu_explicit(args):
    import torch

    from fixtures import disk_nodes, h_for_nodes, manufactured
    from paper_2107_03632_gb300 import rbffd

    ws_, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws_ > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    rbffd.load()
    dt = 1e-6

    def prepare(h, m, n):
        d = disk_nodes(h, SEED)
        u, f, g = manufactured(d.xy)
        xy, mask = torch.from_numpy(d.xy).to(dev), torch.from_numpy(d.is_dirichlet).to(dev)
        idx = rbffd.rbffd_stencils(xy, n)
        w, _ = rbffd.rbffd_weights(xy, idx, m)
        loop = rbffd.ExplicitLoop(idx, w, mask)
        return d, loop, torch.from_numpy(f).to(dev), torch.from_numpy(u).to(dev)

    def time_steps(loop, fT, uT, steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record()
        loop.run(fT, uT, dt, steps)
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1)

    h, m, n = 1.7725e-3, 4, 30
    d, loop, fT, uT = prepare(h, m, n)
    steps = 1024 * max(args.steps, 1)
    for _ in range(args.warmup):
        loop.run(fT, uT, dt, 256)
    clocks = ClockSampler(local)
    clocks.start()
    rbffd.rbffd_profile_read(reset=True)
    ms = time_steps(loop, fT, uT, steps)
    clk = clocks.stop()
    prof = rbffd.rbffd_profile_read(reset=True)
    value, ms = replica_value(dist, ws_, d.N, steps, ms, dev)
    by = explicit_bytes_per_step(d.N, loop.n_interior, n)
    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])
    gbs = by / (ms / steps * 1e-3) / 1e9
    # e2e: the same loop through the API from pinned host buffers
    h_u = torch.from_numpy(manufactured(d.xy)[0]).pin_memory()
    h_out = torch.empty_like(h_u).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record()
    uT.copy_(h_u, non_blocking=True)
    loop.run(fT, uT, dt, steps)
    h_out.copy_(uT, non_blocking=True)
    e1.record()
    torch.cuda.synchronize(dev)
    e2e_value, _ = replica_value(dist, ws_, d.N, steps, e0.elapsed_time(e1), dev)

    sweep = []
    if not args.no_sweep:
        for nn in EXPLICIT_SWEEP_n:
            for Nt in EXPLICIT_SWEEP_N:
                ds, lp, fs, us = prepare(h_for_nodes(Nt), 2, nn)
                lp.run(fs, us, dt, 128)
                k = 512
                t = time_steps(lp, fs, us, k)
                b = explicit_bytes_per_step(ds.N, lp.n_interior, nn)
                sweep.append({"n": nn, "N": ds.N, "ns_per_node_step": t * 1e6 / (k * ds.N),
                              "gbs": b / (t / k * 1e-3) / 1e9,
                              "table1_bytes": 8 * ds.N * (4 + nn) + 4 * (lp.n_interior + ds.N * nn)})
                del ds, lp, fs, us
    line = {
        "metric": EXPLICIT_METRIC, "value": value, "unit": "node-steps/s", "n_gpus": ws_, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": EXPLICIT_WORKLOAD, "N": d.N, "N_interior": loop.n_interior, "m": m, "n": n,
                   "dt": dt, "parallelism": f"replicas x{ws_}",
                   "l2": "inputs larger than L2 (%.0f MB per step)" % (by / 1e6)},
        "roofline": {"kernel": "explicit_step_kernel (packed ELL, one thread per interior row)", "bound": "hbm",
                     "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm, "traffic": None,
                     "peak_kind": peak_kind, "bytes_per_launch": by, "ms_per_launch": ms / steps, "launches": steps},
        "e2e": {"value": e2e_value, "unit": "node-steps/s", "h2d_bytes_per_step": d.N * 8 / steps,
                "d2h_bytes_per_step": d.N * 8 / steps, "steps": steps},
        "gpu_launches": prof["launches"],
        "clocks": clk,
        "sweep": sweep,
    }
    if rank == 0 and ws_ == 1 and not args.no_cpu_baseline:
        cv, csecs, csample = cpu_explicit(0, 1)
        line["cpu_baseline"] = {"value": cv, "unit": "node-steps/s", "cores": 1, "kind": "oracle",
                                "sample": csample + f", {csecs:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------- adjoint workload ----
def run_gpu_adjoint(args):
    import numpy as np
    import torch

    from fixtures import disk_nodes, fourier_sources, manufactured
    from paper_2107_03632_gb300 import rbffd

    ws_, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws_ > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    rbffd.load()
    h, m, n = 1.7725e-3, 4, 30
    d = disk_nodes(h, SEED)
    N = d.N
    u_ex, f, g = manufactured(d.xy)
    fstar = fourier_sources(d.xy, 1, SEED + 1)[0]
    xy, mask = torch.from_numpy(d.xy).to(dev), torch.from_numpy(d.is_dirichlet).to(dev)
    fT, gT, fsT = (torch.from_numpy(a).to(dev) for a in (f, g, fstar))
    idx = rbffd.rbffd_stencils(xy, n)
    wcfg = rbffd.rbffd_weights_autotune(xy, idx, m)
    w, st = rbffd.rbffd_weights(xy, idx, m)
    A = rbffd.rbffd_assemble(idx, w, mask, want_f32=True)
    AT = rbffd.rbffd_transpose(A, want_f32=True)
    mg = rbffd.Multigrid(xy, mask, A)
    galerkin = args.adjoint_mg == "galerkin"
    mga = (rbffd.Multigrid.galerkin_adjoint_of if galerkin else rbffd.Multigrid.adjoint_of)(mg, AT)
    opts = rbffd.make_opts(tol=1e-10, precision="mixed", mg=mg)
    opts_a = rbffd.make_opts(tol=1e-10, precision="mixed", mg=mga)
    ws_s = rbffd.solve_workspace(N, opts, dev)
    # target u* (fixed, outside the timed steps)
    ustar, _ = rbffd.rbffd_solve(A, rbffd.rbffd_rhs(fsT, gT, mask), opts=opts, ws=ws_s)
    b = torch.empty(N, dtype=torch.float64, device=dev)
    u = torch.empty(N, dtype=torch.float64, device=dev)
    lam = torch.empty(N, dtype=torch.float64, device=dev)
    dLdu = torch.empty(N, dtype=torch.float64, device=dev)
    ws_knn = rbffd.stencils_workspace(N, n, dev)
    ws_asm = rbffd.assemble_workspace(N, dev)

    stage_names = ("stencils", "weights", "assemble_transpose_rhs", "mg_setup_forward", "mg_setup_adjoint",
                   "forward_solve", "adjoint_solve")

    def step(ev=None):
        mark = (lambda k: ev[k].record()) if ev is not None else (lambda k: None)
        mark(0)
        rbffd.rbffd_stencils(xy, n, idx, ws_knn)
        mark(1)
        rbffd.rbffd_weights(xy, idx, m, w, st)
        mark(2)
        rbffd.rbffd_assemble_pattern(mask, n, A.row_ptr, ws_asm)
        rbffd.rbffd_assemble(idx, w, mask, out=A)
        AT2 = rbffd.rbffd_transpose(A, want_f32=True)
        rbffd.rbffd_rhs(fT, gT, mask, b)
        mark(3)
        mg.setup(xy, mask, A)
        mark(4)
        mga.rebuild_from(mg, AT2)
        mark(5)
        u.zero_()
        _, info = rbffd.rbffd_solve(A, b, u, opts, ws_s, raise_on_error=False)
        mark(6)
        rbffd.rbffd_misfit_grad(u, ustar, mask, dLdu)
        lam.zero_()
        _, dLdf, dLdg, info_a = rbffd.rbffd_solve_adjoint(AT2, mask, dLdu, lam, opts_a, ws_s, raise_on_error=False)
        mark(7)
        if info["status_code"] != 0 or info_a["status_code"] != 0:
            raise rbffd.RbffdError(max(info["status_code"], info_a["status_code"]), "differentiable solve",
                                   f"{info} {info_a}")
        return info, info_a, dLdf, dLdg

    for _ in range(args.warmup):
        step()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize(dev)
    rbffd.rbffd_profile_read(reset=True)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        info, info_a, dLdf, dLdg = step()
    t1.record()
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    prof = rbffd.rbffd_profile_read(reset=True)
    value, ms = replica_value(dist, ws_, N, args.steps, t0.elapsed_time(t1), dev)
    # stage times: one more (untimed) step with events between the stages
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(stage_names) + 1)]
    step(evs)
    torch.cuda.synchronize(dev)
    stages = {k: evs[i].elapsed_time(evs[i + 1]) for i, k in enumerate(stage_names)}
    # e2e: geometry, sources, boundary data and the target from pinned host
    # memory, both gradients back, every step
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    h_xy, h_mask, h_f, h_g, h_us = pin(d.xy), pin(d.is_dirichlet), pin(f), pin(g), pin(ustar.cpu().numpy())
    h_df = torch.empty(N, dtype=torch.float64).pin_memory()
    h_dg = torch.empty(N, dtype=torch.float64).pin_memory()
    h2d = N * (16 + 1 + 8 + 8 + 8)
    d2h = 2 * N * 8
    e2e_value = None
    if args.e2e_steps > 0:
        if dist is not None:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.e2e_steps):
            xy.copy_(h_xy, non_blocking=True)
            mask.copy_(h_mask, non_blocking=True)
            fT.copy_(h_f, non_blocking=True)
            gT.copy_(h_g, non_blocking=True)
            ustar.copy_(h_us, non_blocking=True)
            _, _, dLdf, dLdg = step()
            h_df.copy_(dLdf, non_blocking=True)
            h_dg.copy_(dLdg, non_blocking=True)
        e1.record()
        torch.cuda.synchronize(dev)
        e2e_value, _ = replica_value(dist, ws_, N, args.e2e_steps, e0.elapsed_time(e1), dev)
    cpu = None
    if rank == 0 and ws_ == 1 and not args.no_cpu_baseline:
        cv, csecs, cnodes, csample = cpu_adjoint(0, 1)
        cpu = {"value": cv, "unit": "nodes/s", "cores": 1, "kind": "oracle", "sample": csample + f", {csecs:.1f} s"}
    line = {
        "metric": ADJOINT_METRIC, "value": value, "unit": "nodes/s", "n_gpus": ws_, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": ADJOINT_WORKLOAD, "N": N, "m": m, "n": n, "tol": 1e-10,
                   "precond": ("multigrid (forward) and " +
                               ("Galerkin multigrid, right-preconditioned" if galerkin else
                                "transposed multigrid, left-preconditioned") + " (adjoint), float32 V-cycles"),
                   "weights_config": wcfg, "parallelism": f"replicas x{ws_}",
                   "l2": "inputs larger than L2 (CSR + transpose ~%.1f GB)" % (2 * A.nnz * 16 / 1e9)},
        "solve": {"forward_iters": info["iters"], "adjoint_iters": info_a["iters"],
                  "forward_rel_residual": info["rel_residual"], "adjoint_rel_residual": info_a["rel_residual"],
                  "grad_f_norm": float(dLdf.norm()), "grad_g_norm": float(dLdg.norm())},
        "stages_ms": stages,
        "roofline": weights_roofline(wcfg["kernel"], n, m, N, stages["weights"], {}),
        "e2e": ({"value": e2e_value, "unit": "nodes/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                 "steps": args.e2e_steps} if e2e_value is not None else None),
        "cpu_baseline": cpu,
        "gpu_launches": prof["launches"],
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def oracle_adjoint_sample(h: float, m: int, n: int):
    """The oracle's differentiable solve on the sample disk: forward direct
    solve, misfit gradient, adjoint direct solve; returns (nodes, seconds)."""
    import oracle
    from fixtures import disk_nodes, fourier_sources, manufactured

    d = disk_nodes(h, SEED)
    u, f, g = manufactured(d.xy)
    fstar = fourier_sources(d.xy, 1, SEED + 1)[0]
    ustar, _ = oracle.poisson_solve(d.xy, d.is_dirichlet, fstar, g, m, n)
    t0 = time.perf_counter()
    uu, (idx, w, rp, col, val, b) = oracle.poisson_solve(d.xy, d.is_dirichlet, f, g, m, n)
    dLdu = np.where(d.is_dirichlet == 1, 0.0, 2.0 * (uu - ustar))
    oracle.adjoint_gradient(rp, col, val, d.is_dirichlet, dLdu)
    return d.N, time.perf_counter() - t0


def cpu_adjoint(warmup: int, steps: int):
    """(value nodes/s, seconds per step, sample nodes, sample text) of the oracle's differentiable solve."""
    res = oracle_subprocess("[bench.oracle_adjoint_sample(%r, 4, 30) for _ in range(%d)]"
                            % (CPU_SAMPLE_H, warmup + steps))[warmup:]
    nodes = res[0][0]
    secs = sum(t for _, t in res)
    sample = (f"oracle differentiable solve (brute-force kNN, per-stencil LU, SuperLU forward and adjoint solves) "
              f"on the same disk recipe at h={CPU_SAMPLE_H} ({nodes} nodes, m=4, n=30), one core")
    return nodes * len(res) / secs, secs / len(res), nodes, sample


def run_reference_adjoint(args):
    value, secs, nodes, sample = cpu_adjoint(args.warmup, args.steps)
    line = {
        "impl": "reference", "metric": ADJOINT_METRIC, "value": value, "unit": "nodes/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample_h": CPU_SAMPLE_H, "sample_nodes": nodes, "m": 4, "n": 30},
        "cpu_baseline": {"value": value, "unit": "nodes/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "nodes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------- support sweep ----
def run_gpu_sweep(args):
    """Per (n, m): stencils, autotuned weights, assembly, multigrid setup and
    the mixed multigrid solve (tol 1e-10) on the 1M-node disk; CUDA-event
    stage times (median of args.steps runs after args.warmup)."""
    import torch

    from fixtures import disk_nodes, manufactured
    from paper_2107_03632_gb300 import rbffd

    ws_, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rbffd.load()
    h = 1.7725e-3
    d = disk_nodes(h, SEED)
    N = d.N
    _, f, g = manufactured(d.xy)
    xy, mask = torch.from_numpy(d.xy).to(dev), torch.from_numpy(d.is_dirichlet).to(dev)
    fT, gT = torch.from_numpy(f).to(dev), torch.from_numpy(g).to(dev)
    clocks = ClockSampler(local)
    clocks.start()
    points = []
    for m in SWEEP_M:
        s = (m + 1) * (m + 2) // 2
        for n in SWEEP_N:
            if n < s:
                continue
            idx = rbffd.rbffd_stencils(xy, n)
            cfg = rbffd.rbffd_weights_autotune(xy, idx, m)
            w, st = rbffd.rbffd_weights(xy, idx, m)
            A = rbffd.rbffd_assemble(idx, w, mask, want_f32=True)
            mg = rbffd.Multigrid(xy, mask, A)
            opts = rbffd.make_opts(tol=1e-10, precision="mixed", mg=mg)
            wsol = rbffd.solve_workspace(N, opts, dev)
            b = rbffd.rbffd_rhs(fT, gT, mask)
            u = torch.zeros(N, dtype=torch.float64, device=dev)
            times = {k: [] for k in ("stencils", "weights", "assemble", "mg_setup", "solve")}
            info = None
            for r in range(args.warmup + args.steps):
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
                ev[0].record()
                rbffd.rbffd_stencils(xy, n, idx)
                ev[1].record()
                rbffd.rbffd_weights(xy, idx, m, w, st)
                ev[2].record()
                rbffd.rbffd_assemble(idx, w, mask, out=A)
                ev[3].record()
                mg.setup(xy, mask, A)
                ev[4].record()
                u.zero_()
                _, info = rbffd.rbffd_solve(A, b, u, opts, wsol, raise_on_error=False)
                ev[5].record()
                torch.cuda.synchronize(dev)
                if r >= args.warmup:
                    for i, k in enumerate(times):
                        times[k].append(ev[i].elapsed_time(ev[i + 1]))
            # a point whose solve does not reach 1e-10 (or has singular stencils)
            # is reported with its status, not dropped
            status = rbffd.STATUS_NAMES.get(info["status_code"], str(info["status_code"]))
            if int(st.sum()) != 0:
                status = f"{int(st.sum())} singular stencils"
            med = {k: float(np.median(v)) for k, v in times.items()}
            roof = weights_roofline(cfg["kernel"], n, m, N, med["weights"], {})
            points.append({"n": n, "m": m, "s": s, "status": status, "stages_ms": med, "iters": info["iters"],
                           "rel_residual": info["rel_residual"], "weights_config": cfg,
                           "weights_ns_per_node": 1e6 * med["weights"] / N,
                           "weights_roofline_frac": roof["frac"], "weights_roofline_unit": roof["unit"],
                           "fp64_equivalent_tflops": weights_flops(n, m) * N / (med["weights"] * 1e-3) / 1e12,
                           "nodes_per_s_weights_solve": N / ((med["weights"] + med["assemble"] + med["mg_setup"]
                                                              + med["solve"]) * 1e-3)})
            print(json.dumps({"sweep_point": points[-1]}), file=sys.stderr, flush=True)
            del A, mg, w, st, idx, wsol
            torch.cuda.empty_cache()
    clk = clocks.stop()
    ref = next(p for p in points if p["n"] == 30 and p["m"] == 4)
    line = {
        "metric": SWEEP_METRIC, "value": ref["nodes_per_s_weights_solve"], "unit": "nodes/s", "n_gpus": ws_,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * N / ref["nodes_per_s_weights_solve"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": SWEEP_WORKLOAD, "N": N, "h": h, "n": list(SWEEP_N), "m": list(SWEEP_M),
                   "timing": "median over steps of CUDA-event stage times", "parallelism": f"replicas x{ws_}",
                   "l2": "inputs larger than L2 at n >= 30 (CSR >= 0.36 GB)"},
        "sweep": points, "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm -----
def run_gpu(args):
    import numpy as np
    import torch

    from fixtures import disk_nodes, manufactured
    from paper_2107_03632_gb300 import rbffd

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    rbffd.load()

    h, m, n = WORKLOADS[args.workload]
    d = disk_nodes(h, SEED)
    u_ex, f, g = manufactured(d.xy)
    N = d.N
    s = (m + 1) * (m + 2) // 2
    M = n + s

    # host (pinned) and device buffers
    h_xy = torch.from_numpy(d.xy).pin_memory()
    h_mask = torch.from_numpy(d.is_dirichlet).pin_memory()
    h_f = torch.from_numpy(f).pin_memory()
    h_g = torch.from_numpy(g).pin_memory()
    h_u = torch.empty(N, dtype=torch.float64).pin_memory()
    xy, mask = h_xy.to(dev), h_mask.to(dev)
    fT, gT = h_f.to(dev), h_g.to(dev)
    idx = torch.empty((N, n), dtype=torch.int32, device=dev)
    w = torch.empty((N, n), dtype=torch.float64, device=dev)
    st = torch.empty(N, dtype=torch.int32, device=dev)
    b = torch.empty(N, dtype=torch.float64, device=dev)
    x = torch.empty(N, dtype=torch.float64, device=dev)
    ws_knn = rbffd.stencils_workspace(N, n, dev)
    ws_asm = rbffd.assemble_workspace(N, dev)
    row_ptr = rbffd.rbffd_assemble_pattern(mask, n, ws=ws_asm)
    nnz = int(row_ptr[-1].item())
    A = rbffd.CsrMatrix(row_ptr, torch.empty(nnz, dtype=torch.int32, device=dev),
                        torch.empty(nnz, dtype=torch.float64, device=dev),
                        torch.empty(nnz, dtype=torch.float32, device=dev))
    # one-time tuning of the weight solve's launch configuration for (n, m):
    # the double-float candidates (for the labelled df leg), then the FP64
    # ones, which stay in force for the headline
    rbffd.rbffd_stencils(xy, n, idx, ws_knn)
    wcfg_df = rbffd.rbffd_weights_autotune(xy, idx, m, "df") if (args.df_steps > 0 and m <= 6) else None
    if args.weights_config:  # pinned, e.g. "null-space-4warp:4" (profiling runs)
        kern, wpb = args.weights_config.split(":")
        rbffd.set_weights_config(n, m, kern, int(wpb))
        wcfg = rbffd.weights_config(n, m)
    elif args.no_autotune:  # the library's default configuration (FP64)
        wcfg = rbffd.weights_config(n, m)
    else:
        wcfg = rbffd.rbffd_weights_autotune(xy, idx, m, "fp64")

    def use_weights(cfg):
        rbffd.set_weights_config(n, m, cfg["kernel"], cfg["warps_per_block"])

    use_mg = args.precond == "mg"
    mg = None
    if use_mg:
        # first build (allocates the hierarchy's workspace); every step rebuilds it
        rbffd.rbffd_stencils(xy, n, idx, ws_knn)
        rbffd.rbffd_weights(xy, idx, m, w, st)
        rbffd.rbffd_assemble(idx, w, mask, out=A)
        mg = rbffd.Multigrid(xy, mask, A, nu=args.mg_nu, omega=args.mg_omega)
        opts = {"mixed": rbffd.make_opts(tol=args.tol, precision="mixed", inner_tol=args.mg_pass_tol, mg=mg),
                "fp64": rbffd.make_opts(tol=args.tol, precision="fp64", inner_tol=args.mg_pass_tol, mg=mg)}
    else:
        opts = {"mixed": rbffd.make_opts(tol=args.tol, precision="mixed", inner_tol=args.inner_tol),
                "fp64": rbffd.make_opts(tol=args.tol, precision="fp64", inner_tol=args.inner_tol64)}
    ws_solve = rbffd.solve_workspace(N, opts["mixed"], dev)
    if use_mg:
        ws_solve64 = ws_solve
    else:
        ws_solve64 = rbffd.solve_workspace(N, opts["fp64"], dev)

    # --mg-overlap: the hierarchy's geometry (coarse node sets, their
    # operators, transfers) depends on the nodes and the mask only, so it can
    # be built on a second stream while the fine weights are solved, and the
    # fine operator attached after (measured: +0.7 % per step, the weight
    # solve slowed by the kernels sharing its SMs; off by default)
    side = torch.cuda.Stream(dev) if (mg is not None and args.mg_overlap) else None
    geom_ms = []

    def step(precision, ev=None):
        main = torch.cuda.current_stream(dev)
        if side is not None:
            ready = torch.cuda.Event()
            ready.record(main)  # the step's inputs are in place
        if ev:
            ev[0].record()
        rbffd.rbffd_stencils(xy, n, idx, ws_knn)
        if ev:
            ev[1].record()
        rbffd.rbffd_weights(xy, idx, m, w, st)
        if ev:
            ev[2].record()
        if side is not None:
            side.wait_event(ready)
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(side)
            mg.setup_geometry(xy, mask, nu=args.mg_nu, omega=args.mg_omega, stream=side)  # host waits here
            g1.record(side)
            if ev:
                geom_ms.append((g0, g1))
        rbffd.rbffd_assemble_pattern(mask, n, row_ptr, ws_asm)
        rbffd.rbffd_assemble(idx, w, mask, out=A)
        rbffd.rbffd_rhs(fT, gT, mask, b)
        if ev:
            ev[3].record()
        if mg is not None:
            if side is not None:
                mg.setup_operator(A)
            else:
                mg.setup(xy, mask, A, nu=args.mg_nu, omega=args.mg_omega)
        if ev:
            ev[4].record()
        x.zero_()
        _, info = rbffd.rbffd_solve(A, b, x, opts[precision], ws_solve if precision == "mixed" else ws_solve64,
                                    raise_on_error=False)
        if info["status_code"] != 0:  # a step that did not reach the tolerance measures nothing
            raise rbffd.RbffdError(info["status_code"], "rbffd_solve", f"{info}")
        if ev:
            ev[5].record()
        return info

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed_loop(precision, k, profile=False):
        """k steps bracketed by events; per-stage events (six records per step,
        on the launching stream) give the stage times; profile=True also
        brackets every SpMV and finest V-cycle sweep (a separate loop)."""
        stage = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(k)]
        infos = []
        geom_ms.clear()
        barrier()
        rbffd.rbffd_profile_read(reset=True)
        if profile:
            rbffd.rbffd_profile_enable(True)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        wall0 = time.perf_counter()
        t0.record()
        for i in range(k):
            infos.append(step(precision, stage[i]))
        t1.record()
        barrier()
        wall = time.perf_counter() - wall0
        prof = rbffd.rbffd_profile_read(reset=True)
        rbffd.rbffd_profile_enable(False)
        ms = t0.elapsed_time(t1)
        st_ms = np.array([[stage[i][j].elapsed_time(stage[i][j + 1]) for j in range(5)] for i in range(k)]).mean(0)
        if geom_ms:  # the geometry phase's own time on the second stream
            st_ms = np.append(st_ms, np.mean([a.elapsed_time(b_) for a, b_ in geom_ms]))
        return ms, wall, st_ms, infos, prof

    def stages(st_ms):
        out = {"stencils": st_ms[0], "weights": st_ms[1], "assemble_rhs": st_ms[2], "mg_setup": st_ms[3],
               "solve": st_ms[4]}
        if len(st_ms) > 5:  # the hierarchy built in two phases
            out["mg_setup"] = st_ms[3]
            out["mg_geometry_overlapped"] = st_ms[5]
            out["note"] = ("mg_geometry_overlapped: the hierarchy's geometry phase on a second stream, "
                           "concurrent with the weights; mg_setup: the fine-operator phase after assembly")
        return out

    def solve_summary(infos):
        return {"iters": [i["iters"] for i in infos], "passes": [i["outer_sweeps"] for i in infos],
                "status": [rbffd.STATUS_NAMES.get(i["status_code"], i["status_code"]) for i in infos],
                "rel_residual": [i["rel_residual"] for i in infos]}

    # ---- warm-up, then the timed steps: FP64 weights, mixed solve ----------
    for _ in range(args.warmup):
        step("mixed")
    clocks = ClockSampler(local)
    clocks.start()
    ms, wall, st_ms, infos, prof_main = timed_loop("mixed", args.steps)
    value, ms = replica_value(dist, ws, N, args.steps, ms, dev)
    ms_step = ms / args.steps

    # ---- the same steps with the FP64 solve (FP64 V-cycle) ------------------
    k64 = args.fp64_steps if args.fp64_steps is not None else args.steps
    fp64_line = None
    if k64 > 0:
        step("fp64")
        ms64, wall64, st64, infos64, _ = timed_loop("fp64", k64)
        value64, ms64 = replica_value(dist, ws, N, k64, ms64, dev)
        fp64_line = {"value": value64, "ms_per_step": ms64 / k64, "steps": k64,
                     "precision": "FP64 weights, FP64 BiCGSTAB right-preconditioned by an FP64 V-cycle",
                     "stages_ms": stages(st64), **solve_summary(infos64)}
    clk = clocks.stop()

    # ---- labelled extra: the same mixed step with double-float weights ------
    df_line = None
    kdf = min(args.df_steps, args.steps)
    if wcfg_df is not None and kdf > 0:
        use_weights(wcfg_df)
        step("mixed")
        msdf, _, stdf, infosdf, _ = timed_loop("mixed", kdf)
        use_weights(wcfg)
        valuedf, msdf = replica_value(dist, ws, N, kdf, msdf, dev)
        df_line = {"value": valuedf, "ms_per_step": msdf / kdf, "steps": kdf, "weights_precision": "df32",
                   "weights_config": wcfg_df,
                   "note": ("weight solves in double-float arithmetic (pairs of floats, ~48 significant bits, "
                            "FP32 pipe); not the FP64 weights the headline uses"),
                   "stages_ms": stages(stdf),
                   "weights_roofline": weights_roofline(wcfg_df["kernel"], n, m, N, stdf[1], {}),
                   **solve_summary(infosdf)}

    # ---- per-kernel figures of the solve: a separate, profiled loop ---------
    kp = max(1, min(2, args.steps))
    _, _, _, _, prof = timed_loop("mixed", kp, profile=True)
    prof64 = None
    if k64 > 0:
        _, _, _, _, prof64 = timed_loop("fp64", kp, profile=True)

    # ---- end to end through the API from pinned host buffers ----
    h2d = (h_xy.numel() * 8 + h_mask.numel() + h_f.numel() * 8 + h_g.numel() * 8)
    d2h = N * 8
    e2e_value = None
    if args.e2e_steps > 0:
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.e2e_steps):
            xy.copy_(h_xy, non_blocking=True)
            mask.copy_(h_mask, non_blocking=True)
            fT.copy_(h_f, non_blocking=True)
            gT.copy_(h_g, non_blocking=True)
            step("mixed")
            h_u.copy_(x, non_blocking=True)
        e1.record()
        barrier()
        e2e_value, _ = replica_value(dist, ws, N, args.e2e_steps, e0.elapsed_time(e1), dev)
    else:
        h_u.copy_(x)

    # ---- correctness of the timed solves (host check, outside timing) ----
    err_exact = float(np.abs(h_u.numpy() - u_ex).max())

    peaks, peak_kind = measured_peaks()
    hbm = float(peaks["hbm_gbs"])

    def per_launch(pr, kind):
        nl = pr[kind + "_launches"]
        if not nl:
            return 0.0, 0.0, 0.0, 0
        ms_ = pr[kind + "_ms"] / nl
        by = pr[kind + "_bytes"] / nl
        return ms_, by, by / (ms_ * 1e-3) / 1e9, nl

    dom = "mg" if use_mg else "spmv32"
    sp_ms, sp_bytes, sp_gbs, sp_n = per_launch(prof, dom)
    dom_name = ("mg_jacobi_kernel<float> (finest-level damped Jacobi sweep of the float32 V-cycle)" if use_mg
                else "spmv_df_kernel (inner BiCGSTAB SpMV, float32 values)")
    outer_ms, outer_bytes, outer_gbs, outer_n = per_launch(prof, "spmv64")
    if fp64_line is not None:
        sp64_ms, sp64_bytes, sp64_gbs, _ = per_launch(prof64, "mg" if use_mg else "spmv64")
        o64_ms, o64_bytes, o64_gbs, _ = per_launch(prof64, "spmv64")
        fp64_line.update({
            "dominant_solve_kernel": ("mg_jacobi_kernel<double> (finest-level sweep, FP64 V-cycle)" if use_mg
                                      else "spmv64_kernel"),
            "dominant_gbs": sp64_gbs, "dominant_frac_hbm": sp64_gbs / hbm, "dominant_ms_per_launch": sp64_ms,
            "spmv64_gbs": o64_gbs, "spmv64_frac_hbm": o64_gbs / hbm, "spmv64_ms_per_launch": o64_ms})

    fp64_peak = fp64_peak_tflops(torch, dev) if not args.no_peak_probe else float("nan")
    lu_equiv = N * (2.0 / 3.0 * M ** 3 + 2.0 * M * M) / (st_ms[1] * 1e-3) / 1e12

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        res = cpu_baseline_subprocess(CPU_SAMPLE_H, m, n, steps=1)
        nodes, secs = res[0]
        cpu = {"value": nodes / secs, "unit": "nodes/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle pipeline (brute-force kNN, per-stencil LU, CSR assembly, SuperLU) on the same "
                         f"disk recipe at h={CPU_SAMPLE_H} ({nodes} nodes, m={m}, n={n}), one core, {secs:.1f} s"}
        procs = os.cpu_count() or 1
        resp = cpu_baseline_parallel_subprocess(CPU_SAMPLE_H, m, n, procs)
        nodes_p, secs_p, stage_p = resp
        cpu["all_cores"] = {
            "value": nodes_p / secs_p, "unit": "nodes/s", "cores": procs, "nproc": procs,
            "sample": (f"the same oracle pipeline with kNN and weights split over {procs} worker processes "
                       f"(one thread each), assembly and SuperLU sequential; {secs_p:.1f} s"),
            "stages_s": stage_p}

    roof_solve = {"kernel": dom_name, "bound": "hbm", "achieved": sp_gbs,
                  "peak": hbm, "unit": "GB/s", "frac": sp_gbs / hbm,
                  "traffic": (None if use_mg else
                              (SPMV_DF_TRAFFIC["traffic_over_algorithmic"] * sp_bytes
                               if spmv_df_source_hash() == SPMV_DF_TRAFFIC["source_sha256_16"] else None)),
                  "peak_kind": peak_kind, "bytes_per_launch": sp_bytes, "ms_per_launch": sp_ms,
                  "launches": sp_n, "ms_per_step": sp_ms * sp_n / max(kp, 1),
                  "measured_in": "separate profiled loop (events around every sweep)"}
    roof_weights = weights_roofline(wcfg["kernel"], n, m, N, st_ms[1],
                                    {"cublas_dgemm_tflops": fp64_peak,
                                     "frac_of_dgemm": (weights_flops(n, m) * N / (st_ms[1] * 1e-3) / 1e12
                                                       / fp64_peak if fp64_peak == fp64_peak else None),
                                     "lu_equivalent_tflops": lu_equiv,
                                     "measured_in": "timed region (events around the weights launch)"})
    weights_dominate = st_ms[1] > roof_solve["ms_per_step"]
    line = {
        "metric": METRIC, "value": value, "unit": "nodes/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": args.workload, "N": N, "nnz": nnz, "h": h, "m": m, "n": n, "seed": SEED,
                   "tol": args.tol,
                   "precision_by_stage": {
                       "stencils": "f64 distance keys (f32 pruning bounds)",
                       "weights": "f64 (null-space elimination + L D L^T, FP64 throughout)",
                       "assembly": "f64 values (+ f32 copy for the preconditioner)",
                       "krylov": "f64 BiCGSTAB, f64 residual and updates",
                       "preconditioner": ("float32 multigrid V-cycle (coarse weights in double-float)" if use_mg
                                          else "f32 inner BiCGSTAB inside f64 refinement")},
                   "precision": ("mixed: FP64 BiCGSTAB right-preconditioned by a float32 multigrid V-cycle "
                                 "(float32 preconditioner)" if use_mg else
                                 "mixed (f32 inner BiCGSTAB, f64 refinement)"),
                   "precond": (f"multigrid V({args.mg_nu},{args.mg_nu}) omega {args.mg_omega}, levels "
                               f"{mg.levels()}" if use_mg else "jacobi"),
                   "inner_tol": args.mg_pass_tol if use_mg else args.inner_tol,
                   "mg_setup": (None if not use_mg else
                                "one call after assembly" if side is None else
                                "geometry phase on a second stream during the weight solve, then the fine operator"),
                   "parallelism": f"replicas x{ws}", "weights_config": wcfg, "weights_precision": "f64",
                   "l2": "inputs larger than L2 (CSR ~%.1f GB)" % ((nnz * 16) / 1e9)},
        "stages_ms": stages(st_ms),
        "solve": {**solve_summary(infos), "max_err_vs_exact": err_exact},
        "fp64": fp64_line,
        "df_weights": df_line,
        # the dominant kernel of the step (largest device time) and the solver's own
        "roofline": roof_weights if weights_dominate else roof_solve,
        "solve_roofline": roof_solve if weights_dominate else roof_weights,
        "outer_spmv": {"kernel": "spmv64_kernel (outer BiCGSTAB SpMV, float64 values)", "achieved_gbs": outer_gbs,
                       "frac": outer_gbs / hbm, "ms_per_launch": outer_ms, "launches": outer_n},
        "e2e": ({"value": e2e_value, "unit": "nodes/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                 "steps": args.e2e_steps} if e2e_value is not None else None),
        "gpu_launches": prof_main["launches"],
        "clocks": clk,
        "cpu_baseline": cpu,
        "wall_s_timed": wall,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="disk_4M_m6_n56",
                    choices=sorted(WORKLOADS) + [BATCH_WORKLOAD, EXPLICIT_WORKLOAD, ADJOINT_WORKLOAD, SWEEP_WORKLOAD])
    ap.add_argument("--no-sweep", action="store_true", help="explicit workload: skip the N x n sweep")
    ap.add_argument("--inner-tol", type=float, default=1e-5, help="mixed: residual drop per refinement pass")
    ap.add_argument("--inner-tol64", type=float, default=1e-3, help="FP64: residual drop per restarted pass")
    ap.add_argument("--precond", default="mg", choices=["mg", "jacobi"],
                    help="mg: BiCGSTAB right-preconditioned by the multigrid V-cycle; jacobi: the plain solvers")
    ap.add_argument("--mg-nu", type=int, default=2, help="Jacobi sweeps before and after the coarse correction")
    ap.add_argument("--mg-omega", type=float, default=0.6, help="Jacobi damping of the V-cycle")
    ap.add_argument("--mg-overlap", action="store_true",
                    help="build the multigrid hierarchy's geometry on a second stream during the weight solve "
                         "(default: the whole hierarchy in one call after assembly)")
    ap.add_argument("--mg-pass-tol", type=float, default=1e-10,
                    help="multigrid: residual drop per restarted BiCGSTAB pass (1e-10: a single pass)")
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="timed steps with the FP64 solve (default: --steps; 0: skip)")
    ap.add_argument("--df-steps", type=int, default=5,
                    help="timed steps with double-float weights, a labelled extra (at most --steps; 0: skip)")
    ap.add_argument("--adjoint-mg", default="galerkin", choices=["galerkin", "transposed"],
                    help="adjoint workload: the adjoint hierarchy (Galerkin coarse operators, or the transposed "
                         "forward cycle)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default FP64 weight-solve configuration (profiling runs)")
    ap.add_argument("--weights-config", default=None,
                    help="pin the weight-solve configuration KERNEL:WARPS_PER_BLOCK instead of autotuning")
    ap.add_argument("--no-peak-probe", action="store_true", help="skip the cuBLAS DGEMM FP64 peak probe")
    ap.add_argument("--config", default=None,
                    help="a JSON workload {\"h\": spacing or \"N\": nodes, \"m\", \"n\", optional \"seed\", "
                         "\"tol\", \"name\"} for the single-system step, instead of --workload")
    ap.add_argument("--seed", type=int, default=None, help="seed of the node sets and sources (default 2107)")
    ap.add_argument("--tol", type=float, default=1e-10,
                    help="relative residual of the single-system solves (default 1e-10, the metric's)")
    args = ap.parse_args()
    global SEED
    if args.config:
        with open(args.config) as fh:
            c = json.load(fh)
        from fixtures import h_for_nodes

        h = float(c["h"]) if "h" in c else h_for_nodes(float(c["N"]))
        name = "config:" + str(c.get("name", os.path.splitext(os.path.basename(args.config))[0]))
        WORKLOADS[name] = (h, int(c["m"]), int(c["n"]))
        args.workload = name
        if "seed" in c and args.seed is None:
            args.seed = int(c["seed"])
        if "tol" in c:
            args.tol = float(c["tol"])
    if args.seed is not None:
        SEED = args.seed
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == BATCH_WORKLOAD:
        return run_gpu_batched(args)
    if args.workload == EXPLICIT_WORKLOAD:
        return run_gpu_explicit(args)
    if args.workload == ADJOINT_WORKLOAD:
        return run_gpu_adjoint(args)
    if args.workload == SWEEP_WORKLOAD:
        return run_gpu_sweep(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
