#!/usr/bin/env python
"""Benchmark of the matrix-free Stokes operator (RT_k x DGQ_k, Algorithm 1).

Default workload: one FP64 apply y = A x on the unit cube with 64^3 cells at
k = 3 (67,305,472 DoF), the operator throughput sweep's largest k = 3 case.
A step is one whole apply (velocity-row kernel + pressure-row kernel) over the
seeded input vector, which stays resident in HBM (x and y are 539 MB each,
larger than the 129 MB L2, so no flush is needed between steps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The same JSON line carries sub-benchmarks of the other workloads:
`apply_f32` (the FP32 apply of the V-cycle, same mesh), `sweep` (FP64 apply,
64^3 cells, k = 1..5), `smooth` (one smoothing step, 64^3,
k = 3, FP32 and FP64), `solve` (manufactured problem on 96^3 cells, k = 3,
to 1e-8: mixed precision against plain FP64, with the Schur-CG and with the
Direct local solver) and `batch` (64 uneven
problems solved together against one after another); each can be resized or
skipped with its flag (0 skips).

N > 1 runs under torchrun, one independent replica per GPU (the path has no
data exchange between problems: weak scaling); rank 0 prints one JSON line.
`--impl reference` times the CPU oracle (the assembled CSR matrix of the
paper's bilinear form) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Stokes apply GDoF/s (% HBM roofline); MG solve s/MDoF to 1e-8, mixed vs FP64"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
# FP64 ALU peak derived from unit counts and clocks: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


# dram__bytes_read.sum + dram__bytes_write.sum per launch of the velocity
# kernel, keyed by (k, n, dtype): one ncu capture of a single launch on 48^3
# cells (x larger than L2), scaled to the benchmarked mesh by its velocity
# DoFs.  Valid only for the kernel version it was taken on; other keys report
# null.
DRAM_TRAFFIC = {(3, 64, "f64"): 1158800000}


def velocity_flops_per_dof(k: int) -> float:
    """Algorithmic flops of the velocity rows per velocity DoF (Kronecker form, cell-local).

    Per new node: the two 1D interior-penalty operators (block tridiagonal,
    3 (k+1) FMA each) and 3 scalings; per cell line: KC and MC contractions
    (2 (k+2)^2 FMA) and D^T p ((k+1)(k+2) FMA) plus k+1 scalings.
    """
    nd, nc = k + 1, k + 2
    per_cell = nd * (6 * nd + 3) + 2 * nc * nc + nd * nc + nd
    return 2.0 * per_cell / nd


def velocity_flops_banded(k: int) -> float:
    """The hot path's reference algorithmic count: about 8k+14 multiply-adds
    per velocity DoF (block-tridiagonal 1D penalty operators in the two
    discontinuous directions, a banded continuous direction, B^T p)."""
    return 2.0 * (8 * k + 14)


def velocity_flops_kernel(k: int) -> float:
    """Operations per velocity DoF of the FP64 velocity kernel as written: per
    new node the two folded penalty rows (6 (k+1) multiply-adds); per cell line
    the even-odd contraction along c (sums and differences of mirrored layers
    and pressure nodes, the half-size blocks, the recombination and the carried
    node's add).  Multiply-adds count 2, adds 1."""
    nd, nc = k + 1, k + 2
    p, q = nc // 2, nd // 2
    ne, qe = p + nc % 2, q + nd % 2
    fma = nd * 6 * nd + ne * (2 * ne + q) + p * (2 * p + qe)
    add = 4 * p + 2 * q + 2 * p + 1
    return (2.0 * fma + add) / nd


def pressure_flops_per_dof(k: int) -> float:
    return 2.0 * (3 * (k + 2) + 6)


def patch_flops(k: int, cg_iters: int) -> float:
    """Algorithmic flops of one vertex-patch solve (Sec. 3.2, dense 1D transforms,
    unpadded extents): S^T F and B S Lam^{-1} S^T F at the start, cg_iters
    Schur-operator products (B S)^T then B S, and (B S)^T P and S at the end, for
    the three velocity components; a line transform from n_in to n_out nodes
    costs n_in n_out multiply-adds."""
    npc, npd = 2 * k + 1, 2 * k + 2

    def chain(src, dst):
        ext, f = list(src), 0
        for d in range(3):
            lines = 1
            for e in range(3):
                if e != d:
                    lines *= ext[e]
            f += lines * ext[d] * dst[d]
            ext[d] = dst[d]
        return f

    total = 0
    for c in range(3):
        vel = [npc if e == c else npd for e in range(3)]
        p = [npd] * 3
        total += 2 * chain(vel, vel) + (cg_iters + 1) * (chain(p, vel) + chain(vel, p))
    return 2.0 * total


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return PEAKS_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(ws, v: float) -> float:
    """The slowest rank's time (NCCL reduces on the GPU, gloo on the host)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, ws: int, steps: int, seconds: float) -> float:
    """Units all ranks processed per second of the slowest rank (weak scaling:
    every rank runs its own replica of the workload)."""
    return units_per_rank * ws * steps / seconds


class OracleSpMV:
    """The oracle's assembled CSR matrix on an n^3 sample and its product with
    a seeded vector, on `threads` host threads: row blocks of the same matrix
    multiplied concurrently (SciPy's CSR product releases the GIL), the
    oracle's own arithmetic in every block."""

    def __init__(self, n: int, k: int, threads: int = 1):
        from concurrent.futures import ThreadPoolExecutor

        import numpy as np

        from oracle.discretization import Discretization
        from seeded_inputs import random_vector

        d = Discretization(n, k)
        self.n, self.k, self.N = n, k, d.N
        self.A = d.assemble()
        self.x = random_vector(1001, d.N) * d.free_mask()
        self.threads = max(1, int(threads))
        cut = np.linspace(0, d.N, self.threads + 1).astype(np.int64)
        self.blocks = [(cut[i], cut[i + 1], self.A[cut[i]:cut[i + 1]]) for i in range(self.threads)]
        self.y = np.empty(d.N)
        self.pool = ThreadPoolExecutor(self.threads) if self.threads > 1 else None

    def _block(self, i):
        lo, hi, Ab = self.blocks[i]
        self.y[lo:hi] = Ab @ self.x

    def spmv(self):
        if self.pool is None:
            self.y[:] = self.A @ self.x
        else:
            list(self.pool.map(self._block, range(self.threads)))

    def rate(self, min_seconds: float):
        """DoF/s over repeated products for at least min_seconds."""
        self.spmv()
        reps = 0
        t0 = time.perf_counter()
        while True:
            self.spmv()
            reps += 1
            if time.perf_counter() - t0 >= min_seconds:
                break
        dt = time.perf_counter() - t0
        return self.N * reps / dt, {"n": self.n, "k": self.k, "dofs": self.N, "reps": reps, "seconds": dt,
                                    "threads": self.threads}

    def close(self):
        if self.pool is not None:
            self.pool.shutdown()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_spmv_baselines(n: int, k: int, seconds: float):
    """cpu_baseline objects of the oracle's SpMV on all host cores and on one."""
    out = {}
    for name, threads in (("all", host_cores()), ("one", 1)):
        o = OracleSpMV(n, k, threads)
        rate, info = o.rate(seconds)
        o.close()
        out[name] = {"value": rate / 1e9, "unit": "GDoF/s", "cores": info["threads"], "kind": "oracle",
                     "sample": f"CSR SpMV of the oracle's assembled matrix on {info['n']}^3 cells, k={k} "
                               f"({info['dofs']} DoF), {info['threads']} thread(s) over row blocks, "
                               f"{info['reps']} SpMVs in {info['seconds']:.1f} s"}
    return out


def oracle_solve_rate(n: int, k: int):
    """The oracle's FGMRES + V-cycle solve to 1e-8 on an n^3 sample, with the
    Schur-complement local solver (15 CG steps with dense-Cholesky velocity
    solves), the GPU solve's local solver; single-threaded."""
    from oracle.manufactured import Manufactured, rhs
    from oracle.multigrid import Hierarchy
    from seeded_inputs import manufactured_coefficients

    H = Hierarchy(n, k, local=("schur", 15))
    d = H.levels[-1].disc
    b = rhs(d, Manufactured(manufactured_coefficients(3000)))
    t0 = time.perf_counter()
    _, info = H.solve(b, tol=1e-8)
    dt = time.perf_counter() - t0
    return {"value": dt / (d.N / 1e6), "unit": "s/MDoF", "cores": 1, "kind": "oracle",
            "sample": f"oracle FGMRES(20) + V-cycle (Schur-CG 15 local solver) to 1e-8 on {n}^3 cells, k={k} ({d.N} DoF), {info['iterations']} iterations, {dt:.1f} s"}


def run_solve_pair(args, stream, ws):
    """Mixed-precision and FP64 multigrid solves of the seeded manufactured problem to 1e-8."""
    import torch

    from paper_2410_09497_gb300 import CG_FIXED, LOCAL_DIRECT, PREC_FP64, PREC_MIXED, StokesMG
    from seeded_inputs import manufactured_coefficients

    n, k = args.solve_n, args.solve_k
    out = {"workload": f"manufactured Stokes solve, RT_{k} x DGQ_{k}, {n}^3 cells, FGMRES(20) + V-cycle to 1e-8",
           "unit": "s/MDoF", "higher_is_better": False}
    coef = manufactured_coefficients(3000)
    runs = (("mixed", PREC_MIXED, CG_FIXED), ("fp64", PREC_FP64, CG_FIXED),
            ("mixed_direct", PREC_MIXED, LOCAL_DIRECT), ("fp64_direct", PREC_FP64, LOCAL_DIRECT))
    for name, prec, local in runs:
        with torch.cuda.stream(stream):
            P = StokesMG(n, k, 1.0, precision=prec, stream=stream, local_cg_mode=local)
            N = P.layout()["n_total"]
            b = torch.empty(N, dtype=torch.float64, device="cuda")
            x = torch.zeros_like(b)
            P.rhs(coef, b)
            P.solve(b, x, 1e-8)  # warm-up: workspace, coarse pseudo-inverse
            times = []
            for _ in range(max(1, args.solve_reps)):
                torch.cuda.synchronize()
                barrier(ws)
                t0 = time.perf_counter()
                info = P.solve(b, x, 1e-8)
                torch.cuda.synchronize()
                times.append(max_over_ranks(ws, time.perf_counter() - t0))
            P.close()
        t = statistics.median(times)
        out[name] = {"seconds": t, "s_per_MDoF": t / (N / 1e6), "dofs": N, "iterations": info["iterations"],
                     "nu": info["nu"], "relres": info["relres"], "converged": info["converged"],
                     "timed_solves": len(times), "seconds_min": min(times), "seconds_max": max(times)}
    out["mixed_speedup"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    out["mixed_speedup_direct"] = out["fp64_direct"]["seconds"] / out["mixed_direct"]["seconds"]
    out["local_solvers"] = ("mixed / fp64: Schur-complement CG, 15 steps (the paper's method); "
                            "*_direct: the exact local solver (precomputed Schur-complement inverses)")
    out["value"] = out["mixed"]["s_per_MDoF"]
    # iterations as levels are added (the V-cycle's contraction does not depend
    # on h): the same manufactured problem on 4^3 .. 64^3 cells, mixed precision
    levels = {}
    with torch.cuda.stream(stream):
        for nl in (4, 8, 16, 32, 64):
            P = StokesMG(nl, k, 1.0, precision=PREC_MIXED, stream=stream)
            b = torch.empty(P.layout()["n_total"], dtype=torch.float64, device="cuda")
            x = torch.zeros_like(b)
            P.rhs(coef, b)
            info = P.solve(b, x, 1e-8)
            levels[str(nl)] = {"levels": P.num_levels, "iterations": info["iterations"], "nu": info["nu"]}
            P.close()
    out["iterations_by_mesh"] = levels
    return out


def run_batch(args):
    """Batched uneven solves: seeded sides from {8, 12, 16, 24, 32} and degrees from
    {2, 3, 4}, mixed precision, FGMRES + graph-captured V-cycle to 1e-8 each, one
    stream per problem; total DoF/s of stk_solve_batch against a sequential loop."""
    import torch

    from paper_2410_09497_gb300 import PREC_MIXED, StokesMG, smooth_batch, solve_batch
    from seeded_inputs import manufactured_coefficients, splitmix64_stream

    z = splitmix64_stream(4000, 2 * args.batch)
    sides = [8, 12, 16, 24, 32]
    cfg = [(sides[int(z[2 * i]) % 5], 2 + int(z[2 * i + 1]) % 3) for i in range(args.batch)]
    probs, bs, xs = [], [], []
    for i, (n, k) in enumerate(cfg):
        s = torch.cuda.Stream()
        P = StokesMG(n, k, precision=PREC_MIXED, stream=s)
        b = torch.empty(P.layout()["n_total"], dtype=torch.float64, device="cuda")
        P.rhs(manufactured_coefficients(4000 + i), b)
        probs.append(P)
        bs.append(b)
        xs.append(torch.zeros_like(b))
    total = sum(p.layout()["n_total"] for p in probs)
    for P, b, x in zip(probs, bs, xs):  # warm-up: workspace, coarse solvers, graphs
        P.solve(b, x, 1e-8)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for P, b, x in zip(probs, bs, xs):
        P.solve(b, x, 1e-8)
    torch.cuda.synchronize()
    tseq = time.perf_counter() - t0
    t0 = time.perf_counter()
    infos = solve_batch(probs, bs, xs, 1e-8)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0

    # one FP32 smoothing step of every problem's finest level: one patch launch
    # per colour for all problems of a degree (stk_smooth_batch) against every
    # problem's own launches on its own stream
    groups = {}
    for i, (n, k) in enumerate(cfg):
        groups.setdefault(k, []).append(i)
    x32 = [torch.zeros(p.layout()["n_total"], dtype=torch.float32, device="cuda") for p in probs]
    b32 = [b.float() for b in bs]

    def separate():
        for P, x, b in zip(probs, x32, b32):
            P.smooth(x, b)

    def merged():
        for idx in groups.values():
            smooth_batch([probs[i] for i in idx], [x32[i] for i in idx], [b32[i] for i in idx])

    times = {}
    for name, f in (("separate", separate), ("merged", merged)):
        f()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            f()
        torch.cuda.synchronize()
        times[name] = (time.perf_counter() - t0) / 3
    for P in probs:
        P.close()
    return {"workload": f"{args.batch} independent manufactured Stokes solves, sides in {{8,12,16,24,32}}, k in {{2,3,4}}, mixed precision, to 1e-8",
            "problems": cfg, "total_dofs": total, "unit": "MDoF/s", "value": total / tb / 1e6,
            "sequential_value": total / tseq / 1e6, "batch_seconds": tb, "sequential_seconds": tseq,
            "speedup": tseq / tb, "all_converged": all(i["converged"] for i in infos),
            "iterations": [i["iterations"] for i in infos],
            "smoothing_step_ms": {"separate": times["separate"] * 1e3, "merged_per_degree": times["merged"] * 1e3,
                                  "note": "one FP32 smoothing step of all finest levels; merged: one patch launch "
                                          "per colour for all problems of a degree"}}


PLANAR_REFERENCE = {  # the paper's 2D reference solution: psi = G_1(x) G_1(y), p = cos(2 pi x) cos(2 pi y)
    "psi_freq": [[[1, 1, 1]] * 3] * 3, "psi_amp": [[1.0, 0.0, 0.0]] * 3,
    "p_freq": [[2, 2, 1], [1, 1, 1], [1, 1, 1]], "p_amp": [1.0, 0.0, 0.0]}

# Table 1 (Sec. 3.3), Direct solver columns Q_3 .. Q_8, rows L = 3 .. 9: the
# paper's printed fractional GMRES counts in two dimensions (context for the
# GPU counts of the same problems)
TABLE1_DIRECT = {3: [2.8, 2.4, 2.1, 2.2, 1.9, 2.1], 4: [3.2, 2.4, 2.3, 2.2, 2.1, 2.0], 5: [3.2, 2.3, 2.3, 2.0, 2.0, 1.9],
                 6: [3.0, 2.2, 2.2, 1.9, 1.9, 1.8], 7: [2.9, 1.9, 1.9, 1.8, 1.8, 1.7], 8: [2.8, 1.9, 1.8, 1.8, 1.8, 1.8],
                 9: [2.7, 1.9, 1.9, 1.8, 1.8, 1.8]}


def run_planar(args, stream):
    """The two-dimensional results on the GPU: Table 1 (fractional FGMRES
    counts to 1e-8 with the exact local solver, mixed precision, the paper's
    reference solution, L = 3 .. planar_L, Q_3 .. Q_8) and the accuracy study
    (velocity and pressure L2 errors against the time to solution, k = 2..5)."""
    import torch

    from paper_2410_09497_gb300 import PREC_MIXED, StokesMG

    table, diffs = {}, []
    with torch.cuda.stream(stream):
        for L in range(3, args.planar_L + 1):
            row = {}
            for k in range(3, 9):
                n = 2 ** L
                P = StokesMG(n, k, 1.0, dim=2, precision=PREC_MIXED, stream=stream)
                b = torch.empty(P.layout()["n_total"], dtype=torch.float64, device="cuda")
                P.rhs(PLANAR_REFERENCE, b)
                x = torch.zeros_like(b)
                P.solve(b, x, 1e-8)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                info = P.solve(b, x, 1e-8)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                P.close()
                row[f"Q{k}"] = {"nu": round(info["nu"], 3), "iterations": info["iterations"],
                                "paper": TABLE1_DIRECT[L][k - 3], "seconds": dt, "dofs": int(b.numel())}
                diffs.append(info["nu"] - TABLE1_DIRECT[L][k - 3])
            table[str(L)] = row
        study = []
        for k in (2, 3, 4, 5):
            for L in range(3, args.planar_L + 1):
                n = 2 ** L
                P = StokesMG(n, k, 1.0, dim=2, precision=PREC_MIXED, stream=stream)
                b = torch.empty(P.layout()["n_total"], dtype=torch.float64, device="cuda")
                P.rhs(PLANAR_REFERENCE, b)
                x = torch.zeros_like(b)
                P.solve(b, x, 1e-8)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                P.solve(b, x, 1e-8)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                eu, ep = P.planar_errors(PLANAR_REFERENCE, x)
                study.append({"k": k, "n": n, "dofs": int(b.numel()), "seconds": dt, "err_u": eu, "err_p": ep})
                P.close()
    return {"workload": "2D Stokes, unit square, RT_k x DGQ_k, reference solution of the paper, FGMRES(20) + "
                        "V-cycle (exact local solver, FP32 V-cycle) to 1e-8",
            "table1": table, "mean_nu_minus_paper": sum(diffs) / len(diffs),
            "max_abs_nu_minus_paper": max(abs(d) for d in diffs),
            "accuracy_vs_time": study}


def run_sweep(args, stream):
    """FP64 apply throughput over the degrees k = 1..5 on an n^3 mesh (the
    operator sweep); L2 is flushed between timed applies when x and y fit in it."""
    import torch

    from paper_2410_09497_gb300 import StokesMG, layout_sizes
    from seeded_inputs import random_vector

    n = args.sweep_n
    out = {"workload": f"FP64 Stokes apply, {n}^3 cells, k = 1..5", "unit": "GDoF/s", "per_k": {}}
    flush = torch.empty(64 * 2**20, dtype=torch.float32, device="cuda")  # 256 MB > L2
    with torch.cuda.stream(stream):
        for k in range(1, 6):
            P = StokesMG(n, k, 1.0, stream=stream)
            nv, npress, N = layout_sizes(n, k)
            x = torch.from_numpy(random_vector(2000 + k, N)).cuda()
            y = torch.empty_like(x)
            needs_flush = 2 * N * 8 < 2 * 129 * 10**6
            for _ in range(3):
                P.apply(x, y)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
            for a, b in ev:
                if needs_flush:
                    flush.zero_()
                a.record(stream)
                P.apply(x, y)
                b.record(stream)
            torch.cuda.synchronize()
            t = sum(a.elapsed_time(b) for a, b in ev) / len(ev) / 1e3
            flops = velocity_flops_per_dof(k) * 3 * nv + pressure_flops_per_dof(k) * npress
            out["per_k"][str(k)] = {"dofs": N, "gdofs": N / t / 1e9, "ms": t * 1e3,
                                    "frac_fp64_peak": flops / t / 1e12 / FP64_PEAK_TFLOPS,
                                    "l2": "flushed between applies" if needs_flush else "inputs larger than L2"}
            P.close()
            del x, y
    return out


def run_apply_f32(args, stream):
    """The FP32 apply of the V-cycle on the benchmarked mesh (64^3, k = 3): GDoF/s
    and the fraction of the HBM roofline (read x, write y: 8 bytes per DoF)."""
    import torch

    from paper_2410_09497_gb300 import StokesMG, layout_sizes
    from seeded_inputs import random_vector

    n, k = args.n, args.k
    nv, npress, N = layout_sizes(n, k)
    with torch.cuda.stream(stream):
        P = StokesMG(n, k, 1.0, stream=stream)
        x = torch.from_numpy(random_vector(1001, N)).float().cuda()
        y = torch.empty_like(x)
        for _ in range(3):
            P.apply(x, y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(20):
            P.apply(x, y)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 20 / 1e3
        P.close()
    peaks, src = load_peaks()
    hbm = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    flops = velocity_flops_per_dof(k) * 3 * nv + pressure_flops_per_dof(k) * npress
    return {"workload": f"FP32 Stokes apply, RT_{k} x DGQ_{k}, {n}^3 cells", "gdofs": N / t / 1e9, "ms": t * 1e3,
            "hbm_gbs": 8 * N / t / 1e9, "frac_hbm": 8 * N / t / 1e9 / hbm, "peak_source": src,
            "frac_fp32_peak": flops / t / 1e12 / FP32_PEAK_TFLOPS,
            "l2": "inputs larger than L2 (x and y %d MB each)" % (4 * N // 10**6)}


def run_smooth_pair(args, stream):
    """One smoothing step (Algorithm 2: 8 colour residuals and patch solves) in
    FP32 and FP64, ns/DoF (the unit of the paper's smoothing-step row)."""
    import torch

    from paper_2410_09497_gb300 import StokesMG, layout_sizes
    from seeded_inputs import random_vector

    n, k = args.smooth_n, args.solve_k
    out = {"workload": f"one smoothing step, RT_{k} x DGQ_{k}, {n}^3 cells, Schur-CG 15 steps", "unit": "ns/DoF"}
    with torch.cuda.stream(stream):
        P = StokesMG(n, k, 1.0, stream=stream)
        N = P.layout()["n_total"]
        for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
            b = torch.from_numpy(random_vector(5, N)).to(dt).cuda()
            x = torch.zeros_like(b)
            for _ in range(2):
                P.smooth(x, b)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                P.smooth(x, b)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 3
            nv, npress, _ = layout_sizes(n, k)
            flops = (n - 1) ** 3 * patch_flops(k, 15) + 8 * (velocity_flops_per_dof(k) * 3 * nv
                                                              + pressure_flops_per_dof(k) * npress)
            peak = FP32_PEAK_TFLOPS if name == "f32" else FP64_PEAK_TFLOPS
            out[name] = {"ms_per_step": ms, "ns_per_dof": ms * 1e6 / N, "dofs": N,
                         "tflops_algorithmic": flops / ms / 1e9, "frac_peak": flops / ms / 1e9 / peak}
        P.close()
    out["flops_note"] = ("algorithmic flops: dense 1D transforms of every patch solve (15 CG steps) "
                         "plus the 8 colour residuals; frac_peak against the derived FP32 / FP64 ALU peak")
    return out


def run_smooth_mode(args):
    """Time one smoothing step of Algorithm 2 (8 colour residuals + patch solves)
    on an n^3 mesh in FP32 and FP64; prints one JSON line (ns/DoF per step, the
    unit of the paper's Table 2 smoothing row)."""
    import torch

    from paper_2410_09497_gb300 import StokesMG
    from seeded_inputs import random_vector

    n, k = args.n, args.k
    out = {"mode": "smooth", "workload": f"one smoothing step, RT_{k} x DGQ_{k}, {n}^3 cells, Schur-CG 15 steps",
           "unit": "ns/DoF per smoothing step"}
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        P = StokesMG(n, k, 1.0, stream=stream)
        N = P.layout()["n_total"]
        for name, dt in (("f32", torch.float32), ("f64", torch.float64)):
            b = torch.from_numpy(random_vector(5, N)).to(dt).cuda()
            x = torch.zeros_like(b)
            for _ in range(args.warmup):
                P.smooth(x, b)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            stream.synchronize()
            e0.record(stream)
            for _ in range(args.steps):
                P.smooth(x, b)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            out[name] = {"ms_per_step": ms, "ns_per_dof": ms * 1e6 / N, "dofs": N}
        P.close()
    print(json.dumps(out), flush=True)
    return 0


def run_solve_mode(args):
    """One mixed-precision solve of the manufactured problem after a warm-up
    solve (profiling); prints one JSON line."""
    import torch

    from paper_2410_09497_gb300 import PREC_MIXED, StokesMG
    from seeded_inputs import manufactured_coefficients

    n, k = args.solve_n, args.solve_k
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        P = StokesMG(n, k, 1.0, precision=PREC_MIXED, stream=stream)
        b = torch.empty(P.layout()["n_total"], dtype=torch.float64, device="cuda")
        P.rhs(manufactured_coefficients(3000), b)
        x = torch.zeros_like(b)
        P.solve(b, x, 1e-8)
        t0 = time.perf_counter()
        info = P.solve(b, x, 1e-8)
        dt = time.perf_counter() - t0
        P.close()
    print(json.dumps({"mode": "solve", "workload": f"mixed-precision solve, RT_{k} x DGQ_{k}, {n}^3 cells, to 1e-8",
                      "seconds": dt, "iterations": info["iterations"], "relres": info["relres"]}), flush=True)
    return 0


def run_reference(args):
    """The reference arm: the CPU oracle's assembled-matrix SpMV (the operator
    apply as a plain CSR product) on all host cores, each step `ref_reps`
    products on an 8^3-cell sample of the benchmarked workload (the 64^3
    matrix would not fit a host: about 75 GB of CSR)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    sample_n, k = 8, args.k
    o = OracleSpMV(sample_n, k, host_cores())
    reps = args.ref_reps
    for _ in range(args.warmup):
        for _ in range(reps):
            o.spmv()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(reps):
            o.spmv()
    dt = time.perf_counter() - t0
    o.close()
    rate = o.N * reps * args.steps / dt / 1e9
    sample = (f"CSR SpMV of the oracle's assembled matrix, {sample_n}^3 cells k={k} ({o.N} DoF), "
              f"{reps} SpMVs per step, {o.threads} threads over row blocks")
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "GDoF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"FP64 Stokes apply, RT_{k} x DGQ_{k}, CPU oracle on a {sample_n}^3-cell sample "
                               f"of the {args.n}^3-cell workload", "n": sample_n, "k": k, "dofs": o.N,
                   "sample_of_n": args.n},
        "cpu_baseline": {"value": rate, "unit": "GDoF/s", "cores": o.threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_init()
    torch.cuda.set_device(local)
    from paper_2410_09497_gb300 import StokesMG, build, layout_sizes
    from seeded_inputs import random_vector

    if not os.path.exists(os.path.join(ROOT, "paper_2410_09497_gb300", "libstokesmg.so")):
        build.build()
    n, k = args.n, args.k
    dt = torch.float64 if args.dtype == "f64" else torch.float32
    esize = 8 if dt == torch.float64 else 4
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        P = StokesMG(n, k, 1.0, stream=stream)
        nv, npress, N = layout_sizes(n, k)
        x_host = torch.from_numpy(random_vector(1001 + rank, N)).to(dt)
        x = x_host.cuda()
        y = torch.empty_like(x)
        for _ in range(args.warmup):
            P.apply(x, y)
        stream.synchronize()
        K = args.steps
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(ws)
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            time.sleep(0.3)
            start.record(stream)
            for i in range(K):
                ev[i][0].record(stream)
                P.apply_stage(0, x, y)
                ev[i][1].record(stream)
                P.apply_stage(1, x, y)
            end.record(stream)
            torch.cuda.synchronize()
        barrier(ws)
        t_local = start.elapsed_time(end) / 1e3
        t_vel = sum(a.elapsed_time(b) for a, b in ev) / K / 1e3
        t = max_over_ranks(ws, t_local)

        # end to end through the public API: pinned host input, copy in, apply, copy out
        xh = x_host.pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        for _ in range(2):
            x.copy_(xh, non_blocking=True)
            P.apply(x, y)
            yh.copy_(y, non_blocking=True)
        stream.synchronize()
        barrier(ws)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            x.copy_(xh, non_blocking=True)
            P.apply(x, y)
            yh.copy_(y, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(ws, e0.elapsed_time(e1) / 1e3)
        barrier(ws)
        P.close()

    value = whole_job_rate(N, ws, K, t) / 1e9
    e2e = whole_job_rate(N, ws, K, t_e2e) / 1e9
    peaks, peak_src = load_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    vflops = velocity_flops_banded(k) * 3 * nv
    alu_peak = FP64_PEAK_TFLOPS if dt == torch.float64 else FP32_PEAK_TFLOPS
    achieved_tf = vflops / t_vel / 1e12
    traffic = DRAM_TRAFFIC.get((k, n, args.dtype))
    apply_bytes = 2 * N * esize
    line = {
        "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": ws, "steps": K, "warmup": args.warmup,
        "ms_per_step": t / K * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.dtype, "data": "synthetic",
        "config": {"workload": f"{'FP64' if esize == 8 else 'FP32'} Stokes apply, RT_{k} x DGQ_{k}, {n}^3 cells", "n": n, "k": k,
                   "dofs": N, "nu": 1.0, "l2": "inputs larger than L2 (x and y %d MB each)" % (N * esize // 10**6),
                   "parallelism": f"replicas x{ws}"},
        "roofline": {"bound": "alu", "kernel": "apply_velocity_kernel", "achieved": achieved_tf,
                     "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved_tf / alu_peak, "traffic": traffic,
                     "peak_source": "derived: 152 SMs x %s FMA/clk x 2 x 2.07 GHz" % ("2 FP64" if esize == 8 else "128 FP32"),
                     "ms_per_launch": t_vel * 1e3, "flop_per_launch": vflops,
                     "flop_per_velocity_dof": velocity_flops_banded(k), "count": "8k+14 multiply-adds per velocity DoF",
                     "frac_at_dense_count": velocity_flops_per_dof(k) * 3 * nv / t_vel / 1e12 / alu_peak,
                     "frac_at_kernel_count": velocity_flops_kernel(k) * 3 * nv / t_vel / 1e12 / alu_peak},
        "hbm_roofline": {"achieved_gbs": apply_bytes * K / t / 1e9, "peak": hbm_peak, "unit": "GB/s",
                         "frac": apply_bytes * K / t / 1e9 / hbm_peak, "peak_source": peak_src,
                         "bytes_per_step": apply_bytes},
        "e2e": {"value": e2e, "unit": "GDoF/s", "h2d_bytes_per_step": N * esize, "d2h_bytes_per_step": N * esize},
        "gpu_launches": 2 * K,
        "clocks": clk.summary(),
    }
    line["apply_f32"] = run_apply_f32(args, stream)
    if args.sweep_n > 0:
        line["sweep"] = run_sweep(args, stream)
    if args.smooth_n > 0:
        line["smooth"] = run_smooth_pair(args, stream)
    if args.solve_n > 0:
        line["solve"] = run_solve_pair(args, stream, ws)
    if args.batch > 0:
        line["batch"] = run_batch(args)
    if args.planar_L >= 3:
        line["planar"] = run_planar(args, stream)
    if rank == 0 and not args.no_cpu_baseline:
        base = oracle_spmv_baselines(8, k, args.cpu_seconds / 2)
        line["cpu_baseline"] = base["all"]
        line["cpu_baseline_1core"] = base["one"]
        if args.solve_n > 0:
            line["solve"]["cpu_baseline"] = oracle_solve_rate(4, args.solve_k)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--k", type=int, default=3)
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-reps", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--solve-n", type=int, default=96, help="mesh of the mixed-vs-FP64 solve sub-benchmark (0: skip)")
    ap.add_argument("--solve-k", type=int, default=3)
    ap.add_argument("--solve-reps", type=int, default=3, help="timed solves per arm of the solve sub-benchmark (median reported)")
    ap.add_argument("--sweep-n", type=int, default=64, help="mesh of the FP64 apply sweep over k = 1..5 (0: skip)")
    ap.add_argument("--smooth-n", type=int, default=64, help="mesh of the smoothing-step sub-benchmark (0: skip)")
    ap.add_argument("--batch", type=int, default=64, help="batched uneven solves (0: skip)")
    ap.add_argument("--planar-L", type=int, default=8, help="finest level of the 2D Table 1 and accuracy study (0: skip)")
    ap.add_argument("--mode", default="apply", choices=["apply", "smooth", "solve"],
                    help="apply: the benchmark line; smooth / solve: time smoothing steps or one "
                         "mixed-precision solve only (profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "smooth":
        return run_smooth_mode(args)
    if args.mode == "solve":
        return run_solve_mode(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
