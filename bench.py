"""Benchmark of the SGF hot path on GB300.

One step = one whole factor + PCG solve to a 1e-10 relative residual
(sgf_factor of a coefficient field, then sgf_pcg_solve of one right-hand
side) on the 3D high-contrast diffusion workload: 7-point two-point-flux
finite volumes on a 128^3 grid (n = 2,097,152), two-phase coefficients 1 and
1e4 with 30% of the 4^3-cell blocks (seeded) at 1e4, Dirichlet on the x-
face, Nest-All-All, piecewise-quadratic preservation, leaf 8.  The headline
is the mixed-precision path (FP32 factor and apply, 3xTF32 tensor-core
products, FP64 PCG, SpMV and dot products); the plain FP64 GPU path is timed
beside it on the same inputs, and the mixed solution's distance to the FP64
one is stated.

Beside the headline the line carries (unless --quick):
  * table51: E_1 = ||(A - A_l) v_1|| / lambda_1 and E_n (largest and smallest
    eigenvectors, closed-form sines) of the FP64 factor on constant-
    coefficient 3D Poisson at 32^3, 64^3 and 128^3 (Table 5.1 quantities);
  * sweep: mixed factor + PCG on 3D Poisson at 64^3, 128^3 and 192^3
    (iterations and time per unknown as n grows, the paper's scaling study);
  * serve: the continuous-batching serving workload (p50 / p99, solves/s);
  * cpu_baseline: the CPU oracle on the same recipe at 32^3, timed once with
    all host cores and once with one thread (no scaling to 128^3).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--quick]
Under torchrun (N > 1) every rank solves its own seeded instance (weak
scaling, no data-path collective); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import sgf_inputs as si  # noqa: E402

METRIC = "factor+PCG time to 1e-10 residual, mixed vs FP64 GPU; serve p50/p99 latency"
WORKLOAD = "twophase3d_128"
WORKLOAD_DESC = ("3D high-contrast diffusion, 7-pt TPFA on 128^3 (n=2097152), two-phase kappa 1 / 1e4 "
                 "(30% of the 4^3-cell blocks at 1e4, seeded), Dirichlet x-, Nest-All-All, pcw-quadratic, leaf 8")
CPU_SAMPLE = "twophase3d_32"   # CPU oracle baseline: the same recipe on a 32^3 box
REF_SAMPLE = "twophase3d_24"   # reference arm: the same recipe on a 24^3 box per step
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
NOMINAL_SM = 152
NOMINAL_MAX_MHZ = 2070.0


# ---------------------------------------------------------------------------
# distributed helpers (torchrun, one rank per GPU)
# ---------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(backend: str):
    import torch.distributed as dist
    ws, rank, _ = dist_env()
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend, rank=rank, world_size=ws)
    return dist if ws > 1 else None


def reduce_max(value: float, dist=None, device=None) -> float:
    """Max of a float over all ranks (identity on one rank)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist=None):
    if dist is not None:
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample of the same workload)
# ---------------------------------------------------------------------------
def oracle_sample(name: str, seed: int = 0) -> dict:
    """CPU oracle factor + PCG (FP64, to 1e-10) on one named instance; wall
    seconds of the factor and of the solve, iterations and residual."""
    from oracle.assemble import assemble
    from oracle.partition import build_hierarchy
    from oracle.pcg import pcg
    from oracle.sgf import Options, factorize
    cfg = si.config(name, seed)
    A = assemble(cfg)
    H = build_hierarchy(cfg["n"], 3, cfg["leaf"], cfg["stencil"])
    b = si.rhs(A.shape[0], seed)
    t0 = time.perf_counter()
    F = factorize(A, H, Options(degree=cfg["degree"], order="level"))
    t1 = time.perf_counter()
    _, it, res = pcg(lambda v: A @ v, F.solve, b)
    t2 = time.perf_counter()
    return dict(name=name, n=int(A.shape[0]), factor_s=t1 - t0, pcg_s=t2 - t1, seconds=t2 - t0,
                iterations=int(it), rel_residual=float(res))


def oracle_sample_subprocess(name: str, threads: int | None, seed: int = 0) -> dict:
    """oracle_sample in a fresh interpreter; threads = BLAS / OpenMP thread
    count (None: all host cores).  Spawned, never forked from a process that
    holds a CUDA context."""
    env = dict(os.environ)
    if threads is not None:
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[var] = str(threads)
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_sample(%r, %d)))" % (ROOT, name, seed))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def cpu_baseline(name: str = CPU_SAMPLE) -> dict:
    """The oracle as it stands on the host cores: once with every core, once
    with one thread (the paper's sequential setting), on one instance of the
    workload's recipe; reported at that size, without scaling."""
    allc = oracle_sample_subprocess(name, None)
    one = oracle_sample_subprocess(name, 1)
    return {"value": round(1e3 * allc["seconds"], 1), "unit": "ms", "cores": cpu_cores(), "kind": "oracle",
            "sample": (f"oracle factor+PCG to 1e-10 on the {name.split('_')[1]}^3 instance of the same recipe "
                       f"(n={allc['n']}, {allc['iterations']} it), timed once at that size, not scaled"),
            "factor_ms": round(1e3 * allc["factor_s"], 1), "pcg_ms": round(1e3 * allc["pcg_s"], 1),
            "one_thread": {"value": round(1e3 * one["seconds"], 1), "unit": "ms", "cores": 1,
                           "iterations": one["iterations"]}}


def cpu_cores() -> int:
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        v = os.environ.get(var)
        if v and v.isdigit():
            return int(v)
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# roofline of the dominant kernel
# ---------------------------------------------------------------------------
def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def kernel_bound(name: str, precision: str, peaks: dict):
    """(bound, unit, peak, note) for one kernel of the path."""
    if name == "apply":
        return "hbm", "GB/s", peaks["hbm_gbs"], \
            "one A_l^{-1} graph replay (k_gemv_t, k_vgather, k_veccopy nodes) vs measured HBM copy bandwidth"
    if name in ("k_gemv_n", "k_gemv_t", "k_spmv", "k_dot", "k_vector", "k_veccopy", "k_copy", "k_assemble"):
        return "hbm", "GB/s", peaks["hbm_gbs"], "of measured HBM copy bandwidth"
    # The FP32 factor's tile GEMMs run on the tensor cores as 3xTF32 (three
    # TF32 products per FP32 product): the bound is the measured sustained
    # bf16 dense rate x the nominal TF32/bf16 ratio (1.125 / 2.25 PFLOP/s) / 3,
    # against the algorithmic 2 M N K flop.
    if precision == "mixed" and name == "k_gemm" and os.environ.get("SGF_TENSOR_CORES", "1") != "0":
        return "tensor", "TFLOP/s", peaks["bf16_tflops_sustained"] * 0.5 / 3.0, \
            "3xTF32 effective: measured sustained bf16 x nominal TF32/bf16 ratio 0.5 / 3 products"
    # SIMT contractions: FP32 CUDA cores 152 SM x 128 lanes x 2 flop x 2070 MHz;
    # FP64: the cuBLAS DGEMM rate measured in this run when there is one, else
    # the nominal 1.25 TFLOP/s of GB300
    if precision == "mixed":
        return "alu", "TFLOP/s", NOMINAL_SM * 128 * 2 * NOMINAL_MAX_MHZ * 1e6 / 1e12, \
            "FP32 SIMT peak from unit counts and max clock"
    if peaks.get("fp64_tflops"):
        return "alu", "TFLOP/s", peaks["fp64_tflops"], "FP64 DGEMM rate measured in this run (torch.matmul 4096^3)"
    return "alu", "TFLOP/s", 1.25, "nominal GB300 FP64 rate"


def traffic_from_profiles(kernel: str, precision: str = "mixed"):
    """dram bytes per launch recorded from an ncu capture of this kernel on
    this precision's path, if any (the summaries without a suffix are of the
    mixed-precision path)."""
    suffix = "" if precision == "mixed" else f"_{precision}"
    path = os.path.join(ROOT, "profiles", f"{kernel}_{WORKLOAD}{suffix}.txt")
    try:
        with open(path) as f:
            for line in f:
                if line.startswith("traffic_bytes_per_launch:"):
                    v = line.split(":", 1)[1].strip()
                    return None if v == "null" else float(v)
    except OSError:
        pass
    return None


def roofline(prof: dict, precision: str, peaks: dict):
    name, rec = max(prof.items(), key=lambda kv: kv[1]["ms"])
    bound, unit, peak, note = kernel_bound(name, precision, peaks)
    if rec["ms"] <= 0 or rec["launches"] == 0:
        return None
    per_launch_ms = rec["ms"] / rec["launches"]
    if bound == "hbm":
        achieved = rec["bytes"] / (rec["ms"] * 1e-3) / 1e9
    else:
        achieved = rec["flops"] / (rec["ms"] * 1e-3) / 1e12
    return {"kernel": name, "bound": bound, "achieved": round(achieved, 4), "peak": round(peak, 2),
            "unit": unit, "frac": round(achieved / peak, 4), "traffic": traffic_from_profiles(name, precision),
            "launches": rec["launches"], "avg_launch_ms": round(per_launch_ms, 5),
            "share_of_step": None, "peak_note": note}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def measure_fp64_peak(dev) -> float:
    """FP64 DGEMM rate of this GPU (cuBLAS through torch.matmul, 4096^3, best of 5)."""
    import torch
    a = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    b = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    best = float("inf")
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2.0 * 4096 ** 3 / (best * 1e-3) / 1e12


def run_ours(args):
    import torch
    import paper_1907_03406_gb300 as sgf

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init("nccl")
    cfg = si.config(WORKLOAD, seed=rank)
    coeffs_h = np.ascontiguousarray(cfg["coeffs"].ravel())
    b_h = si.rhs(int(np.prod(cfg["n"])), seed=rank)
    coeffs = torch.tensor(coeffs_h, dtype=torch.float64, device=dev)
    b = torch.tensor(b_h, dtype=torch.float64, device=dev)
    plans = {p: sgf.Plan.from_config(cfg, precision=p) for p in ("mixed", "fp64")}
    # launch shapes from the autotuner (untimed setup: factor shapes timed on
    # factorizations, GEMV budgets on applies), reported in config.tuning
    tuned = {p: plans[p].autotune(coeffs, napply=20 if p == "mixed" else 5)[0] for p in plans}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream()

    def one_step(plan, keep=None):
        F = sgf.Factor(plan, coeffs)
        x, info = F.pcg(b, rtol=1e-10, maxit=1000)
        F.close()
        if keep is not None:
            keep.append(x)
        return info

    def timed(plan, steps, profile=False):
        infos, total, xs = [], 0.0, []
        if profile:   # events around the contractions and the apply graph replays only
            sgf.profile_reset(timing="contractions")
        for k in range(steps):
            flush.zero_()
            barrier(dist)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos.append(one_step(plan, xs if k == 0 else None))
            e1.record(stream)
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1)
        prof = sgf.profile_read() if profile else None
        return total, infos, prof, xs[0]

    for _ in range(args.warmup):
        one_step(plans["mixed"])
    one_step(plans["fp64"])
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    ms_mixed, infos_m, prof_m, x_m = timed(plans["mixed"], args.steps, profile=True)
    clk = clocks.stop()
    fp64_steps = max(1, min(args.steps, 5))
    ms_fp64, infos_d, prof_d, x_d = timed(plans["fp64"], fp64_steps, profile=True)
    # the mixed result against the FP64 GPU solution of the same system
    err_vs_fp64 = (torch.linalg.norm(x_m - x_d) / torch.linalg.norm(x_d)).item()
    del x_m, x_d

    # end to end through the host-buffer C ABI call, pinned host memory
    pc = torch.tensor(coeffs_h, dtype=torch.float64).pin_memory()
    pb = torch.tensor(b_h, dtype=torch.float64).pin_memory()
    px = torch.empty_like(pb).pin_memory()
    e2e_ms = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sgf.solve_host_ptr(plans["mixed"], pc.data_ptr(), pb.data_ptr(), px.data_ptr(), 1, maxit=1000)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))

    per_step = ms_mixed / args.steps
    per_step_fp64 = ms_fp64 / fp64_steps
    per_step = reduce_max(per_step, dist, dev)
    per_step_fp64 = reduce_max(per_step_fp64, dist, dev)
    e2e = reduce_max(statistics.median(e2e_ms), dist, dev)
    # kernels launched (an apply graph replay is counted through its nodes)
    launches = sum(v["launches"] for k, v in prof_m.items() if k != "apply")

    if rank != 0:
        barrier(dist)
        return
    peaks, peak_kind = load_peaks()
    peaks = dict(peaks, fp64_tflops=measure_fp64_peak(dev))
    roof = roofline(prof_m, "mixed", peaks)
    if roof is not None:
        # device time of the kernel / wall time of the timed steps
        roof["share_of_step"] = round(prof_m[roof["kernel"]]["ms"] / ms_mixed, 4) if ms_mixed else None
        roof["peak_source"] = peak_kind
    roof_d = roofline(prof_d, "fp64", peaks)
    n = int(np.prod(cfg["n"]))
    line = {
        "metric": METRIC,
        "value": round(per_step, 3),
        "unit": "ms",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(per_step, 3),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC, "name": WORKLOAD,
                   "precision": "mixed (FP32 factor/apply, 3xTF32 tensor-core GEMMs, FP64 PCG/SpMV/dots)",
                   "n": n, "rtol": 1e-10, "per_rank_instances": 1, "parallelism": f"replicas x{ws}",
                   "l2": "256 MB buffer written between timed steps; factor data (13 GB) > L2",
                   "tuning": tuned},
        "iterations": [i["iterations"] for i in infos_m],
        "rel_residual": max(i["rel_residual"] for i in infos_m),
        "error_vs_fp64_solution": err_vs_fp64,
        "fp64": {"ms_per_step": round(per_step_fp64, 3), "steps": fp64_steps,
                 "iterations": [i["iterations"] for i in infos_d],
                 "rel_residual": max(i["rel_residual"] for i in infos_d),
                 "speedup_mixed_over_fp64": round(per_step_fp64 / per_step, 3),
                 "roofline": roof_d},
        "solves_per_s": round(ws * 1e3 / per_step, 3),
        "roofline": roof,
        "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3)} for k, v in prof_m.items() if v["launches"]},
        "gpu_launches": launches,
        "e2e": {"value": round(e2e, 3), "unit": "ms", "h2d_bytes_per_step": 8 * (coeffs_h.size + b_h.size),
                "d2h_bytes_per_step": 8 * b_h.size},
        "clocks": clk,
    }
    del plans, coeffs, b, flush
    sgf.release_cached_memory()
    if not args.quick:
        line["table51"] = run_table51(dev)
        line["sweep"] = run_sweep(dev)
        line["serve"] = run_serve(args)
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    barrier(dist)


def poisson_eigvec(e: int, mode: int):
    """Closed-form eigenpair of the 7-point Dirichlet Laplacian on e^3 points
    (unit coefficients, ghost nodes one step outside): v(x, y, z) =
    prod sin(k pi (x_a + 1) / (e + 1)) with k = mode on every axis,
    lambda = sum over the axes of 2 - 2 cos(k pi / (e + 1))."""
    s = np.sin(mode * np.pi * (np.arange(e) + 1.0) / (e + 1.0))
    v = (s[None, None, :] * s[None, :, None] * s[:, None, None]).ravel()   # [z, y, x]
    lam = 3.0 * (2.0 - 2.0 * np.cos(mode * np.pi / (e + 1.0)))
    return v / np.linalg.norm(v), lam


def run_table51(dev, sizes=(32, 64, 128)):
    """Table 5.1 quantities of the FP64 factor (Nest-All-All, quadratics) on
    constant-coefficient 3D Poisson: E_1 = ||(A - A_l) v_1|| / lambda_1 for
    the largest eigenvector and E_n for the smallest."""
    import torch
    import paper_1907_03406_gb300 as sgf
    rows = []
    for e in sizes:
        cfg = si.config(f"poisson3d_{e}")
        plan = sgf.Plan.from_config(cfg, precision="fp64")
        F = sgf.Factor(plan, torch.tensor(cfg["coeffs"].ravel(), dtype=torch.float64, device=dev))
        out = {"edge": e, "n": plan.n}
        for key, mode in (("E_1", e), ("E_n", 1)):
            v, lam = poisson_eigvec(e, mode)
            vt = torch.tensor(v, dtype=torch.float64, device=dev)
            d = F.spmv(vt) - F.apply_forward(vt)
            out[key] = float(torch.linalg.norm(d).item() / lam)
        F.close()
        rows.append(out)
    sgf.release_cached_memory()
    return {"rows": rows, "what": "FP64 factor, Nest-All-All pcw-quadratic, leaf 8, 7-pt Dirichlet Poisson; "
                                  "E_1: largest eigenvector, E_n: smallest (closed-form sines)"}


def run_sweep(dev, sizes=(64, 128, 192), precision="mixed"):
    """Size sweep on 3D Poisson (7-point, unit coefficients, Dirichlet on every
    face, Nest-All-All quadratics): factor (a repeated factorization, its
    memory already in the pool) + PCG to 1e-10, iterations, time per unknown."""
    import torch
    import paper_1907_03406_gb300 as sgf
    rows = []
    for e in sizes:
        cfg = si.config(f"poisson3d_{e}")
        plan = sgf.Plan.from_config(cfg, precision=precision)
        coeffs = torch.tensor(cfg["coeffs"].ravel(), dtype=torch.float64, device=dev)
        b = torch.tensor(si.rhs(plan.n, 0), dtype=torch.float64, device=dev)
        sgf.Factor(plan, coeffs).close()     # the pool reserves this size's memory
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        F = sgf.Factor(plan, coeffs)
        e1.record()
        _, info = F.pcg(b, rtol=1e-10, maxit=1000)
        e2.record()
        torch.cuda.synchronize()
        fms, pms = e0.elapsed_time(e1), e1.elapsed_time(e2)
        rows.append({"edge": e, "n": plan.n, "factor_ms": round(fms, 2), "pcg_ms": round(pms, 2),
                     "iterations": info["iterations"], "rel_residual": info["rel_residual"],
                     "ns_per_unknown": round(1e6 * (fms + pms) / plan.n, 1)})
        F.close()
        del coeffs, b
        sgf.release_cached_memory()
    return {"rows": rows, "precision": precision,
            "what": "3D Poisson 7-pt, unit coefficients, Dirichlet faces, Nest-All-All pcw-quadratic, leaf 8"}


def run_serve(args, slots: int = 4, count: int = 256, load: float = 0.7):
    """Serving workload: seeded Poisson stream of 3D 7-point diffusion requests
    (edge U{32..96}, log-normal coefficients std 1, 40% factor+solve, 60%
    solve on a resident factor, 1-8 right-hand sides) replayed in real time at
    `load` x the measured single-slot capacity; p50/p99 latency, solves/s."""
    from paper_1907_03406_gb300.serve import Server
    calib = si.request_stream(seed=101, count=10, rate_hz=1e6)
    srv = Server(slots=1)
    srv.run(calib[:2])           # warm-up: plans, graphs, allocator
    srv.records.clear()
    t0 = time.perf_counter()
    srv.run(calib[2:])
    mean_service = (time.perf_counter() - t0) / len(calib[2:])
    srv.close()
    rate = load / mean_service
    reqs = si.request_stream(seed=1, count=count, rate_hz=rate)
    srv = Server(slots=slots)
    summ = srv.run(reqs)
    srv.close()
    summ.update(load=load, rate_hz=round(rate, 3), slots=slots,
                single_slot_service_ms=round(1e3 * mean_service, 2),
                workload="256 requests, Poisson arrivals, edge U{32..96}, 40% factor+solve / 60% solve, "
                         "1-8 RHS, mixed precision, rtol 1e-10")
    for k in ("p50_ms", "p99_ms", "mean_ms", "solves_per_s", "makespan_s"):
        if summ.get(k) is not None:
            summ[k] = round(summ[k], 3)
    return summ


def run_ncu(args):
    """--ncu step: one factor + PCG step inside an NVTX range "sgf_step" after
    warm-up steps outside it (ncu --nvtx --nvtx-include sgf_step/);
    --ncu apply: one apply of A_l^{-1} inside "sgf_apply"."""
    import torch
    import paper_1907_03406_gb300 as sgf
    dev = torch.device("cuda", 0)
    cfg = si.config(args.workload, seed=0)
    coeffs = torch.tensor(np.ascontiguousarray(cfg["coeffs"].ravel()), dtype=torch.float64, device=dev)
    b = torch.tensor(si.rhs(int(np.prod(cfg["n"])), 0), dtype=torch.float64, device=dev)
    plan = sgf.Plan.from_config(cfg, precision=args.precision)

    def step():
        F = sgf.Factor(plan, coeffs)
        _, info = F.pcg(b, rtol=1e-10, maxit=500)
        F.close()
        return info
    if args.ncu == "apply":
        # one application of A_l^{-1} (one graph replay) inside the range,
        # after a factorization and warm-up applies outside it
        F = sgf.Factor(plan, coeffs)
        y = F.apply(b)
        for _ in range(max(1, args.warmup)):
            F.apply(b, out=y)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("sgf_apply")
        F.apply(b, out=y)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        F.close()
        print(json.dumps({"ncu_apply": args.workload, "precision": args.precision}), flush=True)
        return
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("sgf_step")
    info = step()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"ncu_step": args.workload, "precision": args.precision, **info}), flush=True)


def run_reference(args):
    """The reference arm: the CPU oracle (FP64, on the host cores) as it
    stands, each step one factor + PCG solve on the 24^3 instance of the
    workload's recipe (a bounded sample: the 128^3 oracle factor alone is
    minutes of CPU work); the value is the mean time per step at that size."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    vals, det = [], None
    for k in range(args.warmup + args.steps):
        det = oracle_sample(REF_SAMPLE, seed=k % 2)
        if k >= args.warmup:
            vals.append(1e3 * det["seconds"])
    v = statistics.mean(vals)
    sample = (f"each step: oracle factor+PCG to 1e-10 on the 24^3 instance of the same recipe "
              f"(n={det['n']}, {det['iterations']} it), not scaled")
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "ms", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v, 1), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "name": WORKLOAD, "sample": REF_SAMPLE,
                       "precision": "fp64 CPU oracle"},
            "cpu_baseline": {"value": round(v, 1), "unit": "ms", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(v, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="headline only: no Table 5.1 quantities, size sweep or serving measurement")
    ap.add_argument("--ncu", choices=["step", "apply"], default=None,
                    help="one step (or one apply) in an NVTX range, for ncu")
    ap.add_argument("--workload", default=WORKLOAD, help="ncu mode: grf3d_<edge> / twophase3d_<edge>")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    args = ap.parse_args(argv)
    if args.ncu:
        return run_ncu(args)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
