#!/usr/bin/env python
"""Benchmark: time to the nev smallest eigenpairs at relative residual 1e-8, mixed
precision vs FP64 on the GPU, and SpMM GB/s.

Headline workload (one step = one complete gcge_solve, Algorithm 1 to convergence):
the 3D Q1 FEM pencil on 64^3 interior nodes (n = 262,144, 27-point pattern,
nnz = 6,859,000), A = K(x)M(x)M + ..., B = M(x)M(x)M, nev = 100, blockSize = 20,
tol 1e-8, seeded synthetic data.  The matrices are resident in HBM; a 256 MB buffer
(> L2) is written before every timed step.  ``value`` is the median mixed-precision
time to solution over the timed steps (the solves run without per-kernel events);
``fp64`` the median of the plain FP64 GPU path; ``e2e`` the same mixed solve through
the public API from host CSR (create with the CSR upload, solve, eigenvalues and
eigenvectors back to host memory).  One extra profiled solve (events around every
launch, not timed) gives the kernel classes and the roofline of the dominant one.

``largest`` (on by default, --no-largest skips it): one mixed solve of the largest
single-GPU workload, Q1 on 160^3 nodes with a lognormal coefficient (n = 4,096,000,
nnz = 109,215,352), nev = 1000, blockSize = 100, moving mechanism, with FP64
residuals of 16 eigenpairs recomputed on the host.  Its solve takes minutes, so the
driver's --steps/--warmup repeat the headline workload, not this one.

``--impl reference`` times the FP64 CPU oracle (the reference arm; there is no code of
the paper to run): each step runs its start-up and first two GCG iterations on the
same workload; the line's value extrapolates the per-iteration time to a whole solve
(see ``cpu_baseline.sample``), ms_per_step is what a step actually took.
``--table`` runs every synthetic workload once (mixed and FP64) and prints one JSON
line per run (the per-config table); ``--ablation`` the option studies (dynamic shift,
CG steps, Algorithm 2 vs 3, preconditioner).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "time to nev eigenpairs at rel. residual 1e-8: mixed vs FP64 GPU; SpMM GB/s"
WORKLOAD = "q1_64"
LARGEST = "q1_160"
DESCR = {
    "fd2d_64": "fd2d_64: 5-point FD 64^2 (n=4096), B=I, nev=20, blockSize=10",
    "q1_64": "q1_64: Q1 FEM 64^3 (n=262144, nnz=6859000), B=consistent mass, nev=100, "
             "blockSize=20, tol=1e-8 relative residual",
    "fd3d_128": "fd3d_128: 7-point FD 128^3 (n=2097152), lognormal coefficient, lumped "
                "mass +-10%, nev=200, blockSize=40",
    "q1grad_48": "q1grad_48: Q1 FEM 48^3 (n=110592), coefficient exp(0.5 N(0,1)), nev=10, "
                 "blockSize=2",
    "q1_160": "q1_160: Q1 FEM 160^3 (n=4096000, nnz=109215352), lognormal coefficient "
              "(sigma=1), consistent mass, nev=1000, blockSize=100, moving mechanism",
    "rand_200k": "rand_200k: random symmetric pattern (n=200000, ~61 nonzeros per row), "
                 "diagonally dominant, B=I, nev=50, blockSize=10",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=WORKLOAD)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-largest", action="store_true")
    ap.add_argument("--table", action="store_true",
                    help="one mixed and one FP64 solve of every workload, one JSON line each")
    ap.add_argument("--workloads", default=None,
                    help="comma-separated workload names for --table (default: all)")
    ap.add_argument("--ablation", action="store_true",
                    help="shift / CG-step / orthogonaliser / preconditioner studies")
    ap.add_argument("--kernel-case", default=None,
                    choices=["spmm32", "spmm64", "gram_tc", "vc_tc", "gram64", "vc64",
                             "gram64tc", "vc64tc", "cg32"],
                    help="run one kernel class three times on the workload's shapes (for ncu)")
    return ap.parse_args()


def dist_init(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(name):
    import workloads as W
    p = W.make_config(name)
    nev, bs = W.CONFIGS[name]["nev"], W.CONFIGS[name]["bs"]
    return p, nev, bs


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            for key in ("model name", "CPU part"):
                if line.startswith(key):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


# ------------------------------------------------------------------ clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index):
        self.dev = dev_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"gcge_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return parse_clock_lines(open(self.path).read().splitlines())


def parse_clock_lines(lines):
    """Median SM clock, max clock and the throttle reasons seen in nvidia-smi CSV lines."""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            mx.append(float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


# ------------------------------------------------------------------ rooflines
# FP64 arithmetic peak of GB300 derived from its unit count and clock: FP64 FMA runs
# at 1/64 of the 128 FP32 lanes of an SM, i.e. 2 FMA = 4 flop per clock per SM, and
# 152 SMs x 2.07 GHz x 4 = 1.26 TFLOP/s (NVIDIA's nominal figure is 1.25).
FP64_PEAK_TFLOPS = 1.25
# Digit-plane products per FP64 product in the tensor-core FP64 emulation (pairs of the
# seven 7-bit digits with i + j <= 8): their bf16 flops are 28 x the FP64 flops.
OZ_PAIRS = 28

# DRAM traffic (read + write) over algorithmic bytes per kernel class, measured by ncu
# on each class's kernel at the headline workload's shapes (k = 20 for the SpMM: the CG
# variant with the fused dot 0.83, the plain one 0.84; FP64 SpMM 0.87); None where the
# kernel changed after its counters were taken or the class mixes shapes whose traffic
# differs (the emulated FP64 products).
TRAFFIC_RATIO = {"q1_64": {"spmm": 0.83, "gram": 1.05, "vc": 0.88, "spmm64": 0.87,
                           "gram64": None, "vc64": None, "gram64tc": None, "vc64tc": None}}


def traffic_per_launch(config, cls, prof):
    r = TRAFFIC_RATIO.get(config, {}).get(cls)
    if r is None or not prof or prof["calls"] == 0:
        return None
    return round(r * prof["bytes"] / prof["calls"])


def kernel_rooflines(prof, peaks):
    """Per kernel class: time share and achieved rate against its own roof."""
    hbm, bf16_sust, src = peaks["hbm"], peaks["bf16_sustained"], peaks["source"]
    out = {}
    for k, v in prof.items():
        if k in ("syev", "other") or v["calls"] == 0 or v["ms"] <= 0:
            continue
        sec = v["ms"] / 1e3
        if k.endswith("tc") and k.startswith(("gram64", "vc64")):
            ach = OZ_PAIRS * v["flops"] / sec / 1e12
            out[k] = {"bound": "tensor", "achieved": round(ach, 1), "peak": bf16_sust,
                      "unit": "TFLOP/s", "frac": round(ach / bf16_sust, 4),
                      "peak_source": f"{src} bf16 sustained",
                      "fp64_equiv_tflops": round(v["flops"] / sec / 1e12, 2)}
        elif k in ("gram64", "vc64") or (
                k == "spmm64" and v["flops"] / sec / 1e12 / FP64_PEAK_TFLOPS >
                v["bytes"] / sec / 1e9 / hbm):
            ach = v["flops"] / sec / 1e12
            out[k] = {"bound": "alu", "achieved": round(ach, 3), "peak": FP64_PEAK_TFLOPS,
                      "unit": "TFLOP/s", "frac": round(ach / FP64_PEAK_TFLOPS, 4),
                      "peak_source": "FP64 rate from unit count and clock"}
        else:
            ach = v["bytes"] / sec / 1e9
            out[k] = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                      "frac": round(ach / hbm, 4), "peak_source": src}
        out[k].update(ms=round(v["ms"], 2), calls=int(v["calls"]))
    return out


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm": d.get("hbm_gbs", 6800.0), "bf16": d.get("bf16_tflops", 1900.0),
                "bf16_sustained": d.get("bf16_tflops_sustained", d.get("bf16_tflops", 1700.0)),
                "source": "measured"}
    return {"hbm": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "source": "fallback"}


# ------------------------------------------------------------------ ours
def solve_times(g, torch, p, nev, bs, precision, steps, warmup, stream, flush, evd, world,
                **opts):
    """Median-ready per-solve device times (CUDA events on the solve's stream)."""
    s = g.Solver(p.A, p.B, nev, bs, 1e-8, precision=precision, seed=0, **opts)
    for _ in range(warmup):
        flush.zero_()
        s.solve(evecs_device=evd)
    ms, its, launches = [], [], 0
    for _ in range(steps):
        flush.zero_()
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.solve(evecs_device=evd)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        ms.append(e0.elapsed_time(e1))
        st = s.stats()
        its.append(st["iterations"])
        launches += st["kernel_launches"]
    st = s.stats()
    ev, _ = g.gcge_eigenpairs(s.h, nev, p.n, evd, True)
    s.close()
    return ms, its, launches, st, ev


def run_ours(args, rank, world, local):
    import torch
    import paper_2111_06552_gb300 as g
    import workloads as W

    torch.cuda.set_device(local)
    g.lib()
    p, nev, bs = workload(args.config)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    evd = torch.empty((nev, p.n), dtype=torch.float64, device="cuda")
    with Clocks(local) as clk:
        ms_mx, its_mx, launches_mx, st_mx, ev_mx = solve_times(
            g, torch, p, nev, bs, g.GCGE_MIXED, args.steps, args.warmup, stream, flush, evd,
            world)
        ms_64, its_64, ev_64 = [float("nan")], [None], None
        if args.fp64_steps > 0:
            ms_64, its_64, _, _, ev_64 = solve_times(
                g, torch, p, nev, bs, g.GCGE_FP64, args.fp64_steps, 1, stream, flush, evd, world)
    clocks = clk.summary()
    # profiled solve (events around every launch; not timed): kernel classes, roofline
    sp = g.Solver(p.A, p.B, nev, bs, 1e-8, precision=g.GCGE_MIXED, seed=0, profile=1)
    sp.solve(evecs_device=evd)
    prof = sp.stats()["prof"]
    sp.close()

    exact = W.q1_eigs(64, nev) if args.config == "q1_64" else None
    err = float(np.abs(ev_mx - exact).max() / exact[0]) if exact is not None else None
    err64 = (float(np.abs(ev_mx - ev_64).max() / np.abs(ev_64).max())
             if ev_64 is not None else None)

    t_mx = max_over_ranks(float(np.median(ms_mx)) / 1e3, world)
    t_64 = max_over_ranks(float(np.median(ms_64)) / 1e3, world)
    peaks = measured_peaks()
    kernels = kernel_rooflines(prof, peaks)
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    d = kernels[dom]
    spmm = prof["spmm"]
    spmm_gbs = spmm["bytes"] / (spmm["ms"] / 1e3) / 1e9 if spmm["ms"] > 0 else 0.0
    tot_ms = sum(v["ms"] for v in prof.values())
    roof = {"bound": d["bound"], "kernel": dom, "achieved": d["achieved"], "peak": d["peak"],
            "unit": d["unit"], "frac": d["frac"], "peak_source": d["peak_source"],
            "traffic": traffic_per_launch(args.config, dom, prof.get(dom)),
            "avg_launch_us": round(1e3 * d["ms"] / max(d["calls"], 1), 2),
            "timed_in": "one profiled mixed solve (CUDA events on the solve's stream)"}
    e2e = None if args.no_e2e else run_e2e(g, p, nev, bs, args)
    line = {
        "metric": METRIC, "value": round(t_mx, 5), "unit": "s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t_mx, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": DESCR[args.config],
                   "precision": "mixed (FP32 SpMM/CG/Gram/update, FP64 small dense + FP64 "
                                "phase with tensor-core FP64 products)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "256 MB buffer written before every timed step",
                   "statistic": "median of the timed solves"},
        "fp64": {"value": round(t_64, 5), "unit": "s", "dtype": "f64",
                 "iterations": its_64[0], "steps": args.fp64_steps, "statistic": "median"},
        "iterations": its_mx[0], "iterations_fp32": st_mx["iterations_fp32"],
        "max_rel_eig_err_vs_closed_form": err,
        "max_rel_eig_diff_mixed_vs_fp64": err64,
        "spmm_gbs": round(spmm_gbs, 1),
        "roofline": roof,
        "kernel_share": {k: round(v["ms"] / tot_ms, 4) for k, v in prof.items()} if tot_ms else {},
        "kernels": kernels,
        "gpu_launches": int(launches_mx),
        "clocks": clocks,
    }
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_largest and world == 1:
        del evd
        torch.cuda.empty_cache()
        line["largest"] = run_largest(g, torch, stream)
    return line


def run_e2e(g, p, nev, bs, args):
    """Public-API solve from host buffers: create (H2D CSR), solve, eigenpairs (D2H)."""
    import torch
    csr_bytes = 0
    for M in (p.A, p.B):
        csr_bytes += M.indptr.astype(np.int32).nbytes + M.indices.nbytes + M.data.nbytes
    out_bytes = 8 * nev + 8 * p.n * nev
    times = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = g.Solver(p.A, p.B, nev, bs, 1e-8, precision=g.GCGE_MIXED, seed=0)
        ev, X = s.solve()
        s.close()
        torch.cuda.synchronize()
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    return {"value": round(float(np.median(times)), 5), "unit": "s",
            "h2d_bytes_per_step": int(csr_bytes), "d2h_bytes_per_step": int(out_bytes),
            "statistic": "median"}


def run_largest(g, torch, stream):
    """One mixed solve of the largest workload, with host-side FP64 residuals."""
    import workloads as W
    p, nev, bs = workload(LARGEST)
    evd = torch.empty((nev, p.n), dtype=torch.float64, device="cuda")
    s = g.Solver(p.A, p.B, nev, bs, 1e-8, precision=g.GCGE_MIXED, seed=0, profile=1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    status = g.gcge_solve(s.h)
    e1.record(stream)
    torch.cuda.synchronize()
    ev, nconv = g.gcge_eigenpairs(s.h, nev, p.n, evd, True)
    st = s.stats()
    s.close()
    cols = sorted(set(np.linspace(0, nev - 1, 16).astype(int).tolist()))
    X = evd[cols].cpu().numpy().T
    AX, BX = p.A @ X, p.B @ X
    lam = ev[cols]
    res = np.linalg.norm(AX - BX * lam, axis=0) / (np.abs(lam) * np.sqrt(np.einsum("ij,ij->j", X, BX)))
    spmm = st["prof"]["spmm"]
    del evd
    torch.cuda.empty_cache()
    return {"workload": DESCR[LARGEST], "status": int(status), "nconv": int(nconv),
            "value": round(e0.elapsed_time(e1) / 1e3, 2), "unit": "s", "solves": 1,
            "iterations": st["iterations"], "iterations_fp32": st["iterations_fp32"],
            "cg_steps": st["cg_steps"], "moves": st["moves"],
            "max_sampled_rel_residual": float(res.max()), "sampled_columns": len(cols),
            "spmm_gbs": round(spmm["bytes"] / (spmm["ms"] / 1e3) / 1e9, 1) if spmm["ms"] else None,
            "class_ms": {k: round(v["ms"], 1) for k, v in st["prof"].items() if v["ms"] > 0},
            "note": "one solve per bench run (minutes); timed with per-kernel events on"}


# ------------------------------------------------------------------ oracle (CPU)
def oracle_sample(config):
    """The FP64 oracle's start-up and first two GCG iterations on the workload.

    Returns (wall seconds of the sample, start-up seconds, seconds of one whole GCG
    iteration) -- the iteration is the first one, timed from its STEP 3 to the STEP 3
    of the second, which the sample reaches before it stops."""
    import workloads as W
    from oracle.gcg import gcg, Params
    p, nev, bs = workload(config)
    X0 = W.initial_block(p.n, nev + 3 * bs, 0)
    marks = {}

    def trace(e):
        if e["step"] == 3:
            marks[e["it"]] = time.perf_counter()

    t0 = time.perf_counter()
    gcg(p.A, p.B, nev, bs, 1e-8, X0, Params(max_iter=2, trace=trace))
    t1 = time.perf_counter()
    return t1 - t0, marks[1] - t0, marks[2] - marks[1]


def oracle_iterations(config):
    path = os.path.join(ROOT, "tests", "golden", f"oracle_{config}.json")
    if os.path.exists(path):
        return json.load(open(path)).get("iterations")
    return None


def oracle_threads():
    """Threads the oracle's dense algebra may use (BLAS); its sparse products are
    single-threaded (scipy.sparse)."""
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        v = os.environ.get(var)
        if v and v.isdigit():
            return int(v)
    return os.cpu_count()


def cpu_baseline(config, gpu_iters):
    wall, init, per_it = oracle_sample(config)
    iters = oracle_iterations(config) or gpu_iters
    value = init + per_it * iters
    return {"value": round(value, 2), "unit": "s", "cores": oracle_threads(),
            "sparse_threads": 1, "cpu_model": cpu_model(), "kind": "oracle",
            "sample": f"start-up ({init:.1f} s) and first GCG iteration ({per_it:.1f} s) of the "
                      f"FP64 oracle on the same workload; value = start-up + {iters} "
                      f"iterations (the iteration count of a full oracle run of this "
                      f"workload); the sample took {wall:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    walls, inits, its = [], [], []
    for i in range(args.warmup + args.steps):
        wall, init, per_it = oracle_sample(args.config)
        if i >= args.warmup:
            walls.append(wall)
            inits.append(init)
            its.append(per_it)
    iters = oracle_iterations(args.config) or 60
    v = float(np.median(inits)) + float(np.median(its)) * iters
    ms_step = 1e3 * float(np.median(walls))
    cb = {"value": round(v, 2), "unit": "s", "cores": oracle_threads(), "sparse_threads": 1,
          "cpu_model": cpu_model(), "kind": "oracle",
          "sample": f"each step: the FP64 oracle's start-up and first two GCG iterations on "
                    f"the same workload ({ms_step / 1e3:.1f} s, the step's own time); value = "
                    f"start-up + {iters} whole iterations (median per-iteration time; "
                    f"{iters} = iterations of a full oracle run)"}
    return {"metric": METRIC, "value": round(v, 2), "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 1),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": DESCR[args.config], "statistic": "median"},
            "cpu_baseline": cb,
            "e2e": {"value": round(v, 2), "unit": "s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------------ per-config table
TABLE_WORKLOADS = ("fd2d_64", "q1_64", "fd3d_128", "q1grad_48", "rand_200k", "q1_160")


def run_table(names=None):
    """One mixed and one FP64 solve (after one warm-up each, none for the 160^3 pencil)
    of every workload (or of those named)."""
    import torch
    import paper_2111_06552_gb300 as g
    g.lib()
    stream = torch.cuda.current_stream()
    for name in names or TABLE_WORKLOADS:
        p, nev, bs = workload(name)
        for prec, tag in ((g.GCGE_MIXED, "mixed"), (g.GCGE_FP64, "fp64")):
            s = g.Solver(p.A, p.B, nev, bs, 1e-8, precision=prec, seed=0, profile=1)
            if name != "q1_160":
                s.solve()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            status = g.gcge_solve(s.h)
            e1.record(stream)
            torch.cuda.synchronize()
            st = s.stats()
            ev, nconv = g.gcge_eigenpairs(s.h, nev, p.n)
            s.close()
            prof = st["prof"]
            peaks = measured_peaks()
            ks = kernel_rooflines(prof, peaks)
            print(json.dumps({"workload": name, "precision": tag, "status": int(status),
                              "seconds": round(e0.elapsed_time(e1) / 1e3, 3),
                              "iterations": st["iterations"], "nconv": int(nconv),
                              "evals_head": [float(x) for x in ev[:3]],
                              "evals": [float(x) for x in ev],
                              "kernels": ks}), flush=True)


# ------------------------------------------------------------------ ablations
def run_ablation():
    """The paper's option studies on the synthetic workloads, one solve each (after one
    warm-up solve of the workload): dynamic shift on/off x CG steps per GCG iteration
    (Section 4.1, Table 3), Algorithm 2 vs Algorithm 3 (Table 8), and the Jacobi-
    preconditioned inner solve.  One JSON line per solve with the per-STEP split."""
    import torch
    import paper_2111_06552_gb300 as g
    g.lib()
    stream = torch.cuda.current_stream()
    runs = []
    for name, cgs in (("fd2d_64", (5, 10, 20, 30)), ("q1_64", (5, 10, 20, 30)),
                      ("fd3d_128", (10, 30))):
        for shift in (1, 0):
            for cg in cgs:
                runs.append((name, g.GCGE_MIXED, dict(use_shift=shift, cg_max_iter=cg)))
        for prec in (g.GCGE_FP64, g.GCGE_MIXED):
            runs.append((name, prec, dict(orth=g.GCGE_ORTH_ALG2)))
            runs.append((name, prec, dict(orth=g.GCGE_ORTH_ALG3)))
        runs.append((name, g.GCGE_MIXED, dict(precond=g.GCGE_PRECOND_JACOBI)))
    warmed = set()
    cache = {}
    for name, prec, opts in runs:
        if name not in cache:
            cache.clear()
            cache[name] = workload(name)
        p, nev, bs = cache[name]
        if name not in warmed:
            s = g.Solver(p.A, p.B, nev, bs, 1e-8, precision=prec, seed=0)
            s.solve()
            s.close()
            warmed.add(name)
        s = g.Solver(p.A, p.B, nev, bs, 1e-8, precision=prec, seed=0, **opts)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        status = g.gcge_solve(s.h)
        e1.record(stream)
        torch.cuda.synchronize()
        st = s.stats()
        ev, nconv = g.gcge_eigenpairs(s.h, nev, p.n)
        s.close()
        print(json.dumps({"workload": name, "precision": "mixed" if prec else "fp64",
                          **opts, "status": int(status),
                          "seconds": round(e0.elapsed_time(e1) / 1e3, 3),
                          "iterations": st["iterations"],
                          "iterations_fp32": st["iterations_fp32"],
                          "cg_steps": st["cg_steps"], "nconv": int(nconv),
                          "ms_step": [round(x, 1) for x in st["ms_step"]],
                          "ev_sum": float(np.sum(ev))}), flush=True)


# ------------------------------------------------------------------ ncu cases
def kernel_case(args):
    """Three launches of one kernel class on the benchmark workload's shapes, no timing:
    the command that the committed ncu summaries capture."""
    import torch
    import paper_2111_06552_gb300 as g
    g.lib()
    p, nev, bs = workload(args.config)
    n = p.n
    torch.manual_seed(0)
    rp = torch.tensor(p.A.indptr.astype(np.int32), device="cuda")
    ci = torch.tensor(p.A.indices.astype(np.int32), device="cuda")
    d, q, k = nev + 3 * bs + 2 * bs, nev + 3 * bs, bs   # RR basis width, X width, block
    for _ in range(3):
        if args.kernel_case in ("spmm32", "spmm64"):
            dt = torch.float32 if args.kernel_case == "spmm32" else torch.float64
            val = torch.tensor(p.A.data, device="cuda").to(dt)
            X = torch.randn(n, k, device="cuda", dtype=dt)
            Y = torch.empty(n, k, device="cuda", dtype=dt)
            f = g.gcge_spmm_f32 if dt == torch.float32 else g.gcge_spmm_f64
            f(n, rp, ci, val, k, 1.0, X, k, 0.0, Y, k)
        elif args.kernel_case == "cg32":
            val = torch.tensor(p.A.data, device="cuda").float()
            Bm = torch.randn(n, k, device="cuda")
            X = torch.zeros(n, k, device="cuda")
            g.gcge_block_cg_f32(n, rp, ci, val, k, Bm, k, X, k, 2, 1e-30)
        elif args.kernel_case in ("gram_tc", "gram64", "gram64tc"):
            dt = torch.float32 if args.kernel_case == "gram_tc" else torch.float64
            X = torch.randn(n, d, device="cuda", dtype=dt)
            Y = torch.randn(n, k, device="cuda", dtype=dt)
            C = torch.zeros(k, d, device="cuda", dtype=torch.float64)
            if args.kernel_case == "gram_tc":
                g.gcge_gram_f32(n, d, k, 1.0, X, d, Y, k, 0.0, C, d, tc=1)
            elif args.kernel_case == "gram64tc":
                g.gcge_gram_f64_tc(n, d, k, 1.0, X, d, Y, k, 0.0, C, d)
            else:
                g.gcge_gram_f64(n, d, k, 1.0, X, d, Y, k, 0.0, C, d)
        else:
            dt = torch.float32 if args.kernel_case == "vc_tc" else torch.float64
            V = torch.randn(n, d, device="cuda", dtype=dt)
            Cm = torch.randn(q, d, device="cuda", dtype=torch.float64)
            Z = torch.empty(n, q, device="cuda", dtype=dt)
            if args.kernel_case == "vc_tc":
                g.gcge_vc_f32(n, d, q, 1.0, V, d, Cm, d, 0.0, Z, q, tc=1)
            elif args.kernel_case == "vc64tc":
                g.gcge_vc_f64_tc(n, d, q, 1.0, V, d, Cm, d, 0.0, Z, q)
            else:
                g.gcge_vc_f64(n, d, q, 1.0, V, d, Cm, d, 0.0, Z, q)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_case": args.kernel_case, "n": n, "d": d, "q": q, "k": k}))


def main():
    args = parse()
    if args.kernel_case:
        kernel_case(args)
        return
    if args.table:
        names = [w for w in args.workloads.split(",") if w] if args.workloads else None
        for w in names or ():
            if w not in TABLE_WORKLOADS:
                raise SystemExit(f"unknown workload {w!r}; choose from {TABLE_WORKLOADS}")
        run_table(names)
        return
    if args.ablation:
        run_ablation()
        return
    rank, world, local = dist_init(args.gpus)
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    line = run_ours(args, rank, world, local)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(args.config, line["iterations"])
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
