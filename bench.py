#!/usr/bin/env python
"""Benchmark: time to the nev smallest eigenpairs at relative residual 1e-8.

Workload: 3D Q1 FEM Laplacian on 64^3 interior nodes (n = 262,144, 27-point
pattern, nnz = 6,859,000), generalized pencil A = K(x)M(x)M + ..., B = M(x)M(x)M,
nev = 100, blockSize = 20, seeded synthetic data (no external matrix).

One step = one complete gcge_solve (Algorithm 1 to convergence) with the
matrices already resident in HBM.  ``value`` is the mixed-precision time to
solution (seconds, lower is better); the plain FP64 GPU path is reported
beside it.  ``e2e`` repeats the measurement through the public C API from host
buffers: gcge_create (CSR upload), gcge_solve and gcge_eigenpairs (eigenvalues
and eigenvectors back to the host) inside the timed region.

``--impl reference`` times the FP64 CPU oracle instead (a bounded sample per step,
scaled to the time-to-solution unit).
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
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "time to nev eigenpairs at rel. residual 1e-8: mixed vs FP64 GPU; SpMM GB/s"
WORKLOAD = "q1_64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=WORKLOAD)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-profile", action="store_true",
                    help="no per-kernel CUDA-event profile (fewer API calls under ncu)")
    ap.add_argument("--kernel-case", default=None,
                    choices=["spmm32", "spmm64", "gram_tc", "vc_tc", "gram64", "vc64"],
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
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
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


# FP64 arithmetic peak of GB300 (nominal; the FP64 classes are bound by it, not by HBM)
FP64_PEAK_TFLOPS = 1.25

# DRAM traffic (read + write) over algorithmic bytes, per kernel class, from one full
# ncu capture of each class on the q1_64 shapes (profiles/kernels_q1_64_shapes.md);
# traffic per launch = this ratio x the class's algorithmic bytes per launch.
TRAFFIC_RATIO = {"q1_64": {"spmm": 0.84, "gram": 1.05, "vc": 0.88, "spmm64": 0.98,
                           "gram64": 1.01, "vc64": 3.30}}


def traffic_per_launch(config, cls, prof):
    r = TRAFFIC_RATIO.get(config, {}).get(cls)
    if r is None or not prof or prof["calls"] == 0:
        return None
    return round(r * prof["bytes"] / prof["calls"])


def kernel_rooflines(prof, hbm, src):
    """Per kernel class: time share and achieved rate against its own roof."""
    out = {}
    for k, v in prof.items():
        if k in ("syev", "other") or v["calls"] == 0 or v["ms"] <= 0:
            continue
        if k.endswith("64") and k != "spmm64":
            ach = v["flops"] / (v["ms"] / 1e3) / 1e12
            out[k] = {"bound": "alu", "achieved": round(ach, 3), "peak": FP64_PEAK_TFLOPS,
                      "unit": "TFLOP/s", "frac": round(ach / FP64_PEAK_TFLOPS, 4),
                      "peak_source": "nominal FP64 rate"}
        elif k == "spmm64" and v["flops"] / (v["ms"] / 1e3) / 1e12 / FP64_PEAK_TFLOPS > \
                v["bytes"] / (v["ms"] / 1e3) / 1e9 / hbm:
            ach = v["flops"] / (v["ms"] / 1e3) / 1e12
            out[k] = {"bound": "alu", "achieved": round(ach, 3), "peak": FP64_PEAK_TFLOPS,
                      "unit": "TFLOP/s", "frac": round(ach / FP64_PEAK_TFLOPS, 4),
                      "peak_source": "nominal FP64 rate"}
        else:
            ach = v["bytes"] / (v["ms"] / 1e3) / 1e9
            out[k] = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                      "frac": round(ach / hbm, 4), "peak_source": src}
        out[k].update(ms=round(v["ms"], 2), calls=int(v["calls"]))
    return out


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


# ------------------------------------------------------------------ ours
def run_ours(args, rank, world, local):
    import torch
    import paper_2111_06552_gb300 as g

    torch.cuda.set_device(local)
    g.lib()
    p, nev, bs = workload(args.config)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2

    def make(precision):
        return g.Solver(p.A, p.B, nev, bs, 1e-8, precision=precision, seed=0,
                        profile=0 if args.no_profile else 1)

    def timed(solver, steps, warmup):
        for _ in range(warmup):
            flush.zero_()
            solver.solve(evecs_device=evd)
        ms = []
        prof_tot = None
        its = []
        for _ in range(steps):
            flush.zero_()
            barrier(world)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            solver.solve(evecs_device=evd)
            e1.record(stream)
            torch.cuda.synchronize()
            barrier(world)
            ms.append(e0.elapsed_time(e1))
            st = solver.stats()
            its.append(st["iterations"])
            if prof_tot is None:
                prof_tot = {k: dict(v) for k, v in st["prof"].items()}
                launches = st["kernel_launches"]
                stats0 = st
            else:
                for k, v in st["prof"].items():
                    for f in v:
                        prof_tot[k][f] += v[f]
                launches += st["kernel_launches"]
        return ms, prof_tot, launches, its, stats0

    evd = torch.empty((nev, p.n), dtype=torch.float64, device="cuda")
    res = {}
    with Clocks(local) as clk:
        sm = make(g.GCGE_MIXED)
        ms_mx, prof_mx, launches_mx, its_mx, st_mx = timed(sm, args.steps, args.warmup)
        ev_mx, _ = g.gcge_eigenpairs(sm.h, nev, p.n, evd, True)
        sm.close()
        ms_64, its_64 = [float("nan")], [None]
        if args.fp64_steps > 0:
            s64 = make(g.GCGE_FP64)
            ms_64, prof_64, launches_64, its_64, st_64 = timed(s64, args.fp64_steps, 1)
            s64.close()
    clocks = clk.summary()
    # accuracy of the timed result against the closed-form spectrum
    import workloads as W
    exact = W.q1_eigs(64, nev) if args.config == "q1_64" else None
    err = float(np.abs(ev_mx - exact).max() / exact[0]) if exact is not None else None

    t_mx = max_over_ranks(float(np.mean(ms_mx)) / 1e3, world)
    t_64 = max_over_ranks(float(np.mean(ms_64)) / 1e3, world)

    # roofline of the dominant kernel class inside the timed mixed solves
    hbm, bf16, src = measured_peaks()
    kernels = kernel_rooflines(prof_mx, hbm, src)
    if not kernels:   # --no-profile: no per-kernel times
        kernels = {"none": {"bound": None, "achieved": None, "peak": None, "unit": None,
                            "frac": None, "peak_source": None, "ms": 0.0, "calls": 0}}
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    d = kernels[dom]
    spmm = prof_mx["spmm"]
    spmm_gbs = spmm["bytes"] / (spmm["ms"] / 1e3) / 1e9 if spmm["ms"] > 0 else 0.0
    tot_ms = sum(v["ms"] for v in prof_mx.values())
    roof = {"bound": d["bound"], "kernel": dom, "achieved": d["achieved"], "peak": d["peak"],
            "unit": d["unit"], "frac": d["frac"], "peak_source": d["peak_source"],
            "traffic": traffic_per_launch(args.config, dom, prof_mx.get(dom)),
            "avg_launch_us": round(1e3 * d["ms"] / max(d["calls"], 1), 2)}
    res.update(t_mx=t_mx, t_64=t_64)

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(g, p, nev, bs, args, stream)
    line = {
        "metric": METRIC, "value": round(t_mx, 5), "unit": "s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t_mx, 3),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": "q1_64: Q1 FEM 64^3 (n=262144, nnz=6859000), B=consistent mass, "
                               "nev=100, blockSize=20, tol=1e-8 relative residual",
                   "precision": "mixed (FP32 SpMM/CG/Gram/update, FP64 small dense + FP64 refinement)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "256 MB buffer written between timed steps"},
        "fp64": {"value": round(t_64, 5), "unit": "s", "dtype": "f64",
                 "iterations": its_64[0], "steps": args.fp64_steps},
        "iterations": its_mx[0], "iterations_fp32": st_mx["iterations_fp32"],
        "max_rel_eig_err_vs_closed_form": err,
        "spmm_gbs": round(spmm_gbs, 1),
        "roofline": roof,
        "kernel_share": {k: round(v["ms"] / tot_ms, 4) for k, v in prof_mx.items()} if tot_ms else {},
        "kernels": kernels,
        "gpu_launches": int(launches_mx),
        "clocks": clocks,
    }
    if e2e is not None:
        line["e2e"] = e2e
    return line


def run_e2e(g, p, nev, bs, args, stream):
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
    return {"value": round(float(np.mean(times)), 5), "unit": "s", "h2d_bytes_per_step": int(csr_bytes),
            "d2h_bytes_per_step": int(out_bytes)}


# ------------------------------------------------------------------ oracle (CPU)
def oracle_sample(config, iters=2):
    """Time the FP64 oracle on the first `iters` GCG iterations of the workload."""
    import workloads as W
    from oracle.gcg import gcg, Params
    p, nev, bs = workload(config)
    X0 = W.initial_block(p.n, nev + 3 * bs, 0)
    t0 = time.perf_counter()
    r = gcg(p.A, p.B, nev, bs, 1e-8, X0, Params(max_iter=iters))
    dt = time.perf_counter() - t0
    return dt, r.iterations


def oracle_iterations(config):
    path = os.path.join(ROOT, "tests", "golden", f"oracle_{config}.json")
    if os.path.exists(path):
        return json.load(open(path)).get("iterations")
    return None


def cpu_baseline(config, gpu_iters):
    dt, it = oracle_sample(config)
    iters = oracle_iterations(config) or gpu_iters
    per_it = dt / it
    return {"value": round(per_it * iters, 2), "unit": "s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"first {it} GCG iterations of the same workload (incl. the initial "
                      f"orthonormalisation) took {dt:.1f} s; scaled by {iters} iterations to solution"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    times = []
    for i in range(args.warmup + args.steps):
        dt, it = oracle_sample(args.config, iters=1 if i < args.warmup else 2)
        if i >= args.warmup:
            times.append(dt / it)
    iters = oracle_iterations(args.config) or 60
    v = float(np.mean(times)) * iters
    return {"metric": METRIC, "value": round(v, 2), "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * v, 1),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "q1_64: Q1 FEM 64^3 (n=262144, nnz=6859000), nev=100, "
                                   "blockSize=20, tol=1e-8"},
            "cpu_baseline": {"value": round(v, 2), "unit": "s", "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"per step: 2 GCG iterations of the FP64 oracle, "
                                       f"scaled by {iters} iterations to solution"},
            "e2e": {"value": round(v, 2), "unit": "s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


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
        elif args.kernel_case in ("gram_tc", "gram64"):
            dt = torch.float32 if args.kernel_case == "gram_tc" else torch.float64
            X = torch.randn(n, d, device="cuda", dtype=dt)
            Y = torch.randn(n, k, device="cuda", dtype=dt)
            C = torch.zeros(k, d, device="cuda", dtype=torch.float64)
            if dt == torch.float32:
                g.gcge_gram_f32(n, d, k, 1.0, X, d, Y, k, 0.0, C, d, tc=1)
            else:
                g.gcge_gram_f64(n, d, k, 1.0, X, d, Y, k, 0.0, C, d)
        else:
            dt = torch.float32 if args.kernel_case == "vc_tc" else torch.float64
            V = torch.randn(n, d, device="cuda", dtype=dt)
            Cm = torch.randn(q, d, device="cuda", dtype=torch.float64)
            Z = torch.empty(n, q, device="cuda", dtype=dt)
            if dt == torch.float32:
                g.gcge_vc_f32(n, d, q, 1.0, V, d, Cm, d, 0.0, Z, q, tc=1)
            else:
                g.gcge_vc_f64(n, d, q, 1.0, V, d, Cm, d, 0.0, Z, q)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_case": args.kernel_case, "n": n, "d": d, "q": q, "k": k}))


def main():
    args = parse()
    if args.kernel_case:
        kernel_case(args)
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
