"""Benchmark: adaptive outer iterations per second on one GB300.

Workload "full_adaptive": random hypergraph with n = 1,000,000 vertices, m = 2,000,000
hyperedges, truncated power-law hyperedge sizes on 2..2000 (exponent solved for a mean
of 10, about 20M incidences), Y n x 512 binary with 0.5% ones, lam = 0.5, w0 = 1/m,
eta = 1e-2.  A step is one outer iteration of the alternation (solve M F = lam Y at w,
warm-started from the previous F, to a relative residual that bounds the relative
error by 1e-5; then the gradient of P(w) and the projected step on w), computed by
libhgl in mixed precision (FP32 panels, FP64 refinement and reductions).  The plain
FP64 block CG of the same library is timed on the same GPU as the comparator.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Prints one JSON line on rank 0.
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

import synth  # noqa: E402

WORKLOAD = "full_adaptive"
METRIC = "adaptive outer iterations/sec (rel err <= 1e-5)"
UNIT = "iters/s"
TOL = 3e-6          # relative residual; kappa(M) <= 3 at lam = 0.5 -> relative error <= 9e-6
SEED = 20190822


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hgl", choices=["hgl", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--scale", type=float, default=1.0, help="shrink n and m (testing only)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparator")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) < 9:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def make_inputs(scale: float):
    wl = synth.WORKLOADS[WORKLOAD]
    n = int(wl.n * scale)
    m = int(wl.m * scale)
    t0 = time.time()
    d = synth.make_hypergraph(wl, SEED, n=n, m=m, tags_dtype=np.float64)
    d["gen_s"] = time.time() - t0
    d["wl"] = wl
    return d


def theta_algorithmic_bytes(n, m, nnz, c, elt):
    """Compulsory bytes of one operator apply Z = a X + b Theta X (one column chunk):
    index arrays once, X read by both passes, the intermediate m x c panel written
    and read once, Z written once, and the scaling vectors."""
    index = 2 * 4 * nnz + 8 * (n + 1) + 8 * (m + 1)
    panels = 2 * n * c * elt + 2 * m * c * 4 + n * c * elt
    scal = 8 * (2 * n + m)
    return index + panels + scal


def cpu_baseline(d, gpu_iters_per_step: float, sample_cols: int = 8, max_s: float = 25.0):
    """Time the oracle's FP64 CG iteration (scipy.sparse operator) on the full graph with
    a few columns, and scale to one outer iteration at c columns."""
    from oracle import core, incidence
    t0 = time.time()
    og = incidence.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
    H = incidence.incidence_matrix(og)
    build_s = time.time() - t0
    w = d["w0"]
    Y = d["Y"][:, :sample_cols]
    lam = d["wl"].lam
    t1 = time.time()
    its = 0
    out = None
    # a single CG iteration block: one operator apply + vector updates per iteration
    while True:
        its += 1
        out = core.cg_solve(H, w, lam, Y, tol=1e-30, max_iter=its)
        if time.time() - t1 > max_s / 3 or its >= 3:
            break
    per_call = (time.time() - t1)
    # cg_solve(max_iter=k) runs k iterations + 2 operator applies (initial, final residual)
    total_iters = its * (its + 1) // 2
    total_applies = total_iters + 2 * its
    per_apply = per_call / total_applies
    c = d["c"]
    per_outer = (gpu_iters_per_step + 2) * per_apply * (c / sample_cols)
    return {"value": 1.0 / per_outer, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"FP64 oracle CG (scipy.sparse) on the full n={d['n']} m={d['m']} graph with "
                       f"{sample_cols} of {c} columns, {total_iters} iterations timed; one outer iteration "
                       f"= {gpu_iters_per_step:.0f} CG iterations + gradient, scaled by {c}/{sample_cols} columns"),
            "seconds_per_outer_iter_extrapolated": per_outer, "oracle_build_s": build_s}


def run_reference(args, rank):
    """--impl reference: the oracle (FP64, numpy/scipy on host cores) on a bounded sample."""
    if rank != 0:
        return
    d = make_inputs(args.scale)
    iters = 16.0
    res = []
    for _ in range(args.warmup + args.steps):
        res.append(cpu_baseline(d, iters, sample_cols=4, max_s=6.0))
    vals = [r["value"] for r in res[args.warmup:]]
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": d["n"], "m": d["m"], "nnz": int(d["edge_ptr"][-1]),
                       "c": d["c"], "lam": d["wl"].lam},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": res[-1]["sample"], "value": v},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import torch
    import torch.distributed as dist

    from paper_1908_08281_gb300 import build as _build
    from paper_1908_08281_gb300 import hgl

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _build.build()
    hgl.lib()

    d = make_inputs(args.scale)
    wl = d["wl"]
    n, m, c = d["n"], d["m"], d["c"]
    nnz = int(d["edge_ptr"][-1])
    g = hgl.build_incidence(n, m, d["edge_ptr"], d["members"])
    Yh = torch.from_numpy(d["Y"])
    Y = hgl.padded_panel(n, c, torch.float64, dev)
    Y.copy_(Yh)
    w = torch.tensor(d["w0"], device=dev)
    F = hgl.padded_panel(n, c, torch.float64, dev)
    stream = torch.cuda.current_stream()

    def step(Fp, wp, dtype=hgl.HGL_FP32):
        return hgl.adaptive_step(g, wp, Y, Fp, lam=wl.lam, mu=wl.mu, eta=wl.eta, tol=TOL, dtype=dtype,
                                 raise_on_fail=True)

    # L2 is 129 MB; every panel here (>= 2 GB) is larger, so no flush is needed.
    iters_seen = []
    for _ in range(args.warmup):
        st = step(F, w)
        iters_seen.append(st.solve.iters)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    stats = []
    for _ in range(args.steps):
        stats.append(step(F, w))
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_per_step = ms / args.steps
    value = world * args.steps / (ms / 1000.0)
    solve_iters = float(np.mean([s.solve.iters for s in stats]))
    relres_max = max(s.solve.relres_max for s in stats)

    # dominant kernel family: the operator apply in the inner FP32 CG, timed with events
    X32 = hgl.padded_panel(n, c, torch.float32, dev)
    X32.copy_(F[:, :c].float())
    Z32 = hgl.padded_panel(n, c, torch.float32, dev)
    for _ in range(2):
        hgl.apply_theta(g, w, X32, 1.5, -1.0, Z=Z32)
    torch.cuda.synchronize()
    reps = 5
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(reps):
        hgl.apply_theta(g, w, X32, 1.5, -1.0, Z=Z32)
    a1.record(stream)
    torch.cuda.synchronize()
    theta_ms = a0.elapsed_time(a1) / reps
    peak, peak_kind = measured_peaks()
    alg = theta_algorithmic_bytes(n, m, nnz, c, 4)
    achieved = alg / (theta_ms / 1000.0) / 1e9
    del X32, Z32

    # end to end through the public API: host Y (pinned) and w in, w and statistics out
    Yp = torch.empty((n, Y.stride(0)), dtype=torch.float64).pin_memory()
    Yp[:, :c].copy_(Yh)
    wp_host = w.cpu().pin_memory()
    w_out = torch.empty_like(wp_host).pin_memory()
    e2e_steps = max(1, min(3, args.steps))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        Ybuf = Y.as_strided((n, Y.stride(0)), (Y.stride(0), 1))
        Ybuf.copy_(Yp, non_blocking=True)
        w.copy_(wp_host, non_blocking=True)
        step(F, w)
        w_out.copy_(w, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    h2d = Yp.numel() * 8 + wp_host.numel() * 8
    d2h = w_out.numel() * 8 + 64

    fp64 = None
    if not args.no_fp64:
        F64 = F.clone()
        w64 = w.clone()
        step(F64, w64, hgl.HGL_FP64)  # warm
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        b0.record(stream)
        st64 = step(F64, w64, hgl.HGL_FP64)
        b1.record(stream)
        torch.cuda.synchronize()
        f64_ms = b0.elapsed_time(b1)
        fp64 = {"ms_per_step": f64_ms, "value": 1000.0 / f64_ms, "unit": UNIT, "cg_iters": st64.solve.iters,
                "relres_max": st64.solve.relres_max, "speedup_of_mixed": f64_ms / ms_per_step}
        del F64, w64

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(d, solve_iters)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "m": m, "nnz": nnz, "c": c, "lam": wl.lam, "mu": wl.mu,
                       "eta": wl.eta, "tol_relres": TOL, "size_law": synth.describe_sizes(wl),
                       "panel_dtype": "fp32", "route": "cg", "l2_flush": "inputs larger than L2 (>= 2 GB panels)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "solve": {"cg_iters_per_step": solve_iters, "relres_max": relres_max},
            "roofline": {"kernel": "operator apply (hyperedge + vertex gather passes), FP32, c=512",
                         "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": peak_kind, "traffic": None,
                         "algorithmic_bytes": alg, "ms_per_launch": theta_ms},
            "e2e": {"value": 1.0 / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "fp64_block_cg": fp64,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": None,
            "gen_s": d["gen_s"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
