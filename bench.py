"""Benchmark: adaptive outer iterations per second on one GB300.

Workload "full_adaptive": random hypergraph with n = 1,000,000 vertices, m = 2,000,000
hyperedges, truncated power-law hyperedge sizes on 2..2000 (exponent solved for a mean
of 10, about 20M incidences), Y n x 512 binary with 0.5% ones, lam = 0.5, w0 = 1/m,
eta = 2e-13 (each step moves w by 4-5% of its norm), 20 outer iterations.

A step is one outer iteration of that 20-iteration adaptive loop (the state w, F is
reset to w0, 0 every 20 steps): the block rSVD preconditioner at the current w
(diagonal blocks of 1,024-8,192 vertices, k = 64, p = 10, q = 2, BF16 tensor cores),
the preconditioned CG solve warm-started from the previous F to a relative residual
that bounds the relative error by 1e-5 (FP32 panels inside FP64-accurate
refinement), the gradient of P(w) and the projected step on w -- replayed as one
captured CUDA graph per outer iteration (--no-graph: eager launches).  The comparator is
the plain FP64 conjugate gradient of the same library (one CG per column, Eqs. 16-20,
no preconditioner) on the same loop on the same GPU; the mixed-precision CG without the
block preconditioner is timed beside both.  Accuracy is judged at the loop level: the
final F and w of each timed loop against a tight FP64 loop (tol 1e-10) of the same
20 outer iterations.

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
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per call of a kernel family on
# the full workload at a given panel type and column chunk, from one ncu capture of this
# bench (summarised under profiles/); reported as roofline.traffic only for a run of that
# workload with that chunk.
NCU_TRAFFIC_PER_LAUNCH = {("operator", "bf16", 256): 49.15e9}
LOOP = 20           # outer iterations of one adaptive loop
K_RANK, P_OVER, Q_ITERS = 64, 10, 2
BCG_S, BCG_STEPS = 32, 4   # block CG comparator: columns per group, outer iterations timed


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hgl", choices=["hgl", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="shrink n and m (testing only)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparator")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end measurement")
    ap.add_argument("--eta", type=float, default=None, help="override the workload's step size")
    ap.add_argument("--no-tune", action="store_true", help="keep the default column chunks (no autotuning)")
    ap.add_argument("--no-graph", action="store_true", help="run each outer iteration eagerly (no CUDA graph)")
    ap.add_argument("--panels", default="bf16", choices=["fp32", "bf16"],
                    help="search-direction storage of the headline loop's inner CG (the other is timed beside it)")
    ap.add_argument("--schur", default=None,
                    help="time the nested Schur-complement inverse at these vertex counts (comma list) and exit")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(ms: float, world: int, device) -> float:
    """The job's time: the slowest rank's timed region (all-reduce MAX over the group)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


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
            threading.Thread(target=self._read, daemon=True).start()
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

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in self.rows if len(r) >= 9 and num(r[1]) is not None]
        mx = [num(r[2]) for r in self.rows if len(r) >= 9 and num(r[2]) is not None]
        pw = [num(r[3]) for r in self.rows if len(r) >= 9 and num(r[3]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) >= 9:
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("bf16_tflops", 1925.6)), "measured"
    return 6800.0, 1900.0, "fallback"


def make_inputs(scale: float):
    wl = synth.WORKLOADS[WORKLOAD]
    t0 = time.time()
    d = synth.make_hypergraph(wl, SEED, n=int(wl.n * scale), m=int(wl.m * scale), tags_dtype=np.float64)
    d["gen_s"] = time.time() - t0
    d["wl"] = wl
    return d


# ---- algorithmic bytes per launch of each kernel family (index + panels + vectors) ----

def bytes_operator(n, m, nnz, c, elt, chunks=1, elt_z=None):
    """Operator apply Z = a X + b Theta X: per column chunk the indices; X read by both
    passes, the m x c intermediate (FP32) written and read once, Z written once."""
    elt_z = elt if elt_z is None else elt_z
    return chunks * (2 * 4 * nnz + 8 * (n + m + 2)) + 2 * n * c * elt + 2 * m * c * 4 + n * c * elt_z \
        + 8 * (2 * n + m)


def bytes_residual(n, m, nnz, c, chunks):
    """Pair-arithmetic residual: per chunk the indices; F as two FP32 panels read by both
    passes, the intermediate pair panel written and read, Y (FP64) read, R (FP32) written."""
    return chunks * (2 * 4 * nnz + 8 * (n + m + 2)) + 2 * (8 * n * c) + 2 * (8 * m * c) + 8 * n * c + 4 * n * c \
        + 4 * 2 * (n + m)


def bytes_opresid(n, m, nnz, c, chunks):
    """FP32 residual estimate by one operator pass: per chunk the indices; F (FP32 high
    part) read by both passes, the m x c intermediate written and read, Y (FP64) read,
    R (FP32) written."""
    return chunks * (2 * 4 * nnz + 8 * (n + m + 2)) + 2 * (4 * n * c) + 2 * (4 * m * c) + 8 * n * c + 4 * n * c \
        + 8 * (2 * n + m)


def bytes_gemm(block_ptr, lpad):
    """Grouped GEMM: every dense block once (BF16, padded to 128 rows x 64 columns), the
    transposed basis once, the FP32 output once."""
    sizes = np.diff(np.asarray(block_ptr, dtype=np.int64))
    rows = ((sizes + 127) // 128) * 128
    cols = ((sizes + 63) // 64) * 64
    a = int((rows * cols).sum()) * 2
    return a + lpad * int(cols.sum()) * 2 + int(rows.sum()) * lpad * 4


def flops_gemm(block_ptr, lpad):
    sizes = np.diff(np.asarray(block_ptr, dtype=np.int64))
    return 2.0 * float((sizes.astype(np.float64) ** 2).sum()) * lpad


def bytes_gradient(n, m, nnz, c):
    """Gradient (FP32 panel, one chunk): as the operator apply without the Z write, plus
    the per-hyperedge and per-vertex scalar vectors and the final hyperedge pass."""
    return 2 * 4 * nnz + 8 * (n + m + 2) + 2 * n * c * 4 + 2 * m * c * 4 + 8 * (2 * n + m) + 4 * nnz + 8 * (2 * m + n)


# CG iterations per outer iteration of the GPU loop on this workload (its mean over a
# 20-iteration loop: 7.0 on the BR route, 6.35 for the plain FP64 CG); the oracle's
# sampled step is scaled to this many
REF_ITERS_PER_STEP = 7.0


def oracle_prepare(d):
    """The oracle's incidence matrix of the workload (built once, outside the samples)."""
    from oracle import incidence
    t0 = time.time()
    H = incidence.incidence_matrix(incidence.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"]))
    return H, time.time() - t0


def oracle_step_sample(d, H, block_ptr, iters_per_step: float, sample_cols: int, sample_blocks: int):
    """The oracle (numpy/scipy, FP64, host cores) on a bounded sample of one outer
    iteration, scaled to the full step: 2 CG iterations and 2 residual applies on the
    full graph with a few columns (scaled by c / columns), the gradient on the same
    columns, Algorithm 1 on the smallest blocks (scaled by sum b^2 over the sampled
    b^2: the dense block products dominate), the projection."""
    from oracle import core, philox, rsvd
    wl = d["wl"]
    w = d["w0"]
    c = d["c"]
    Y = d["Y"][:, :sample_cols]
    t1 = time.time()
    core.cg_solve(H, w, wl.lam, Y, tol=1e-30, max_iter=2)   # 2 iterations + 2 residual applies
    t_apply = (time.time() - t1) / 4.0 * (c / sample_cols)
    t2 = time.time()
    core.weight_grad(H, w, Y, wl.mu)
    t_grad = (time.time() - t2) * (c / sample_cols)
    sizes = np.diff(np.asarray(block_ptr, dtype=np.int64))
    pick = np.argsort(sizes, kind="stable")[:sample_blocks]
    t3 = time.time()
    for b in pick:
        Tb = rsvd.block_theta(H, w, [block_ptr[b], block_ptr[b + 1]])[0]
        Om = philox.omega(np.arange(block_ptr[b], block_ptr[b + 1]), K_RANK + P_OVER, SEED)
        rsvd.rsvd_ritz(Tb, Om, Q_ITERS, K_RANK)
    t_rsvd = (time.time() - t3) * float((sizes.astype(np.float64) ** 2).sum() / (sizes[pick].astype(np.float64) ** 2).sum())
    t4 = time.time()
    core.project_simplex(w - wl.eta * np.ones_like(w))
    t_proj = time.time() - t4
    per_step = t_rsvd + (iters_per_step + 2.0) * t_apply + t_grad + t_proj
    nb = len(block_ptr) - 1
    desc = (f"FP64 oracle on n={d['n']} m={d['m']}: 2 CG iterations + 2 residuals with {sample_cols} of {c} "
            f"columns (scaled by {c}/{sample_cols}), gradient on the same columns, Algorithm 1 on the "
            f"{sample_blocks} smallest of {nb} blocks (scaled by sum b^2), projection; one step = rSVD + "
            f"{iters_per_step:.1f} CG iterations + 2 residuals + gradient")
    return per_step, {"rsvd": t_rsvd, "apply": t_apply, "grad": t_grad, "proj": t_proj}, desc


def cpu_baseline(d, block_ptr, iters_per_step: float, sample_cols: int = 4, sample_blocks: int = 2):
    t0 = time.time()
    H, build_s = oracle_prepare(d)
    per_step, parts, desc = oracle_step_sample(d, H, block_ptr, iters_per_step, sample_cols, sample_blocks)
    return {"value": 1.0 / per_step, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
            "seconds_per_step_extrapolated": per_step, "oracle_build_s": build_s, "parts_s": parts,
            "measured_s": time.time() - t0}


def run_reference(args, rank):
    """--impl reference: the oracle (FP64, numpy/scipy on host cores) on a bounded sample of
    each outer iteration of the same workload."""
    if rank != 0:
        return
    d = make_inputs(args.scale)
    bp = synth_blocks(d)
    H, _ = oracle_prepare(d)
    vals, wall = [], []
    desc = ""
    for _ in range(max(1, args.warmup + args.steps)):
        t0 = time.time()
        per_step, _, desc = oracle_step_sample(d, H, bp, REF_ITERS_PER_STEP, sample_cols=2, sample_blocks=1)
        wall.append(time.time() - t0)
        vals.append(1.0 / per_step)
    timed = slice(args.warmup, None) if len(vals) > args.warmup else slice(None)
    v = float(np.mean(vals[timed]))
    sample_ms = 1000.0 * float(np.mean(wall[timed]))
    # value: the sampled step scaled to a whole outer iteration (about 1,800-2,300 s of
    # one core each); ms_per_step: the wall time actually spent per timed (sampled) step
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sample_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(config_dict(d, bp), parallelism="single",
                           cuda_graph="one captured graph per outer iteration"),
            "extrapolated": {"ms_per_full_step": 1000.0 / v, "measured_ms_per_sampled_step": sample_ms,
                             "note": "value = 1 / (sampled step time scaled to a full outer iteration)"},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": desc, "value": v},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def synth_blocks(d):
    return np.asarray(d["block_ptr"], dtype=np.int64)


def config_dict(d, bp, panels="bf16"):
    wl = d["wl"]
    return {"workload": WORKLOAD, "n": d["n"], "m": d["m"], "nnz": int(d["edge_ptr"][-1]), "c": d["c"],
            "lam": wl.lam, "mu": wl.mu, "eta": d.get("eta", wl.eta), "outer_loop": LOOP, "tol_relres": TOL,
            "size_law": synth.describe_sizes(wl), "route": "block rSVD preconditioned CG (BR)",
            "blocks": int(len(bp) - 1), "block_sizes": "U{1024..8192}", "k": K_RANK, "p": P_OVER, "q": Q_ITERS,
            "panel_dtype": ("bf16 search directions, fp32 products, residual and iterate" if panels == "bf16"
                            else "fp32") + " (fp64-accurate refinement)",
            "block_products": "auto by block fill: fp32 from the incidence lists, or bf16 dense blocks on tcgen05",
            "precond_apply": "tcgen05 tf32, operands split hi+lo (3 products), fp32 accumulate",
            "l2_flush": "inputs larger than L2 (>= 2 GB panels)"}


def run_schur(sizes):
    """The nested 2 x 2 Schur-complement inverse (Eqs. 12-14) at the paper's scale: a
    hypergraph of n vertices and 1.5 n hyperedges of U{2..20} members, r_min = k = 50,
    p = 10, q = 2; the dense products on tcgen05 (3xTF32) and on FP64 CUDA cores.  One
    JSON line per size."""
    import torch

    from paper_1908_08281_gb300 import build as _build
    from paper_1908_08281_gb300 import hgl
    _build.build()
    hgl.lib()
    wl = synth.WORKLOADS["small_fp64"]
    for n in sizes:
        d = synth.make_hypergraph(wl, 3, n=n, m=int(1.5 * n), c=1)
        g = hgl.build_incidence(d["n"], d["m"], d["edge_ptr"], d["members"])
        w = torch.full((d["m"],), 1.0 / d["m"], dtype=torch.float64, device="cuda")
        line = {"measurement": "nested Schur-complement inverse", "n": n, "m": d["m"], "r_min": 50, "k": 50,
                "p": 10, "q": 2}
        for dt, name in ((hgl.HGL_FP32, "tcgen05_3xtf32"), (hgl.HGL_FP64, "fp64_cuda_cores")):
            hgl.schur_inverse(g, w, 0.5, 0, n, 50, 50, 10, 2, 1, dt)
            torch.cuda.synchronize()
            hgl.profile_enable(True)
            t0 = time.perf_counter()
            hgl.schur_inverse(g, w, 0.5, 0, n, 50, 50, 10, 2, 1, dt)
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            ms, cnt = hgl.profile_read(hgl.PROF_SCHUR_GEMM)
            gm, gc = hgl.profile_read(hgl.PROF_GEMM)
            hgl.profile_enable(False)
            line[name] = {"seconds": t, "dense_products_ms": ms, "dense_product_launches": cnt,
                          "useful_TFLOPs": 2.67 * 2.0 * float(n) ** 3 / (ms / 1e3) / 1e12,
                          "algorithm1_products_ms": gm}
        print(json.dumps(line), flush=True)
        g.close()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.schur:
        run_schur([int(x) for x in args.schur.split(",")])
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
    bp = synth_blocks(d)
    g = hgl.build_incidence(n, m, d["edge_ptr"], d["members"])
    Yh = torch.from_numpy(d["Y"])
    Y = hgl.padded_panel(n, c, torch.float64, dev)
    Y.copy_(Yh)
    w0 = torch.tensor(d["w0"], device=dev)
    w = w0.clone()
    F = hgl.padded_panel(n, c, torch.float64, dev)
    stream = torch.cuda.current_stream()
    tuned = None
    if not args.no_tune:
        # pick the column chunks of the gather passes on this graph (untimed setup)
        t0 = time.time()
        op32, pair32, grid32 = hgl.tune_operator(g, w0, c, hgl.HGL_FP32)
        op16, _, grid16 = hgl.tune_operator(g, w0, c, hgl.HGL_BF16)
        op64, _, grid64 = hgl.tune_operator(g, w0, c, hgl.HGL_FP64)
        policy = ("one wave", "eight per SM")
        broute, b_dense, b_sparse = hgl.tune_block_rsvd(g, w0, bp, K_RANK, P_OVER, Q_ITERS)
        tuned = {"operator_chunk_fp32": op32, "operator_chunk_bf16": op16, "residual_chunk": pair32,
                 "operator_chunk_fp64": op64,
                 "grid_fp32": policy[grid32], "grid_bf16": policy[grid16], "grid_fp64": policy[grid64],
                 "block_products": {"route": "sparse" if broute == hgl.HGL_BLOCKS_SPARSE else "dense (tcgen05)",
                                    "ms_per_build_dense": b_dense, "ms_per_build_sparse": b_sparse},
                 "tune_s": time.time() - t0}

    def reset():
        w.copy_(w0)
        F.zero_()

    eta = wl.eta if args.eta is None else args.eta
    d["eta"] = eta

    graph_flag = 0 if args.no_graph else hgl.HGL_STEP_GRAPH
    # inner-CG search directions of the headline loop (the other type is an arm)
    head_dt = hgl.HGL_BF16 if args.panels == "bf16" else hgl.HGL_FP32
    other_dt = hgl.HGL_FP32 if head_dt == hgl.HGL_BF16 else hgl.HGL_BF16
    pname = {hgl.HGL_FP32: "fp32", hgl.HGL_BF16: "bf16"}

    def step(Fp, wp, i, dtype=head_dt, route=hgl.HGL_ROUTE_BR, reset=True):
        # one outer iteration; with the graph flag the library replays one captured CUDA
        # graph per call (the first call with these buffers runs eagerly, the second captures)
        if reset and i % LOOP == 0:
            wp.copy_(w0)
            Fp.zero_()
        return hgl.adaptive_step(g, wp, Y, Fp, lam=wl.lam, mu=wl.mu, eta=eta, tol=TOL, dtype=dtype, route=route,
                                 block_ptr=bp, k=K_RANK, p=P_OVER, q=Q_ITERS, seed=SEED + (i % LOOP),
                                 flags=graph_flag)

    # warm-up: W outer iterations of a loop, then the timed steps start a fresh loop
    for i in range(args.warmup):
        step(F, w, i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    hgl.profile_enable(True)
    l0 = hgl.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    stats = []
    for i in range(args.steps):
        stats.append(step(F, w, i))
    e1.record(stream)
    torch.cuda.synchronize()
    launches = hgl.launch_count() - l0
    prof = {f: hgl.profile_read(f) for f in range(len(hgl.PROF_NAMES))}
    hgl.profile_enable(False)
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    ms_per_step = ms / args.steps
    value = world * args.steps / (ms / 1000.0)
    iters = [s.solve.iters for s in stats]
    relres_max = max(s.solve.relres_max for s in stats)
    # ||w_new - w_old|| / ||w_old||, with ||w|| ~ 1/sqrt(m) near the uniform start
    dw_rel = [s.dw_norm * float(np.sqrt(m)) for s in stats]

    # the timed loop's final state (the accuracy step and the end-to-end run go on from it)
    F_loop, w_loop = F.clone(), w.clone()

    # accuracy (untimed): one more mixed-precision step, then the same system solved by
    # FP64 CG to 1e-12 at that step's w; per-column relative error of the mixed F
    w_in = w.clone()
    st_acc = step(F, w, args.steps, reset=False)
    Fref = hgl.padded_panel(n, c, torch.float64, dev)
    Fref.copy_(F)
    _, _, _, st_ref = hgl.cg_solve(g, w_in, wl.lam, Y, F=Fref, tol=1e-12, max_iter=400, warm_start=True)
    col_err = ((F - Fref).norm(dim=0) / Fref.norm(dim=0).clamp_min(1e-300)).max().item()
    accuracy = {"max_col_rel_err_F_vs_fp64": col_err, "step_relres_max": st_acc.solve.relres_max,
                "fp64_reference_relres": st_ref.relres_max, "bound_from_tol": (1 + wl.lam) / wl.lam * TOL}
    del Fref, w_in

    # roofline of the dominant kernel family (event-timed inside the timed region)
    hbm_peak, bf16_peak, peak_kind = measured_peaks()
    kernel_names = {hgl.PROF_OPERATOR: "operator apply (k_edge_pass + k_vertex_pass), "
                                        + ("BF16 search directions into FP32 products" if head_dt == hgl.HGL_BF16
                                           else "FP32 panels") + ", c=512",
                    hgl.PROF_RESIDUAL: "pair-arithmetic residual (df::k_edge + df::k_vertex), c=512",
                    hgl.PROF_OPRESID: "FP32 residual estimate (k_edge_pass + k_vertex_pass, residual epilogue)",
                    hgl.PROF_GEMM: "grouped block GEMM on tcgen05 (umma::k_block_gemm), BF16 in / FP32 out",
                    hgl.PROF_GRADIENT: "weight gradient (k_grad_edge + k_grad_vertex + k_grad_final), FP32"}
    lpad = ((K_RANK + P_OVER + 15) // 16) * 16
    op_chunk = (tuned or {}).get("operator_chunk_" + pname[head_dt]) or 128
    op32_chunk = (tuned or {}).get("operator_chunk_fp32") or 128
    pair_chunk = (tuned or {}).get("residual_chunk") or 128
    elt_x = 2 if head_dt == hgl.HGL_BF16 else 4
    per_launch_bytes = {hgl.PROF_OPERATOR: bytes_operator(n, m, nnz, c, elt_x, -(-c // op_chunk), elt_z=4),
                        hgl.PROF_RESIDUAL: bytes_residual(n, m, nnz, c, -(-c // pair_chunk)),
                        hgl.PROF_OPRESID: bytes_opresid(n, m, nnz, c, -(-c // op32_chunk)),
                        hgl.PROF_GEMM: bytes_gemm(bp, lpad),
                        hgl.PROF_GRADIENT: bytes_gradient(n, m, nnz, c)}
    # executed calls of the solver's families: a captured step launches a fixed sequence
    # whose calls beyond convergence return at once (recorded, but not work); one operator
    # apply per CG iteration, one residual per sweep plus the first, one preconditioner
    # apply per iteration plus one per sweep; at loose tolerances the first residual of a
    # solve is an FP32 estimate by one operator pass (its own family), not a pair residual
    refinements = [s.solve.refinements for s in stats]
    first_estimated = prof[hgl.PROF_OPRESID][1] > 0
    executed = {hgl.PROF_OPERATOR: int(sum(iters)),
                hgl.PROF_RESIDUAL: int(sum(2 + r - first_estimated for r in refinements)),
                hgl.PROF_PRECOND: int(sum(it + 1 + r for it, r in zip(iters, refinements)))}
    families = {}
    for f, (fms, cnt) in prof.items():
        if cnt > 0:
            calls = min(executed.get(f, cnt), cnt)
            avg = fms / calls
            ent = {"ms_total": fms, "launches": cnt, "executed": calls, "ms_per_launch": avg,
                   "share_of_step_time": fms / ms}
            if f in per_launch_bytes:
                ent["achieved_GBps"] = per_launch_bytes[f] / (avg / 1000.0) / 1e9
            families[hgl.PROF_NAMES[f]] = ent
    dom = max(per_launch_bytes, key=lambda f: prof[f][0])
    dms, dcnt = prof[dom]
    dcnt = min(executed.get(dom, dcnt), dcnt)
    davg = dms / max(dcnt, 1)
    achieved = per_launch_bytes[dom] / (davg / 1000.0) / 1e9
    fam_key = {hgl.PROF_OPERATOR: ("operator", pname[head_dt], op_chunk),
               hgl.PROF_RESIDUAL: ("residual", "fp32", pair_chunk)}.get(dom)
    traffic = NCU_TRAFFIC_PER_LAUNCH.get(fam_key) if (args.scale == 1.0 and fam_key) else None
    roofline = {"kernel": kernel_names[dom], "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_kind": peak_kind, "traffic": traffic,
                "algorithmic_bytes_per_launch": per_launch_bytes[dom], "ms_per_launch": davg, "launches": dcnt}
    if prof[hgl.PROF_GEMM][1] > 0:
        gavg = prof[hgl.PROF_GEMM][0] / prof[hgl.PROF_GEMM][1]
        roofline["gemm"] = {"kernel": kernel_names[hgl.PROF_GEMM], "bound": "hbm",
                            "achieved_GBps": per_launch_bytes[hgl.PROF_GEMM] / (gavg / 1000.0) / 1e9,
                            "frac_hbm": per_launch_bytes[hgl.PROF_GEMM] / (gavg / 1000.0) / 1e9 / hbm_peak,
                            "tensor_TFLOPs": flops_gemm(bp, lpad) / (gavg / 1000.0) / 1e12,
                            "frac_bf16_peak": flops_gemm(bp, lpad) / (gavg / 1000.0) / 1e12 / bf16_peak,
                            "ms_per_launch": gavg}

    # end to end through the public API: every step copies Y (pinned host) in and reads
    # w and the step statistics back; a loop's first step also copies w0 in
    e2e = None
    if not args.no_e2e:
        Yp = torch.empty((n, Y.stride(0)), dtype=torch.float64).pin_memory()
        Yp[:, :c].copy_(Yh)
        w_host = w0.cpu().pin_memory()
        w_out = torch.empty_like(w_host).pin_memory()
        Ybuf = Y.as_strided((n, Y.stride(0)), (Y.stride(0), 1))
        e2e_steps = args.steps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            Ybuf.copy_(Yp, non_blocking=True)
            if i % LOOP == 0:
                w.copy_(w_host, non_blocking=True)
                F.zero_()
            step(F, w, i, reset=False)
            w_out.copy_(w, non_blocking=True)
            torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        e2e = {"value": 1.0 / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(Yp.numel() * 8) + int(8 * m / LOOP),
               "d2h_bytes_per_step": int(w_out.numel() * 8 + 48), "steps": e2e_steps}

    loops_compared = args.steps % LOOP == 0  # the timed loops end on a whole 20-iteration loop

    def timed_loop(dtype, route):
        """The same 20-iteration loop with another solver, timed like the headline (a
        first eager call and the capture before the timed steps); returns its timing,
        statistics and final (F, w)."""
        Fx = hgl.padded_panel(n, c, torch.float64, dev)
        wx = w0.clone()
        for i in range(2):  # eager call, then the capture (graph mode)
            step(Fx, wx, 0, dtype, route)
        torch.cuda.synchronize()
        b0 = torch.cuda.Event(enable_timing=True)
        b1 = torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        stx = [step(Fx, wx, i, dtype, route) for i in range(args.steps)]
        b1.record(stream)
        torch.cuda.synchronize()
        xms = b0.elapsed_time(b1) / args.steps
        return xms, stx, Fx, wx

    def loop_diff(Fa, wa, Fb, wb):
        dF = (Fa - Fb).norm(dim=0) / Fb.norm(dim=0).clamp_min(1e-300)
        return {"F_max_col_rel": float(dF.max().item()),
                "w_rel": float((torch.linalg.norm(wa - wb) / torch.linalg.norm(wb)).item())}

    fp64 = mixed_cg = mixed_other = fp64_bcg = loop_acc = None
    plabel = {hgl.HGL_FP32: "FP32 panels", hgl.HGL_BF16: "BF16 search directions (FP32 products, residual and iterate)"}
    if not args.no_fp64:
        f64_ms, st64, F64, w64 = timed_loop(hgl.HGL_FP64, hgl.HGL_ROUTE_CG)
        fp64 = {"ms_per_step": f64_ms, "value": 1000.0 / f64_ms, "unit": UNIT,
                "route": "plain CG per column (Eqs. 16-20), FP64, no preconditioner",
                "cg_iters_per_step": float(np.mean([s.solve.iters for s in st64])),
                "relres_max": max(s.solve.relres_max for s in st64),
                "speedup_of_mixed": f64_ms / ms_per_step}
        cg_ms, stc, Fc, wc = timed_loop(head_dt, hgl.HGL_ROUTE_CG)
        mixed_cg = {"ms_per_step": cg_ms, "value": 1000.0 / cg_ms, "unit": UNIT,
                    "route": f"CG per column, {plabel[head_dt]} with FP64-accurate refinement, no preconditioner",
                    "cg_iters_per_step": float(np.mean([s.solve.iters for s in stc])),
                    "relres_max": max(s.solve.relres_max for s in stc),
                    "speedup_over_fp64": f64_ms / cg_ms}
        # O'Leary's block CG (FP64, groups of 32 columns, eager launches: its host
        # synchronisations per iteration keep it out of a captured graph), timed on the
        # first BCG_STEPS outer iterations of the same loop
        Fk = hgl.padded_panel(n, c, torch.float64, dev)
        Fk.zero_()
        wk = w0.clone()
        torch.cuda.synchronize()
        k0 = torch.cuda.Event(enable_timing=True)
        k1 = torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        stk = [hgl.adaptive_step(g, wk, Y, Fk, lam=wl.lam, mu=wl.mu, eta=eta, tol=TOL, dtype=hgl.HGL_FP64,
                                 route=hgl.HGL_ROUTE_BCG, k=BCG_S) for _ in range(BCG_STEPS)]
        k1.record(stream)
        torch.cuda.synchronize()
        bcg_ms = k0.elapsed_time(k1) / BCG_STEPS
        f64_cg_first = float(np.mean([s.solve.iters for s in st64[:BCG_STEPS]]))
        fp64_bcg = {"ms_per_step": bcg_ms, "value": 1000.0 / bcg_ms, "unit": UNIT,
                    "route": f"block CG (O'Leary), FP64, groups of {BCG_S} columns, eager launches",
                    "steps_timed": BCG_STEPS, "iters_per_step": float(np.mean([s.solve.iters for s in stk])),
                    "fp64_cg_iters_same_steps": f64_cg_first,
                    "relres_max": max(s.solve.relres_max for s in stk)}
        del Fk, wk
        bf_ms, stb, Fb, wb = timed_loop(other_dt, hgl.HGL_ROUTE_BR)
        mixed_other = {"ms_per_step": bf_ms, "value": 1000.0 / bf_ms, "unit": UNIT,
                       "route": f"block rSVD preconditioned CG, {plabel[other_dt]} with FP64-accurate refinement",
                       "cg_iters_per_step": float(np.mean([s.solve.iters for s in stb])),
                       "refinements_per_step": float(np.mean([s.solve.refinements for s in stb])),
                       "relres_max": max(s.solve.relres_max for s in stb),
                       "speedup_over_fp64": f64_ms / bf_ms}
        if loops_compared:
            # the loop's exact trajectory to within 3e-10 per step: FP64 CG to 1e-10,
            # eager launches, the same 20 outer iterations from w0 (untimed)
            Ft = hgl.padded_panel(n, c, torch.float64, dev)
            wt = w0.clone()
            Ft.zero_()
            for i in range(LOOP):
                hgl.adaptive_step(g, wt, Y, Ft, lam=wl.lam, mu=wl.mu, eta=eta, tol=1e-10, max_iter=400,
                                  dtype=hgl.HGL_FP64, route=hgl.HGL_ROUTE_CG, flags=0)
            torch.cuda.synchronize()
            loop_acc = {"reference": "FP64 CG to relres 1e-10, same 20 outer iterations from w0",
                        "mixed_br": loop_diff(F_loop, w_loop, Ft, wt), "fp64_cg": loop_diff(F64, w64, Ft, wt),
                        "mixed_cg": loop_diff(Fc, wc, Ft, wt),
                        f"mixed_{pname[other_dt]}_br": loop_diff(Fb, wb, Ft, wt),
                        "mixed_br_vs_fp64_cg": loop_diff(F_loop, w_loop, F64, w64),
                        "bound_F_from_tol": (1 + wl.lam) / wl.lam * TOL}
            del Ft, wt
        del F64, w64, Fc, wc, Fb, wb
    del F_loop, w_loop

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(d, bp, float(np.mean(iters)))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": ("bf16+f32+f64" if head_dt == hgl.HGL_BF16 else "f32+f64"),
            "data": "synthetic",
            "config": dict(config_dict(d, bp, pname[head_dt]), parallelism="replicas" if world > 1 else "single",
                           cuda_graph="one captured graph per outer iteration" if graph_flag else "eager launches"),
            "solve": {"cg_iters_per_step": iters, "relres_max": relres_max,
                      "dw_rel_to_uniform_w": dw_rel},
            "tuned_chunks": tuned,
            "accuracy": accuracy,
            "roofline": roofline,
            "kernel_families": families,
            "block_product_route": ("sparse (incidence lists)" if prof[hgl.PROF_BLOCKSPMM][1] > 0
                                    else "dense (tcgen05 GEMM)"),
            "e2e": e2e,
            "fp64_cg": fp64,
            "mixed_cg_route": mixed_cg,
            f"mixed_{pname[other_dt]}_route": mixed_other,
            "fp64_block_cg": fp64_bcg,
            "loop_accuracy": loop_acc,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": int(launches),
            "gpu_launches_per_step": launches / args.steps,
            "gen_s": d["gen_s"],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
