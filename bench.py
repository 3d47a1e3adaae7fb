#!/usr/bin/env python3
"""Benchmark: FP64 Jacobi-PCG on the 32x32x32 deformed box (32768 elements, nx=10).

One step is one ``nek_cg_solve`` call of 100 Jacobi-PCG iterations (tol = 0, a
fixed iteration count), i.e. 100 passes of the whole solve path: AX, dssum,
mask, the weighted dot products and the vector updates.  ``value`` is local
grid points x iterations per second (GDOF/s) over all ranks, with the
FP64-accurate float-float operator.  The AX kernel is timed inside the same
region with CUDA events on the solve's stream; it gives the roofline entry.
``e2e`` times the same steps through ``nek_cg_solve_host`` (f and x in pinned
host memory, both copies inside the call).

The default run also carries the rest of the metric (rank 0, after the timed
region): the same solve with the native FP64 operator, the standalone AX sweep
(nx = 8, 10, 12, 16, both FP64 operators), time to a relative residual of 1e-8
for native-FP64 and float-float Jacobi-PCG, FP64 defect correction with FP32 /
BF16 / FP16 inner solves (to 1e-8 and 1e-10), the learned-preconditioner
comparison, the batched uneven solves, and the oracle's CPU time on one and on
all host cores.  ``--extras none`` skips all of that.

Inputs are synthetic (seeded deformed-box mesh, f ~ U[-1,1] per global node);
the geometric factors alone are 1.57 GB, far larger than the 129 MB L2, so no
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--iters 100] [--nx 10]
                  [--impl reference] [--extras native,sweep,solve,mixed,learned,batch,lvec | none]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "AX GDOF/s & % HBM peak; CG s-to-1e-8 residual, FP64 vs mixed/learned"
UNIT = "GDOF/s"
FP64_PEAK_TFLOPS = 1.2586  # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--iters", type=int, default=100, help="PCG iterations per step")
    ap.add_argument("--nx", type=int, default=10)
    ap.add_argument("--elems", type=int, default=32, help="elements per box edge")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--extras", default="native,sweep,solve,mixed,learned,batch",
                    help="comma list of blocks after the timed region (native, sweep, solve, mixed, learned, "
                         "batch, lvec), 'all' or 'none'")
    ap.add_argument("--sweep-elems", type=int, default=32, help="elements per side of the AX sweep's box")
    ap.add_argument("--sweep-nx", type=int, nargs="+", default=[8, 10, 12, 16], help="nx values of the AX sweep")
    ap.add_argument("--sweep", action="store_true", help="add the standalone AX sweep to --extras")
    ap.add_argument("--solve", action="store_true", help="add the solves to 1e-8 to --extras")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-baseline-only", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-threads", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--cpu-seconds", type=float, default=None,
                    help="bound on the oracle's CPU time per sample (default: about 10-15 s for cpu_baseline, "
                         "120 s spread over the steps of --impl reference)")
    ap.add_argument("--mixed", action="store_true", help="add defect correction (FP32/BF16/FP16) to --extras")
    ap.add_argument("--mixed-precisions", default="f32,bf16,f16",
                    help="comma list of the defect-correction block's inner precisions (f32, bf16, f16)")
    ap.add_argument("--batch", type=int, default=256,
                    help="problems of the batched block (nelt log-uniform in [8,4096])")
    ap.add_argument("--learned", action="store_true", help="add the learned-preconditioner block to --extras")
    ap.add_argument("--learned-meshes", type=int, default=200)
    ap.add_argument("--net-elems", type=int, default=13824,
                    help="elements of the --extras net block (network inference rates, random weights)")
    ap.add_argument("--learned-epochs", type=int, default=30)
    ap.add_argument("--lvec", action="store_true", help="add the unique-node (L-vector) block to --extras")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="skip the elements-per-CTA tuning (nek_tune_ax) before timing")
    ap.add_argument("--epb", type=int, default=0,
                    help="fix the AX elements per CTA (1, 2 or 4; nek_set_ax_epb) instead of tuning")
    ap.add_argument("--ax", default="ff", choices=["fp64", "ff", "oz"],
                    help="AX operator inside the solve: native FP64, FP64-accurate float-float, or FP64-accurate "
                         "with the contractions on the tensor cores (BF16 digit slices; even nx up to 10)")
    args = ap.parse_args()
    names = {"native", "sweep", "solve", "mixed", "learned", "batch", "lvec", "net"}
    ex = args.extras.strip().lower()
    sel = set(names) if ex == "all" else set() if ex in ("none", "") else {s.strip() for s in ex.split(",")}
    if sel - names:
        ap.error("unknown --extras: %s" % ",".join(sorted(sel - names)))
    for flag in ("sweep", "solve", "mixed", "learned", "lvec"):
        if getattr(args, flag):
            sel.add(flag)
    args.extra_set = sel
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        import tempfile

        self.proc = None
        self.gpu = gpu_index
        # raw samples go to a private temporary file; their summary goes into the JSON line
        self.path = os.path.join(tempfile.mkdtemp(prefix="nek_clocks_"), "clocks_%d.csv" % gpu_index)

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as fh:
            return summarize_clocks(fh)


def summarize_clocks(lines):
    """Median SM clock, the maximum clock and the throttle reasons seen, from lines of ClockSampler.FIELDS
    (csv, no header, no units); lines that do not parse are skipped; None without a sample."""
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
        for n, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers
AX_SOURCES = {"fp64": ("nek_ax.cu", "ax_fp64_traffic.json"), "ff": ("nek_ax_ff_kernels.cuh", "ax_ff_traffic.json"),
              "oz": ("nek_ax_oz.cu", "ax_oz_traffic.json")}


def kernel_source_sha(which="fp64"):
    with open(os.path.join(ROOT, "paper_2011_04981_gb300", "csrc", AX_SOURCES[which][0]), "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def traffic_from_profile(nx, nelt, which="fp64"):
    """DRAM bytes per AX launch from the committed ncu summary, if it matches this kernel source."""
    try:
        with open(os.path.join(ROOT, "profiles", AX_SOURCES[which][1])) as fh:
            t = json.load(fh)
        if t.get("source_sha") != kernel_source_sha(which) or int(t["nx"]) != nx:
            return None
        return float(t["dram_bytes_per_element"]) * nelt
    except Exception:
        return None


def _oracle_pcg_samples(nx, budget_s, samples=1, lib_path=None, max_iters=200, elems=12):
    """Time the oracle (as it stands) on a bounded sample of the workload: Jacobi-PCG iterations on an
    elems^3-element box of the same family (same nx, perturbation and seed recipe), as many per sample as
    fit in budget_s (at most max_iters).  Returns the mesh's point count and one (iterations, seconds)
    pair per sample."""
    import contextlib

    from oracle import ref
    from paper_2011_04981_gb300 import inputs

    e = elems
    mesh = inputs.box_mesh(e, e, e, nx, perturb=0.1, seed=1)
    P = ref.Problem(mesh)
    f = inputs.random_global_field(mesh, seed=2)
    ctx = ref.using_library(lib_path) if lib_path else contextlib.nullcontext()
    out = []
    with ctx:
        t0 = time.perf_counter()
        ref.pcg(P.D, P.G, P.offsets, P.idx, mesh.mask, P.minv, f, tol=0.0, max_iter=2)
        per_it = (time.perf_counter() - t0) / 2
        iters = max(2, min(max_iters, int(budget_s / max(per_it, 1e-6))))
        for _ in range(samples):
            t0 = time.perf_counter()
            ref.pcg(P.D, P.G, P.offsets, P.idx, mesh.mask, P.minv, f, tol=0.0, max_iter=iters)
            out.append((iters, time.perf_counter() - t0))
    return mesh.npts, out


def cpu_baseline(nx, iters_budget_s=15.0, threads=1, samples=1, warmup=0, elems=12, max_iters=None):
    """The oracle's rate on `threads` host threads: 1 = the default build in this process; more = its
    -fopenmp build (same operations, independent loops split over threads) in a child process with
    OMP_NUM_THREADS set, so that its OpenMP runtime is not the one PyTorch loaded.  `warmup` untimed
    samples come first; the result's 'per_sample' lists (iterations, seconds) of each timed sample."""
    if threads <= 1:
        npts, smp = _oracle_pcg_samples(nx, iters_budget_s, warmup + samples, elems=elems,
                                        max_iters=max_iters or 200)
        smp = smp[warmup:]
        build = "single-threaded C oracle"
    else:
        env = dict(os.environ, OMP_NUM_THREADS=str(threads), OMP_PROC_BIND="false")
        cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-baseline-only", "--cpu-threads", str(threads),
               "--nx", str(nx), "--cpu-seconds", str(iters_budget_s), "--steps", str(samples), "--warmup",
               str(warmup), "--elems", str(elems), "--iters", str(max_iters or 4000)]
        r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=60 + 4 * iters_budget_s * samples)
        lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
        if r.returncode != 0 or not lines:
            return {"unavailable": "OpenMP oracle run failed: %s" % (r.stderr.strip().splitlines() or ["?"])[-1]}
        d = json.loads(lines[-1])
        if "unavailable" in d:
            return d
        npts, smp = d["npts"], [tuple(s) for s in d["samples"]]
        build = "C oracle built with -fopenmp, %d threads" % threads
    its = sum(i for i, _ in smp)
    secs = sum(s for _, s in smp)
    return {"value": npts * its / secs / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d x %d Jacobi-PCG iterations on a %dx%dx%d-element deformed box, nx=%d (%d points), %s, "
                      "%.1f s" % (len(smp), smp[0][0], elems, elems, elems, nx, npts, build, secs),
            "seconds": secs, "per_sample": smp, "host": host_cpu()}


def cpu_baseline_child(args):
    """--cpu-baseline-only: run the -fopenmp oracle sample(s) and print one JSON line."""
    from oracle import ref

    so = ref.openmp_library()
    if so is None:
        print(json.dumps({"unavailable": "no OpenMP-capable C compiler on this host"}))
        return 0
    npts, smp = _oracle_pcg_samples(args.nx, args.cpu_seconds or 15.0, max(1, args.steps + args.warmup), so,
                                    max_iters=args.iters, elems=args.elems)
    print(json.dumps({"npts": npts, "samples": smp[args.warmup:], "threads": args.cpu_threads}))
    return 0


def host_cpu():
    """Logical CPUs and the CPU model of this host (the oracle uses one of them)."""
    model = platform.machine()
    try:
        with open("/proc/cpuinfo") as fh:
            info = fh.read().splitlines()
        names = [ln.split(":", 1)[1].strip() for ln in info if ln.lower().startswith("model name")]
        parts = [ln.split(":", 1)[1].strip() for ln in info if ln.startswith("CPU part")]
        impl = [ln.split(":", 1)[1].strip() for ln in info if ln.startswith("CPU implementer")]
        if names:
            model = names[0]
        elif parts:
            model = "%s implementer %s part %s" % (platform.machine(), impl[0] if impl else "?", parts[0])
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu": model}


def max_over_ranks(dist, values, device):
    """Element-wise maximum of a list of floats over all ranks (every rank gets it)."""
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    """The oracle on the host's cores (all of them, through its -fopenmp build; one if that build is not
    available) on the benchmark's own workload: Jacobi-PCG on the same elems^3 box at the same nx, each
    step as many iterations (up to --iters) as fit in its share of about two minutes."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    budget = args.cpu_seconds if args.cpu_seconds else max(3.0, 120.0 / max(1, args.steps + args.warmup))
    threads = os.cpu_count() or 1
    kw = dict(samples=args.steps, warmup=args.warmup, elems=args.elems, max_iters=args.iters)
    cb = cpu_baseline(args.nx, budget, threads=threads, **kw) if threads > 1 else None
    if cb is None or "unavailable" in cb:
        threads = 1
        cb = cpu_baseline(args.nx, budget, threads=1, **kw)
    steps = cb["per_sample"]
    e = args.elems
    npts = e ** 3 * args.nx ** 3
    tot_s = sum(s for _, s in steps)
    value = npts * sum(i for i, _ in steps) / tot_s / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_s / len(steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "Jacobi-PCG, %d PCG iterations per step (AX+dssum+mask+dots+updates), "
                                   "%dx%dx%d deformed box (perturbation 0.1 h), nx=%d, FP64, the C oracle on %d host "
                                   "threads" % (steps[0][0], e, e, e, args.nx, threads),
                       "elements": e ** 3, "nx": args.nx, "points": npts, "iters_per_step": steps[0][0],
                       "parallelism": "single"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": cb["sample"],
                             "host": cb.get("host")},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ native arm
def ax_sweep(torch, nxs=(8, 10, 12, 16), reps=20, tune=False, elems=32):
    """Standalone AX at each nx on an elems^3-element box (32^3 by default): median over `reps` launches, each
    timed with its own CUDA events (inputs far above L2 at 32^3, so no flush is needed)."""
    from paper_2011_04981_gb300 import inputs, nekax, perfmodel
    from paper_2011_04981_gb300.problem import DeviceProblem

    out = {}
    hbm, _ = peaks()
    for nx in nxs:
        mesh = inputs.box_mesh(elems, elems, elems, nx, perturb=0.1, seed=1)
        P = DeviceProblem(mesh, "cuda", build_minv=False)
        P.prepare_ff()
        ops = [("fp64", P.ax), ("ff", P.ax_ff)]
        if nx % 2 == 0 and nx <= 10:
            P.prepare_oz()
            ops.append(("oz", P.ax_oz))
        u = torch.rand((mesh.nelt, nx ** 3), dtype=torch.float64, device="cuda") * 2 - 1
        w = torch.empty_like(u)
        s = torch.cuda.current_stream()
        res = {}
        for name, fn in ops:
            epb = None
            if tune and name != "oz":
                impl = nekax.AX_FF if name == "ff" else nekax.AX_FP64
                epb, _ = nekax.tune_ax(impl, mesh.nelt, nx, P.D, P.Gff if name == "ff" else P.G, u, w)
            for _ in range(3):
                fn(u, w)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(reps)]
            torch.cuda.synchronize()
            for a, b in evs:
                a.record(s)
                fn(u, w)
                b.record(s)
            evs[-1][1].synchronize()
            t = statistics.median(a.elapsed_time(b) for a, b in evs) / 1e3
            g = mesh.npts / t / 1e9
            res[name] = {"gdofs": g, "ms": t * 1e3, "gflops": g * perfmodel.ax_flops_per_point(nx),
                         "hbm_frac": g * 64 / hbm,
                         "fp64_frac": g * perfmodel.ax_flops_per_point(nx) / 1e3 / FP64_PEAK_TFLOPS,
                         "epb": "2 persistent CTAs per SM" if name == "oz" else epb if epb is not None else
                         nekax.get_ax_epb(nekax.AX_FF if name == "ff" else nekax.AX_FP64, nx)}
        out[str(nx)] = res
        del P, u, w
        torch.cuda.empty_cache()
    return out


def lvec_block(torch, P, iters, reps=3):
    """Unique-node (L-vector) Jacobi-PCG against the E-vector solve on the bench mesh, same operator
    (nek_ax_ff): fixed-iteration rate in E-points x iterations / s, and time to 1e-8."""
    import numpy as np

    from paper_2011_04981_gb300 import nekax

    lv, minvL, _ = P.lvec()
    gL = torch.from_numpy(np.random.default_rng(2).uniform(-1.0, 1.0, lv.size)).to("cuda")
    fE = torch.empty(P.npts, dtype=torch.float64, device="cuda")
    lv.scatter(gL, fE)
    xL = torch.empty_like(gL)
    xE = torch.empty_like(fE)
    s = torch.cuda.current_stream()
    out = {"unique_nodes": lv.size, "element_points": P.npts, "unique_fraction": lv.size / P.npts}
    for name, run in (("evec", lambda it, tol: P.cg(fE, xE, tol=tol, max_iter=it, ax_impl=nekax.AX_FF,
                                                    check_every=20 if tol > 0 else 1)),
                      ("lvec", lambda it, tol: P.cg_lvec(gL, xL, tol=tol, max_iter=it,
                                                         check_every=20 if tol > 0 else 1))):
        run(iters, 0.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            r = run(iters, 0.0)
        e1.record(s)
        e1.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / reps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r8 = run(20000, 1e-8)
        torch.cuda.synchronize()
        out[name] = {"gdofs_element_points": P.npts * iters / t / 1e9, "ms_per_iteration": 1e3 * t / iters,
                     "to_1e-8": {"seconds": time.perf_counter() - t0, "iters": r8["iters"], "relres": r8["relres"],
                                 "status": nekax.status_string(r8["status"])}}
    xLE = torch.empty_like(fE)
    lv.scatter(xL, xLE)
    out["max_rel_diff_x"] = float((xLE - xE).abs().max() / xE.abs().max())
    out["speedup"] = out["evec"]["ms_per_iteration"] / out["lvec"]["ms_per_iteration"]
    return out


def mixed_block(torch, P, f, x, precisions=("f32", "bf16", "f16")):
    """FP64 defect correction with reduced-precision inner PCG on the bench mesh."""
    from paper_2011_04981_gb300 import nekax

    out = {}
    nx, nelt = P.nx, P.nelt
    Gff = P.prepare_ff()
    u = torch.rand((nelt, nx ** 3), dtype=torch.float64, device="cuda") * 2 - 1
    w64 = torch.empty_like(u)
    P.ax_ff(u, w64)
    u32 = u.float()
    w32 = torch.empty_like(u32)
    hbm, _ = peaks()
    for name, prec, dt in (("f32", nekax.PREC_F32, torch.float32), ("bf16", nekax.PREC_BF16, torch.float16),
                           ("f16", nekax.PREC_F16, torch.float16)):
        if name not in precisions:
            continue
        Glp = torch.empty((nelt, nx ** 3, 6), dtype=dt, device="cuda")
        gsc = torch.empty(nelt, dtype=torch.float32, device="cuda")
        nekax.geom_lowp(nelt, nx, prec, P.G, Glp, gsc)
        nekax.ax_lowp(nelt, nx, prec, P.D, Glp, gsc, u32, w32)
        torch.cuda.synchronize()
        err = float((w32.double() - w64).abs().max() / w64.abs().max())
        # standalone AX rate
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            nekax.ax_lowp(nelt, nx, prec, P.D, Glp, gsc, u32, w32)
        e1.record()
        e1.synchronize()
        t_ax = e0.elapsed_time(e1) / 10 / 1e3
        bpp = 8 + 6 * (4 if prec == nekax.PREC_F32 else 2)
        rec = {"ax_rel_err_vs_fp64": err, "ax_gdofs": P.npts / t_ax / 1e9, "ax_bytes_per_point": bpp,
               "ax_hbm_frac": P.npts * bpp / t_ax / 1e9 / hbm}
        if prec != nekax.PREC_F32:  # the same operator with the D-contractions on the tensor cores
            w2 = torch.empty_like(w32)
            nekax.ax_lowp_tc(nelt, nx, prec, P.D, Glp, gsc, u32, w2)
            e0.record()
            for _ in range(10):
                nekax.ax_lowp_tc(nelt, nx, prec, P.D, Glp, gsc, u32, w2)
            e1.record()
            e1.synchronize()
            t_tc = e0.elapsed_time(e1) / 10 / 1e3
            rec["tensor_core_form"] = {"kernel": "mma.sync m16n8k16 (nek_ax_lowp_tc)", "ax_gdofs": P.npts / t_tc / 1e9,
                                       "ax_rel_err_vs_fp64": float((w2.double() - w64).abs().max() / w64.abs().max())}
            if nx <= 11:  # the tcgen05 form, which the solves below use as their inner operator
                nekax.ax_lowp_tc5(nelt, nx, prec, P.D, Glp, gsc, u32, w2)
                e0.record()
                for _ in range(10):
                    nekax.ax_lowp_tc5(nelt, nx, prec, P.D, Glp, gsc, u32, w2)
                e1.record()
                e1.synchronize()
                t5 = e0.elapsed_time(e1) / 10 / 1e3
                rec["tcgen05_form"] = {"kernel": "k_ax_lowp_tc5 (nek_ax_lowp_tc5), the solve's inner operator",
                                       "ax_gdofs": P.npts / t5 / 1e9, "ax_hbm_frac": P.npts * bpp / t5 / 1e9 / hbm,
                                       "ax_rel_err_vs_fp64": float((w2.double() - w64).abs().max() / w64.abs().max())}
        for tol in (1e-8, 1e-10):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = nekax.cg_solve_mixed(P.gs, nelt, nx, P.D, P.G, Gff, prec, Glp, gsc, P.mask, P.minv, f, x, tol=tol,
                                     inner_tol=1e-2, max_outer=100, max_inner=20000)
            torch.cuda.synchronize()
            rec["to_%g" % tol] = {"seconds": time.perf_counter() - t0, "outer": r["outer"], "inner": r["inner"],
                                  "relres": r["relres"], "status": nekax.status_string(r["status"])}
        out[name] = rec
        del Glp, gsc
    return out


def batch_block(torch, nprob, tol=1e-8):
    """Configuration 4: nprob uneven deformed-box problems solved together."""
    from paper_2011_04981_gb300 import inputs
    from paper_2011_04981_gb300.problem import DeviceBatch

    specs = inputs.batch_problem_specs(nprob, seed=1)
    meshes = [inputs.box_mesh(sp["ex"], sp["ey"], sp["ez"], sp["nx"], perturb=0.1, seed=sp["seed"]) for sp in specs]
    fields = [inputs.random_global_field(m, seed=sp["seed"] + 7) for m, sp in zip(meshes, specs)]
    B = DeviceBatch(meshes, fields, "cuda", ff=True)
    x = torch.empty((B.npts,), dtype=torch.float64, device="cuda")
    ws = torch.empty(B.plan.workspace_bytes(False) // 8 + 64, dtype=torch.float64, device="cuda")
    B.solve(x, tol=tol, max_iter=21, iters_per_graph=10, workspace=ws)  # warm-up (graph instantiation too)
    B.solve(x, tol=tol, max_iter=21, iters_per_graph=-1, workspace=ws)
    out = {"problems": nprob, "points": B.npts, "elements": int(sum(m.nelt for m in meshes)),
           "nx_counts": {str(n): sum(1 for m in meshes if m.nx == n) for n in sorted({m.nx for m in meshes})},
           "operator": "nek_ax_ff (FP64-accurate)"}
    # the whole solve as one graph launch (device-side WHILE loop), then graphs of 10 iterations with
    # the host reading the unfinished count between replays
    for name, ipg in (("one_launch", -1), ("graphs_of_10", 10)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = B.solve(x, tol=tol, max_iter=20000, iters_per_graph=ipg, workspace=ws)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        pts_iters = sum(m.npts * int(r["iters"][pos]) for pos, m in enumerate(B.meshes))
        out[name] = {"seconds_to_%g" % tol: dt, "converged": r["converged"], "max_iters": int(r["iters"].max()),
                     "mean_iters": float(r["iters"].mean()), "iterations_run": r["iterations_run"],
                     "graph_launches": r["graph_launches"], "kernel_launches": r["kernel_launches"],
                     "gdofs_useful": pts_iters / dt / 1e9}
    return out


def net_apply_rates(torch, theta, mesh, reps=20):
    """One network application over every element of `mesh`: the FP32 CUDA-core form and the two BF16
    tensor-core forms (warp-level mma.sync, tcgen05), in points/s and useful TFLOP/s (16 416 flop per
    point)."""
    import numpy as np

    from paper_2011_04981_gb300 import nekax

    n = mesh.nelt
    rng = np.random.default_rng(0)
    xin = torch.from_numpy(rng.normal(size=(n, 2, 512)).astype(np.float32)).to("cuda")
    sc = torch.ones(n, dtype=torch.float32, device="cuda")
    c = torch.ones((n, 512), dtype=torch.float64, device="cuda")
    z = torch.empty_like(c)
    flop_pt = 2 * (2 * 16 * 27 + 16 * 16 * 27 + 16 * 27)
    _, bf16_peak = peaks_bf16()
    out = {"elements": n, "flop_per_point": flop_pt}
    for name, fn in (("fp32_cuda_cores", nekax.net_apply), ("bf16_mma_sync", nekax.net_apply_bf16_mma),
                     ("bf16_tcgen05", nekax.net_apply_bf16)):
        fn(n, 8, theta, xin, sc, c, z)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn(n, 8, theta, xin, sc, c, z)
        e1.record()
        e1.synchronize()
        t = e0.elapsed_time(e1) / reps / 1e3
        tf = n * 512 * flop_pt / t / 1e12
        out[name] = {"ms": t * 1e3, "gpts": n * 512 / t / 1e9, "tflops": tf}
    for name in ("bf16_mma_sync", "bf16_tcgen05"):
        out[name]["frac_of_bf16_peak"] = out[name]["tflops"] / bf16_peak
    out["speedup_tcgen05_vs_mma_sync"] = out["bf16_mma_sync"]["ms"] / out["bf16_tcgen05"]["ms"]
    return out


def net_block(torch, nelt):
    """Inference rates of the three network forms on nelt elements with random weights and inputs (the
    network's cost does not depend on the values)."""
    import numpy as np

    from paper_2011_04981_gb300 import nekax

    th = torch.from_numpy(np.random.default_rng(1).normal(scale=0.1, size=nekax.net_param_count())
                          .astype(np.float32)).to("cuda")

    class _M:
        pass

    m = _M()
    m.nelt = nelt
    return net_apply_rates(torch, th, m)


def peaks_bf16():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return "measured", float(p["bf16_tflops"])
    except Exception:
        return "fallback", 1900.0


def learned_block(torch, n_meshes=200, epochs=30, eval_elems=24):
    """Configuration 5: pairs from the solver on n_meshes random meshes of the family, GPU training with the
    library's kernels, then time to 1e-8 on a held-out eval_elems^3 mesh with and without the network."""
    from paper_2011_04981_gb300 import learned

    t0 = time.perf_counter()
    data = learned.make_training_data(n_meshes=n_meshes, pairs_per_mesh=100, seed=0)
    t_data = time.perf_counter() - t0
    val_data = learned.make_training_data(n_meshes=max(2, n_meshes // 20), pairs_per_mesh=100, seed=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    theta, hist = learned.train(data, epochs=epochs, batch=256, lr=2e-3, seed=0, kind="energy")
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    val = learned.validation_loss(theta, val_data)
    theta0 = learned.init_params(0, "cuda")
    val0 = learned.validation_loss(theta0, val_data)
    mesh = learned.mesh_family(seed=777, e=eval_elems)
    cmp = learned.compare_on_mesh(theta, mesh, seed=3, theta_untrained=theta0)
    cmp["net_apply"] = net_apply_rates(torch, theta, mesh)
    return {"pairs": len(data), "data_seconds": t_data, "train_seconds": t_train, "epochs": epochs,
            "loss": "element energy norm", "train_loss_first_last": [hist[0], hist[-1]],
            "val_loss_untrained": val0, "val_loss_trained": val,
            "eval_mesh": "%d^3 elements, nx=8, perturbation 0.15 h, stretch up to 8:1" % eval_elems, **cmp}


def native_fp64_block(torch, P, f, x, ws, iters, steps=3, tune=True):
    """The headline solve with the native FP64 operator (nek_ax on the FP64 pipe): fixed-iteration rate and
    its AX launches timed inside the solve."""
    from paper_2011_04981_gb300 import nekax, perfmodel

    nx = P.nx
    if tune:
        wt = torch.empty_like(f)
        nekax.tune_ax(nekax.AX_FP64, P.nelt, nx, P.D, P.G, f, wt)
        del wt
    out = solve_block(torch, P, f, x, ws, iters, nekax.AX_FP64, steps)
    t_ax = out["ax"]["ms_per_launch"] / 1e3
    hbm, kind = peaks()
    flops = perfmodel.ax_flops_per_point(nx) * P.npts
    out["ax"].update({"kernel": "k_ax_fp64<%d>" % nx, "tflops": flops / t_ax / 1e12,
                      "fp64_pipe_frac": flops / t_ax / 1e12 / FP64_PEAK_TFLOPS,
                      "hbm_frac_64B": 64 * P.npts / t_ax / 1e9 / hbm,
                      "elements_per_cta": nekax.get_ax_epb(nekax.AX_FP64, nx)})
    out["note"] = ("native FP64 (the paper's arithmetic); FP64 peak = 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz "
                   "= %.4f TFLOP/s; HBM %s %.0f GB/s" % (FP64_PEAK_TFLOPS, kind, hbm))
    return out


def solve_block(torch, P, f, x, ws, iters, impl, steps=3):
    """Fixed-iteration Jacobi-PCG rate with operator `impl`, and its AX launches timed inside the solve."""
    from paper_2011_04981_gb300 import nekax

    P.cg(f, x, tol=0.0, max_iter=iters, workspace=ws, ax_impl=impl)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ax_ms, ax_n = 0.0, 0
    e0.record(s)
    for _ in range(steps):
        r = P.cg(f, x, tol=0.0, max_iter=iters, workspace=ws, time_ax=True, ax_impl=impl)
        assert r["status"] == nekax.OK and r["iters"] == iters, r
        ax_ms += r["ax_ms_total"]
        ax_n += r["ax_launches"]
    e1.record(s)
    e1.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    ax_t = ax_ms / max(ax_n, 1) / 1e3
    return {"gdofs": P.npts * iters * steps / t / 1e9, "ms_per_step": 1e3 * t / steps, "steps": steps,
            "iters_per_step": iters,
            "ax": {"gdofs": P.npts / ax_t / 1e9, "ms_per_launch": ax_t * 1e3, "share_of_step": ax_ms / 1e3 / t}}


def tensor_core_block(torch, P, f, x, ws, iters, steps=3):
    """The headline solve with the FP64-accurate operator whose contractions run on the tensor cores
    (nek_ax_oz: BF16 digit slices, exact FP32 level sums in TMEM, float-pair recombination), in its solve
    form (element energies and the fused x / direction update, 104 algorithmic B/point)."""
    from paper_2011_04981_gb300 import nekax

    if not (P.nx % 2 == 0 and P.nx <= 10):
        return {"skipped": "nek_ax_oz takes even nx up to 10"}
    P.prepare_oz()
    out = solve_block(torch, P, f, x, ws, iters, nekax.AX_OZ, steps)
    hbm, kind = peaks()
    t_ax = out["ax"]["ms_per_launch"] / 1e3
    out["ax"].update({"kernel": "k_ax_oz<%d, 2>" % P.nx, "hbm_frac_104B": 104 * P.npts / t_ax / 1e9 / hbm})
    out["note"] = ("FP64-accurate; HBM %s %.0f GB/s.  Standalone (64 B/point) this operator is faster than the "
                   "float-float one (ax_sweep), inside the solve its fused update's FP64 operations (x and p "
                   "updates, energies, the join to FP64: 5 per point on the 2-per-clock FP64 pipe) are not "
                   "hidden by its two CTAs per SM" % (kind, hbm))
    return out


def solves_to_tol(torch, P, f, x, ws, tol=1e-8):
    """Seconds, iterations and final residual of Jacobi-PCG to a relative residual of tol with each FP64
    operator (wall clock around the synchronous call)."""
    from paper_2011_04981_gb300 import nekax

    out = {}
    ops = [("fp64_native", nekax.AX_FP64), ("fp64_float_float", nekax.AX_FF)]
    if P.nx % 2 == 0 and P.nx <= 10:
        P.prepare_oz()
        ops.append(("fp64_tensor_core", nekax.AX_OZ))
    for name, impl in ops:
        P.cg(f, x, tol=tol, max_iter=5, workspace=ws, ax_impl=impl)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = P.cg(f, x, tol=tol, max_iter=20000, workspace=ws, check_every=20, ax_impl=impl)
        torch.cuda.synchronize()
        out[name] = {"seconds": time.perf_counter() - t0, "iters": r["iters"], "relres": r["relres"],
                     "status": nekax.status_string(r["status"])}
    return out


def _guard(name, fn):
    """Run one block of the extras; a failure is recorded in the line instead of losing the line."""
    try:
        return fn()
    except Exception as exc:  # noqa: BLE001 -- the line must still be printed
        import traceback

        traceback.print_exc()
        return {"error": "%s: %s" % (type(exc).__name__, exc)}


def run_native(args):
    import torch

    from paper_2011_04981_gb300 import inputs, nekax, perfmodel
    from paper_2011_04981_gb300.problem import DeviceProblem

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    nx, e = args.nx, args.elems
    mesh = inputs.box_mesh(e, e, e, nx, perturb=0.1, seed=1)
    P = DeviceProblem(mesh, "cuda")
    f_host = torch.from_numpy(inputs.random_global_field(mesh, seed=2)).pin_memory()
    f = f_host.to("cuda")
    x = torch.empty_like(f)
    x_host = torch.empty_like(f_host).pin_memory()
    ws = torch.empty(nekax.cg_workspace_bytes(mesh.nelt, nx, False) // 8 + 64, dtype=torch.float64, device="cuda")
    staging = torch.empty(nekax.cg_host_staging_bytes(mesh.nelt, nx) // 8 + 64, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    iters = args.iters

    ax_impl = {"ff": nekax.AX_FF, "fp64": nekax.AX_FP64, "oz": nekax.AX_OZ}[args.ax]
    if ax_impl == nekax.AX_FF:
        P.prepare_ff()
    if ax_impl == nekax.AX_OZ:
        P.prepare_oz()
    if ax_impl == nekax.AX_OZ:
        pass  # fixed launch shape: two persistent CTAs per SM
    elif args.epb:
        if nekax.load().nek_set_ax_epb(int(ax_impl), nx, args.epb) != nekax.OK:
            raise SystemExit("--epb %d does not fit the AX kernel at nx = %d" % (args.epb, nx))
    elif args.tune:
        wt = torch.empty_like(f)
        nekax.tune_ax(ax_impl, mesh.nelt, nx, P.D, P.Gff if ax_impl == nekax.AX_FF else P.G, f, wt)
        del wt
    ax_epb = (nekax.load().nek_get_ax_epb(int(nekax.AX_FF_ENERGY if ax_impl == nekax.AX_FF else ax_impl), nx)
              if ax_impl != nekax.AX_OZ else "2 persistent CTAs per SM")
    for _ in range(args.warmup):
        P.cg(f, x, tol=0.0, max_iter=iters, workspace=ws, ax_impl=ax_impl)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ax_ms, ax_n, launches = 0.0, 0, 0
    e0.record(stream)
    for _ in range(args.steps):
        r = P.cg(f, x, tol=0.0, max_iter=iters, workspace=ws, time_ax=True, ax_impl=ax_impl)
        ax_ms += r["ax_ms_total"]
        ax_n += r["ax_launches"]
        launches += r["kernel_launches"]
        assert r["status"] == nekax.OK and r["iters"] == iters, r
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    barrier()
    t_dev = e0.elapsed_time(e1) / 1e3
    clk = clocks.stop()

    # end to end through the public host-buffer call: every step, nek_cg_solve_host copies that step's f
    # from pinned host memory to the device, solves, and copies x back before it returns.
    P.cg_host(f_host, x_host, tol=0.0, max_iter=iters, workspace=ws, staging=staging, ax_impl=ax_impl)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = P.cg_host(f_host, x_host, tol=0.0, max_iter=iters, workspace=ws, staging=staging, ax_impl=ax_impl)
        assert r["status"] == nekax.OK and r["iters"] == iters, r
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    barrier()

    if dist is not None:
        t_dev, t_e2e = max_over_ranks(dist, [t_dev, t_e2e], "cuda")

    pts = mesh.npts
    value = pts * iters * args.steps * world / t_dev / 1e9
    e2e = pts * iters * args.steps * world / t_e2e / 1e9
    ax_t = ax_ms / max(ax_n, 1) / 1e3
    ax_gdofs = pts / ax_t / 1e9
    flops = perfmodel.ax_flops_per_point(nx) * pts
    hbm, hbm_kind = peaks()
    traffic = traffic_from_profile(nx, mesh.nelt, args.ax)
    # the float-float operator of the solve also applies the x / direction update
    fused_dir = args.ax in ("ff", "oz")
    ax_bpp = 104 if fused_dir else 64
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "ff": "f64 (AX in f32-pair float-float, FP64-accurate)",
                  "oz": "f64 (AX contractions as BF16 digit slices on tcgen05 with exact FP32 level sums, "
                        "FP64-accurate)"}[args.ax],
        "data": "synthetic",
        "config": {"workload": "Jacobi-PCG, %d PCG iterations per step (AX+dssum+mask+dots+updates), "
                               "%dx%dx%d deformed box (perturbation 0.1 h), nx=%d, FP64-accurate, AX %s"
                               % (iters, e, e, e, nx, {"fp64": "native FP64 (nek_ax)",
                                                       "ff": "float-float on the FP32 pipes (nek_ax_ff)",
                                                       "oz": "contractions on the tensor cores (nek_ax_oz)"}[args.ax]),
                   "elements": mesh.nelt, "nx": nx, "points": pts, "iters_per_step": iters,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (G alone %.2f GB), no flush" % (pts * 48 / 1e9)},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": pts * 8, "d2h_bytes_per_step": pts * 8,
                "api": "nek_cg_solve_host: f and x in pinned host memory, both copies inside the call"},
        "gpu_launches": launches,
        "ax": {"gdofs": ax_gdofs, "ms_per_launch": ax_t * 1e3, "gflops": flops / ax_t / 1e9,
               "bytes_per_point": ax_bpp, "hbm_gbs": ax_bpp * pts / ax_t / 1e9,
               "hbm_frac": ax_bpp * pts / ax_t / 1e9 / hbm, "launches": ax_n,
               "share_of_step": ax_ms / 1e3 / t_dev, "elements_per_cta": ax_epb or "default"},
        "roofline": ({"bound": "alu", "achieved": flops / ax_t / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                      "frac": flops / ax_t / 1e12 / FP64_PEAK_TFLOPS, "traffic": traffic,
                      "kernel": "k_ax_fp64<%d>" % nx,
                      "note": "native FP64: DFMA-pipe bound; peak = 152 SM x 2 DFMA/clk x 2 x 2.07 GHz (nominal "
                              "1.25 TFLOP/s); HBM %s peak %.0f GB/s" % (hbm_kind, hbm)}
                     if args.ax == "fp64" else
                     {"bound": "hbm", "achieved": ax_bpp * pts / ax_t / 1e9, "peak": hbm, "unit": "GB/s",
                      "frac": ax_bpp * pts / ax_t / 1e9 / hbm, "traffic": traffic,
                      "kernel": ("k_ax_oz<%d, 2>" if args.ax == "oz" else
                                 "k_ax_ffi<%d>" if nx in (10, 12) else "k_ax_ff<%d>") % nx,
                      "note": ("FP64-accurate AX (%s) with the fused x / direction update, 104 algorithmic "
                               "B/point (p in and out 16, r 8, minv 8, x in and out 16, G 48, w 8)"
                               % ("tensor-core digit slices" if args.ax == "oz" else "float-float") if fused_dir else
                               "FP64-accurate float-float AX, 64 algorithmic B/point (u 8 + G 48 + w 8)") +
                              "; peak = %s HBM copy (MEASURED_PEAKS hbm_gbs); its instruction limit is the FP32 "
                              "pipe (see profiles)" % hbm_kind}),
        "clocks": clk,
    }
    ex = args.extra_set if rank == 0 else set()
    if "native" in ex and args.ax == "ff":
        line["fp64_native"] = _guard("native", lambda: native_fp64_block(torch, P, f, x, ws, iters,
                                                                         tune=args.tune))
        line["fp64_tensor_core"] = _guard("native", lambda: tensor_core_block(torch, P, f, x, ws, iters))
    if "solve" in ex:
        line["cg_to_1e-8"] = _guard("solve", lambda: solves_to_tol(torch, P, f, x, ws))
    if "mixed" in ex:
        precs = tuple(q.strip() for q in args.mixed_precisions.split(","))
        line["mixed"] = _guard("mixed", lambda: mixed_block(torch, P, f, x, precs))
    if "lvec" in ex:
        line["lvec"] = _guard("lvec", lambda: lvec_block(torch, P, iters))
    if "sweep" in ex:
        line["ax_sweep"] = _guard("sweep", lambda: ax_sweep(torch, nxs=tuple(args.sweep_nx), tune=args.tune,
                                                            elems=args.sweep_elems))
    if "learned" in ex:
        line["learned"] = _guard("learned", lambda: learned_block(torch, args.learned_meshes, args.learned_epochs))
    if "net" in ex:
        line["net_apply"] = _guard("net", lambda: net_block(torch, args.net_elems))
    if "batch" in ex and args.batch > 0:
        del ws, staging
        torch.cuda.empty_cache()
        line["batch"] = _guard("batch", lambda: batch_block(torch, args.batch))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        budget = args.cpu_seconds or 12.0
        single = cpu_baseline(nx, iters_budget_s=budget)
        threads = os.cpu_count() or 1
        allc = cpu_baseline(nx, iters_budget_s=budget, threads=threads) if threads > 1 else {"unavailable": "1 core"}
        if "unavailable" in allc:
            cb = dict(single)
        else:
            cb = dict(allc)
            cb["single_core"] = {"value": single["value"], "cores": 1, "sample": single["sample"]}
        for k in ("seconds", "per_sample"):
            cb.pop(k, None)
        line["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.cpu_baseline_only:
        return cpu_baseline_child(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
