#!/usr/bin/env python
"""Benchmark: GMG-preconditioned CG to a 1e-8 relative residual with the
vertex-patch / local p-multigrid smoother on the 3D Q4 32^3 perturbed-hex
workload (manufactured solution sin(pi x) sin(pi y) sin(pi z)).

One step = one complete solve from u = 0 (patch sweeps with Gather, Evaluate,
local p-MG V-cycles and Scatter on every mesh level, global residuals,
h-transfers, dense coarse solve, CG vector updates and dots).  The headline is
the mixed-precision path (FP32 patch smoother and GMG levels, FP64 CG and
coarse solve); the plain FP64 path is timed beside it.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle instead.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP32_PEAK_DERIVED = 152 * 128 * 2 * 2.070e9      # SMs x FP32 lanes x 2 flops x max SM clock
FP64_PEAK_NOMINAL = 1.25e12                      # GB300 FP64 rate (nominal)
# DRAM bytes (read + write) of one finest-level colour launch of the benchmark workload from an ncu capture of
# the current kernel (variant 10, colour 0: 3,375 patches), scaled to the sweep's average launch (29,791 / 8
# patches); valid for that variant only.  None: the kernel changed after its last full capture (the
# degree-4 FP32 sweep capture under profiles/: 111.6 MB read + 6.7 MB written, 130.5 MB per average
# launch, measured before the geometry loads were split by format), so no DRAM count of the kernel as
# built is on record.
PATCH_LAUNCH_TRAFFIC = {"variant": 10, "bytes": None}
METRIC = "patch-smoother DoFs/s and CG time-to-1e-8 residual: mixed/learned vs plain FP64, 1 GB300"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2_3d_q4_n32_perturbed")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison arm")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-interval arm")
    ap.add_argument("--batch-structured", action="store_true",
                    help="--batch: structured 8^3 cubes instead of the unstructured meshes")
    ap.add_argument("--batch-refined", action="store_true",
                    help="--batch: every unstructured mesh refined once (two mesh levels, ~40k cells)")
    ap.add_argument("--batch", type=int, default=0,
                    help="instead: K independent problems (3D, 8^3 cells, degrees 2/4/6/8) solved together")
    ap.add_argument("--no-c3", action="store_true", help="skip the 48^3 Q7 sub-record (workloads.c3)")
    ap.add_argument("--sweep-only", action="store_true",
                    help="instead: set up one problem and run a few finest-level patch sweeps inside the NVTX "
                         "range 'sweeps' (a small driver for kernel captures)")
    ap.add_argument("--N", type=int, default=16, help="--sweep-only: cells per direction")
    ap.add_argument("--p", type=int, default=4, help="--sweep-only: degree")
    ap.add_argument("--dim", type=int, default=3, help="--sweep-only: dimension")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"], help="--sweep-only")
    ap.add_argument("--sweeps", type=int, default=3, help="--sweep-only: sweeps inside the range")
    ap.add_argument("--geometry-bf16", action="store_true",
                    help="--sweep-only, mixed precision: the patch kernels load BF16 geometry")
    ap.add_argument("--variant", type=int, default=-1,
                    help="--sweep-only: launch-shape variant without set-up timing (default: autotuned)")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------- CPU baseline
# The oracle (plain FP64 numpy, dense patch matrices) timed on the host cores
# of the GPU machine.  It runs in a child process with no GPU visible, which
# spreads a bounded sample of finest-level patches over a spawn pool with one
# single-threaded worker per core: every worker builds its patches' dense
# level matrices and Lanczos intervals (set-up, timed apart), then times
# Evaluate + one local V-cycle per visit.  All workers run at once, so the
# aggregate visit rate includes their contention for memory bandwidth.

def _oracle_sample_worker(task):
    """One worker: (workload name, vertex indices, visits per patch) ->
    timings.  Imports the oracle only here, in the spawned process."""
    import numpy as np
    from oracle import fem, lanczos as lz, patch as pt
    from paper_2510_17785_gb300 import inputs
    wname, vids, reps, dims = task
    w = inputs.WORKLOADS[wname] if wname in inputs.WORKLOADS else inputs.Workload(wname, *dims)
    prob = inputs.make_problem(w)
    m = fem.StructuredMesh(w.dim, w.N, prob.coords, prob.kappa)
    verts = pt.interior_vertices(w.dim, w.N)
    u = inputs.random_vector(5, w.dim, w.p, w.N)
    b = inputs.random_vector(6, w.dim, w.p, w.N)
    t0 = time.perf_counter()
    patches = []
    for vi in vids:
        P = pt.Patch(m, verts[vi], pt.levels_halving(w.p))
        patches.append((P, lz.lanczos_bounds_fn(seed=0)(P, pt.patch_id(w.dim, w.N, verts[vi]))))
    t_build = time.perf_counter() - t0
    sm = pt.Smoother()
    t0 = time.perf_counter()
    for _ in range(reps):
        for P, bd in patches:
            pt.local_solve(P, P.residual(u, b), sm, bd, 1)
    return {"t_build": t_build, "t_visits": time.perf_counter() - t0, "visits": reps * len(vids),
            "patches": len(vids)}


def _oracle_iterations_worker(task):
    """The oracle's own GMG-preconditioned CG iteration count on a small
    problem of the workload's kind (same degree, perturbation law,
    coefficient and right-hand-side kind)."""
    import numpy as np
    from oracle import fem, gmg, lanczos as lz, patch as pt
    from paper_2510_17785_gb300 import inputs
    wname, N = task
    w = inputs.WORKLOADS[wname].with_(name=f"{wname}_small", N=N, seed=inputs.WORKLOADS[wname].seed + 17)
    prob = inputs.make_problem(w)
    m = fem.StructuredMesh(w.dim, N, prob.coords, prob.kappa)
    G = gmg.GMG(m, w.p, w.coarse_N, smoother_args=dict(sm=pt.Smoother(), bounds_fn=lz.lanczos_bounds_fn(seed=0)))
    free = G.free[-1]
    if w.rhs == "manufactured":
        f = lambda X: w.dim * np.pi ** 2 * np.prod(np.sin(np.pi * X), axis=1)
        b = m.load_vector(f, w.p, w.p + 2) * free
    else:
        b = prob.rhs * free
    _, it, hist = gmg.pcg(G.A[-1], b, G.vcycle, 1e-8, 200)
    return {"iterations": it, "relres": hist[-1], "N": N}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def _cpu_child(spec: dict) -> dict:
    """Runs in the GPU-less child: the parallel sample (and, if asked, the
    oracle's iteration count first)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import numpy as np
    from oracle import patch as pt
    from paper_2510_17785_gb300 import inputs
    cores = os.cpu_count() or 1
    w = inputs.WORKLOADS[spec["workload"]]
    nv = len(pt.interior_vertices(w.dim, w.N))
    rng = np.random.default_rng(1234 + spec.get("seed", 0))
    per = spec["patches_per_core"]
    pick = rng.choice(nv, size=min(nv, cores * per), replace=False)
    tasks = [(w.name, [int(v) for v in pick[i::cores]], spec["reps"], None) for i in range(cores)]
    out = {"cores": cores, "cpu": cpu_model()}
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=ctx) as ex:
        if spec.get("iterations_N"):
            out["oracle_cg"] = ex.submit(_oracle_iterations_worker, (w.name, spec["iterations_N"])).result()
        t0 = time.perf_counter()
        res = list(ex.map(_oracle_sample_worker, [t for t in tasks if t[1]]))
        out["wall_s"] = time.perf_counter() - t0
    out["visit_rate"] = sum(r["visits"] / r["t_visits"] for r in res)          # visits / s, all cores together
    out["t_visit_core"] = sum(r["t_visits"] for r in res) / sum(r["visits"] for r in res)
    out["t_build_core"] = sum(r["t_build"] for r in res) / sum(r["patches"] for r in res)
    out["patches"] = sum(r["patches"] for r in res)
    out["visits"] = sum(r["visits"] for r in res)
    return out


def oracle_cpu_sample(workload: str, patches_per_core: int, reps: int, iterations_N: int = 0, seed: int = 0):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    spec = dict(workload=workload, patches_per_core=patches_per_core, reps=reps, iterations_N=iterations_N,
                seed=seed)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-child", json.dumps(spec)],
                       capture_output=True, text=True, env=env, timeout=1200)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def solve_visits(w, levels: int) -> int:
    """Patch visits of one GMG-PCG iteration: every V-cycle sweeps every
    smoothed mesh level twice (forward and reverse)."""
    visits = 0
    for l in range(1, levels):
        Nl = w.N >> (levels - 1 - l)
        visits += 2 * (Nl - 1) ** w.dim
    return visits


def cpu_baseline(w, levels, patches_per_core=2, reps=20):
    """The oracle on all host cores: its own GMG-PCG iteration count (same
    kind of problem at twice the coarsest mesh size; the GPU path is not
    consulted) times the patch work of one iteration, at the visit rate of a
    bounded parallel sample."""
    t = oracle_cpu_sample(w.name, patches_per_core, reps, iterations_N=2 * w.coarse_N)
    iters = t["oracle_cg"]["iterations"]
    t_solve = iters * solve_visits(w, levels) / t["visit_rate"]
    return {
        "value": w.n_free / t_solve, "unit": "DoFs/s", "cores": t["cores"], "kind": "oracle", "cpu": t["cpu"],
        "sample": (f"{t['patches']} seeded finest-level patches on {t['cores']} cores (one single-threaded "
                   f"worker each, all at once), {reps} Evaluate + V-cycle visits per patch: "
                   f"{t['visit_rate']:.0f} visits/s together ({t['t_visit_core'] * 1e3:.3f} ms per visit per "
                   f"core); extrapolated to {iters} CG iterations x 2 sweeps x all patches of levels 1..{levels - 1} "
                   f"(patch work only: the oracle's global matrix-vector products are not counted; building the "
                   f"dense patch matrices is set-up, {t['t_build_core'] * 1e3:.0f} ms per patch per core, not "
                   f"counted); the iteration count is the oracle's own GMG-PCG on the same kind of problem with "
                   f"{t['oracle_cg']['N']} cells per direction (relres {t['oracle_cg']['relres']:.1e}); "
                   f"{t['wall_s']:.1f} s wall"),
        "oracle_iterations": iters,
        "extrapolated": True,
        "t_solve_extrapolated_s": t_solve,
    }


# ------------------------------------------------------------ multi-rank
def aggregate(t_local_ms: float, n_free_local: int, dist: bool):
    """Whole-job time and throughput: every rank solved its own problem, the
    job took as long as the slowest rank (max over ranks), and the job's
    throughput is all ranks' DoFs over that time."""
    t_max, n_total = t_local_ms, n_free_local
    if dist:
        import torch
        import torch.distributed as td
        dev = torch.device("cuda", torch.cuda.current_device()) if td.get_backend() == "nccl" else torch.device("cpu")
        tt = torch.tensor([t_local_ms], dtype=torch.float64, device=dev)
        nn = torch.tensor([float(n_free_local)], dtype=torch.float64, device=dev)
        td.all_reduce(tt, op=td.ReduceOp.MAX)
        td.all_reduce(nn, op=td.ReduceOp.SUM)
        t_max, n_total = float(tt.item()), int(nn.item())
    return t_max, n_total / (t_max * 1e-3)


# ------------------------------------------------------------ sweep only
def run_sweep_only(args):
    """Set up one problem (unit cube/square, N cells per direction, degree p,
    U(-0.25h, 0.25h) vertex perturbation, kappa = 1) and run `sweeps`
    finest-level patch sweeps inside the NVTX range "sweeps", then one
    operator apply.  For kernel captures on cases far smaller than the
    benchmark:  ncu --nvtx --nvtx-include "sweeps/" -k regex:k_patch ..."""
    import torch
    from paper_2510_17785_gb300 import inputs, pmg

    levels, n = 1, args.N
    while n % 2 == 0 and n // 2 >= 2:
        levels, n = levels + 1, n // 2
    w = inputs.Workload(f"sweep_{args.dim}d_q{args.p}_n{args.N}", args.dim, args.N, args.p, 0.25, "uniform",
                        ("const", 1.0), "uniform", 77)
    prob = inputs.make_problem(w)
    prec = pmg.PREC_MIXED if args.precision == "mixed" else pmg.PREC_FP64
    tune = dict(autotune=0, variant=args.variant) if args.variant >= 0 else {}
    if args.geometry_bf16:
        tune["geometry_bf16"] = 1
    ctx = pmg.Context(0, precision=prec, **tune)
    ctx.mesh_structured(w.dim, w.N, w.p, levels, prob.coords, prob.kappa)
    ctx.setup()
    b = torch.tensor(prob.rhs, device="cuda")
    u = torch.zeros_like(b)
    lf = levels - 1
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("sweeps")
    for _ in range(args.sweeps):
        ctx.patch_smooth(lf, b, u, 1, False)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    Au = torch.zeros_like(b)
    ctx.apply(lf, u, Au)
    torch.cuda.synchronize()
    print(json.dumps({"sweep_only": w.name, "sweeps": args.sweeps, "tuning": ctx.tuning(),
                      "level_tuning": [ctx.tuning_level(lv) for lv in range(levels)],
                      "u_max": float(u.abs().max())}))
    ctx.close()


# ------------------------------------------------------------------ ours
def learned_arm(w, levels, local, timed_solves, dev):
    """Mixed precision with MLP-predicted Chebyshev intervals: train on the
    Lanczos estimates of three small problems of the same degree, then time
    the interval computation (MLP vs Lanczos) and the solve on the workload."""
    import numpy as np
    import torch
    from paper_2510_17785_gb300 import inputs, pmg

    t0 = time.perf_counter()
    Xs, Ts = [], []
    train = [(8, 0.25, ("const", 1.0)), (8, 0.15, ("loguniform", -1.0, 1.0)), (6, 0.3, ("loguniform", -2.0, 2.0))]
    for i, (N, pert, kap) in enumerate(train):
        wt = inputs.Workload(f"train{i}", w.dim, N, w.p, pert, "uniform", kap, "uniform", 9000 + i)
        pt_ = inputs.make_problem(wt)
        lv, n = 1, N
        while n % 2 == 0 and n // 2 >= 2:
            lv, n = lv + 1, n // 2
        c = pmg.Context(local, precision=pmg.PREC_MIXED)
        c.mesh_structured(wt.dim, N, wt.p, lv, pt_.coords, pt_.kappa)
        c.setup()
        X, T = pmg.mlp_training_data(c)
        Xs.append(X)
        Ts.append(T)
        c.close()
    X, T = torch.cat(Xs), torch.cat(Ts)
    norm = pmg.mlp_norm(X, T, device=local)
    f32 = lambda a: torch.tensor(np.asarray(a), dtype=torch.float32, device=dev)
    params = f32(pmg.mlp_init(11))
    hist = pmg.mlp_train(params, f32(norm), X, T, device=local, epochs=150, batch=256, lr=2e-3, asym=4.0)
    t_train = time.perf_counter() - t0

    prob = inputs.make_problem(w)
    ctx = pmg.Context(local, precision=pmg.PREC_MIXED, bounds=pmg.BOUNDS_FIXED)
    ctx.mesh_structured(w.dim, w.N, w.p, levels, prob.coords, prob.kappa)
    ctx.setup()
    b = torch.zeros((w.p * w.N + 1) ** w.dim, dtype=torch.float64, device=dev)
    ctx.rhs_manufactured(b)
    out = {}
    ctx.compute_bounds(pmg.BOUNDS_LANCZOS)                    # warm-up of both sources
    ctx.set_mlp(params.cpu().numpy(), norm)
    ctx.compute_bounds(pmg.BOUNDS_MLP)
    for src, key in ((pmg.BOUNDS_LANCZOS, "lanczos"), (pmg.BOUNDS_MLP, "mlp")):
        torch.cuda.synchronize()
        t = time.perf_counter()
        ctx.compute_bounds(src)
        torch.cuda.synchronize()
        out["bounds_" + key] = time.perf_counter() - t
        if key == "lanczos":
            x = torch.zeros_like(b)
            out["its_lanczos"], _, _ = ctx.solve_cg(b, x, 1e-8, 200)
    ms, its, _, _ = timed_solves(ctx, b, 3, 1)
    ctx.close()
    out.update(ms=ms, its=its, train_s=t_train, samples=int(X.shape[0]), train_problems=len(train),
               loss=[float(hist[0]), float(hist[-1])])
    return out


def precision_record(w, local, dev, flush, stream, fma32, sweep_only_fp64=True):
    """One workload in three arms: mixed precision, mixed precision with the
    patch kernels' geometry rounded to BF16, and FP64: set-up, the
    finest-level sweep (time, roofline fraction), a GMG-PCG solve to 1e-8 in
    the mixed arms, and the difference between one sweep of each mixed arm and
    one FP64 sweep from the same state (u = 0).  BF16 geometry is accepted when
    its CG iteration count stays within one of the FP32-geometry count."""
    import torch
    from paper_2510_17785_gb300 import inputs, pmg

    levels = int(round(math.log2(w.N // w.coarse_N))) + 1
    prob = inputs.make_problem(w)
    out = {"workload": w.name, "dim": w.dim, "cells_per_dir": w.N, "p": w.p, "n_free": w.n_free,
           "h_levels": levels}

    def ev_time(fn):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    b = torch.zeros(w.n_dofs, dtype=torch.float64, device=dev)
    u_sw = {}
    arms = (("mixed", dict(precision=pmg.PREC_MIXED)),
            ("mixed_bf16_geometry", dict(precision=pmg.PREC_MIXED, geometry_bf16=1)),
            ("fp64", dict(precision=pmg.PREC_FP64)))
    for name, opt in arms:
        ctx = pmg.Context(local, **opt)
        ctx.mesh_structured(w.dim, w.N, w.p, levels, prob.coords, prob.kappa)
        t0 = time.perf_counter()
        ctx.setup()
        t_setup = time.perf_counter() - t0
        if prob.rhs is None:
            ctx.rhs_manufactured(b)
        else:
            b.copy_(torch.tensor(prob.rhs, device=dev))
        lf = levels - 1
        u = torch.zeros_like(b)
        ctx.patch_smooth(lf, b, u, 1, False)             # one sweep from u = 0, kept for the comparison
        torch.cuda.synchronize()
        u_sw[name] = u.clone()
        nsw = 1 if name == "fp64" else 3
        ms, _ = ev_time(lambda: ctx.patch_smooth(lf, b, u, nsw, False))
        t_sweep = ms / nsw * 1e-3
        flops = ctx.sweep_flops(lf)
        rec = {"setup_s": t_setup, "sweep_ms": t_sweep * 1e3, "sweep_dofs_per_s": w.n_free / t_sweep,
               "sweep_flops": flops}
        if name != "fp64" or not sweep_only_fp64:
            rec["roofline"] = {"bound": "alu", "achieved": flops / t_sweep / 1e12, "unit": "TFLOP/s",
                               "peak": FP32_PEAK_DERIVED / 1e12, "frac": flops / t_sweep / FP32_PEAK_DERIVED,
                               "frac_of_measured_fma": flops / t_sweep / fma32,
                               "kernel": f"k_patch<3,{w.p},float,SWEEP,variant> (finest-level sweep, "
                                         f"one launch per colour or one persistent launch)"}
            x = torch.zeros_like(b)
            ctx.solve_cg(b, x, 1e-8, 300)                 # warm-up (captures the iteration graph)
            x.zero_()
            ms, (it, rel, _) = ev_time(lambda: ctx.solve_cg(b, x, 1e-8, 300))
            rec.update(solve_ms=ms, cg_iterations=it, final_relres=rel, dofs_per_s=w.n_free / (ms * 1e-3),
                       tuning_level_variants=[ctx.tuning_level(lv)[0] for lv in range(levels)],
                       persistent_levels=[lv for lv in range(levels) if ctx.level_persistent(lv)[0]])
        out[name] = rec
        ctx.close()
    ref = u_sw["fp64"]
    rel = lambda a: float((a - ref).abs().max() / ref.abs().max())
    out["mixed_vs_fp64_one_sweep_rel_max_err"] = rel(u_sw["mixed"])
    g = out["mixed_bf16_geometry"]
    out["geometry_bf16"] = {
        "one_sweep_rel_max_err_vs_fp64": rel(u_sw["mixed_bf16_geometry"]),
        "fp32_geometry_one_sweep_rel_max_err_vs_fp64": out["mixed_vs_fp64_one_sweep_rel_max_err"],
        "cg_iterations": g["cg_iterations"], "fp32_geometry_cg_iterations": out["mixed"]["cg_iterations"],
        "sweep_ms": g["sweep_ms"], "fp32_geometry_sweep_ms": out["mixed"]["sweep_ms"],
        "solve_ms": g.get("solve_ms"), "fp32_geometry_solve_ms": out["mixed"].get("solve_ms"),
        "accepted": g["cg_iterations"] <= out["mixed"]["cg_iterations"] + 1,
        "note": "geometry rounded to BF16 and loaded by the patch kernels as packed BF16 pairs (half the bytes "
                "and load instructions of FP32 geometry); the GMG level operators keep FP32 geometry",
    }
    return out


def run_batch(args):
    """K independent problems solved together by pmg_batch_solve_cg, against
    the same problems solved one after another.  Default: the unstructured
    batch (inputs.c4_problems: extruded and split-tetrahedron hexahedral
    meshes and split-triangle quadrilateral meshes of about 5,000 cells,
    degrees 2, 4, 6, 8 in turn, kappa 10^U(-2, 2), Lanczos intervals, the
    two-level preconditioner with the Q1 coarse space).  --batch-structured:
    unit cubes of 8^3 cells with the same degrees and coefficients."""
    import numpy as np
    import torch
    from paper_2510_17785_gb300 import inputs, pmg

    K = args.batch
    ctxs, bs, n_free, desc, kinds = [], [], 0, [], {}
    t0 = time.perf_counter()
    if args.batch_structured:
        N = 8
        for k in range(K):
            p = (2, 4, 6, 8)[k % 4]
            wk = inputs.Workload(f"batch{k}", 3, N, p, 0.2, "sphere", ("loguniform", -2.0, 2.0), "uniform",
                                 4004 * 64 + k)
            pr = inputs.make_problem(wk)
            c = pmg.Context(0, precision=pmg.PREC_MIXED, autotune=2)   # shapes for a shared GPU
            c.mesh_structured(3, N, p, 3, pr.coords, pr.kappa)
            c.setup()
            ctxs.append(c)
            bs.append(torch.tensor(pr.rhs, device="cuda"))
            n_free += wk.n_free
        workload = f"{K} problems, unit cube 8^3 cells, degrees 2/4/6/8, kappa 10^U(-2,2)"
    else:
        meshes = {}
        for u in inputs.c4_problems(K):
            c = pmg.Context(0, precision=pmg.PREC_MIXED, bounds=pmg.BOUNDS_LANCZOS)
            if args.batch_refined:
                X, C, Xf, Cf, par, ch, bnd, kappa = inputs.make_refined_problem(u)
                c.mesh_upload(X.shape[1], X, C, u.p)
                c.mesh_upload(X.shape[1], Xf, Cf, level=1, parent=par, child=ch, vertex_on_boundary=bnd, kappa=kappa)
                C = Cf
            else:
                X, C, bnd, kappa = inputs.make_unstructured_problem(u)
                c.mesh_upload(X.shape[1], X, C, u.p, vertex_on_boundary=bnd, kappa=kappa)
            c.setup()
            lf = 1 if args.batch_refined else 0
            total, free = c.num_dofs(lf)
            rhs = np.random.default_rng(u.seed + 1).uniform(-1.0, 1.0, total)
            ctxs.append(c)
            bs.append(torch.tensor(rhs, device="cuda"))
            n_free += free
            kinds.setdefault(u.kind, {"cells": len(C), "problems": 0, "valences": None})
            kinds[u.kind]["problems"] += 1
            if kinds[u.kind]["valences"] is None:
                pm = c.get_patch_map(lf)
                kinds[u.kind]["valences"] = sorted({int(v) for v in (pm[:, 1:] >= 0).sum(axis=1)})
        if args.batch_refined:
            workload = (f"{K} unstructured problems, each a ~5k-cell mesh (extruded / split-tetrahedron hexahedral, "
                        f"split-triangle quadrilateral) refined once (~40k hexahedra, ~22k quadrilaterals), degrees "
                        f"2/4/6/8, kappa 10^U(-2,2), Lanczos intervals, V-cycle over the two mesh levels with the "
                        f"coarse mesh's Q1 space")
        else:
            workload = (f"{K} unstructured problems (extruded / split-tetrahedron hexahedral and split-triangle "
                        f"quadrilateral meshes, ~5k cells each), degrees 2/4/6/8, kappa 10^U(-2,2), Lanczos "
                        f"intervals, two-level preconditioner with the Q1 coarse space")
    t_setup = time.perf_counter() - t0
    us = [torch.zeros_like(b) for b in bs]
    stream = torch.cuda.current_stream()

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    def batch():
        return pmg.batch_solve_cg(ctxs, bs, us, 1e-8, 200)

    def one_by_one():
        return [c.solve_cg(b, u, 1e-8, 200)[0] for c, b, u in zip(ctxs, bs, us)]

    for _ in range(args.warmup):
        batch()
    tb, ts, its = [], [], None
    for _ in range(args.steps):
        l0 = sum(c.launch_count() for c in ctxs)
        t, (its, _, _) = timed(batch)
        launches = sum(c.launch_count() for c in ctxs) - l0
        tb.append(t)
        t, its1 = timed(one_by_one)
        ts.append(t)
        assert its1 == its
    mb, msq = statistics.mean(tb), statistics.mean(ts)
    print(json.dumps({
        "metric": "batched GMG-PCG to 1e-8: free DoFs of all problems / time, independent problems of mixed degree",
        "value": n_free / (mb * 1e-3), "unit": "DoFs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": mb, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 local/GMG + f64 CG", "data": "synthetic",
        "config": {"workload": workload, "n_free_total": n_free, "setup_s": t_setup, "meshes": kinds or None},
        "one_by_one_ms": msq, "speedup_vs_one_by_one": msq / mb, "cg_iterations": its,
        "gpu_launches": launches,
    }))
    for c in ctxs:
        c.close()


def run_ours(args):
    import torch
    from paper_2510_17785_gb300 import inputs, pmg

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if dist:
        import torch.distributed as td
        torch.cuda.set_device(local)
        td.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w = inputs.WORKLOADS[args.workload]
    if rank > 0:
        w = w.with_(seed=w.seed + 100 * rank)          # independent replica per rank
    levels = int(round(math.log2(w.N // w.coarse_N))) + 1
    prob = inputs.make_problem(w)

    def make(precision):
        ctx = pmg.Context(local, precision=precision)
        ctx.mesh_structured(w.dim, w.N, w.p, levels, prob.coords, prob.kappa)
        t0 = time.perf_counter()
        ctx.setup()
        return ctx, time.perf_counter() - t0

    nd = w.n_dofs
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def timed_solves(ctx, b, nsteps, nwarm):
        x = torch.zeros_like(b)
        its = []
        for _ in range(nwarm):
            x.zero_()
            ctx.solve_cg(b, x, 1e-8, 200)
        ms = []
        launches0 = ctx.launch_count()
        torch.cuda.nvtx.range_push("timed_solves")
        for _ in range(nsteps):
            x.zero_()
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            it, rel, _ = ctx.solve_cg(b, x, 1e-8, 200)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            its.append((it, rel))
        torch.cuda.nvtx.range_pop()
        return ms, its, ctx.launch_count() - launches0, x

    result = {}
    arms = [("mixed", pmg.PREC_MIXED)] + ([] if args.no_fp64 else [("fp64", pmg.PREC_FP64)])
    clocks = Clocks(local)
    for name, prec in arms:
        ctx, t_setup = make(prec)
        b = torch.zeros(nd, dtype=torch.float64, device=dev)
        ctx.rhs_manufactured(b)
        torch.cuda.synchronize()
        if dist:
            torch.distributed.barrier()
        if name == "mixed":
            clocks.start()
        ms, its, launches, x = timed_solves(ctx, b, args.steps, args.warmup)
        if name == "mixed":
            clk = clocks.stop()
        # dominant kernel: the patch sweep on the finest level, timed on this stream
        lf = levels - 1
        u = torch.zeros_like(b)
        for _ in range(2):
            ctx.patch_smooth(lf, b, u, 1, False)
        nsw = 3
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.patch_smooth(lf, b, u, nsw, False)
        e1.record(stream)
        torch.cuda.synchronize()
        t_sweep = e0.elapsed_time(e1) / nsw * 1e-3
        flops = ctx.sweep_flops(lf)
        # end to end through the host-vector entry point (pinned host buffers)
        bh = torch.empty(nd, dtype=torch.float64).pin_memory()
        bh.copy_(b.cpu())
        uh = torch.empty(nd, dtype=torch.float64).pin_memory()
        e2e_ms = []
        for _ in range(max(1, min(args.steps, 3))):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.solve_cg_host(bh.numpy(), uh.numpy(), 1e-8, 200)
            e1.record(stream)
            torch.cuda.synchronize()
            e2e_ms.append(e0.elapsed_time(e1))
        err = float((x - torch.tensor(uh.numpy(), device=dev)).abs().max())
        result[name] = dict(ms=ms, its=its, launches=launches, t_sweep=t_sweep, sweep_flops=flops,
                            e2e_ms=e2e_ms, setup_s=t_setup, maxdiff_e2e=err,
                            umax=float(x.abs().max()), tuning=ctx.tuning(),
                            level_variants=[ctx.tuning_level(lv)[0] for lv in range(levels)],
                            persistent={lv: ctx.level_persistent(lv) for lv in range(levels)},
                            dense_local={lv: ctx.level_dense_local(lv) for lv in range(levels)})
        if name == "mixed":
            result["fma32"] = ctx.fma_peak(pmg.PREC_MIXED)
            result["fma64"] = ctx.fma_peak(pmg.PREC_FP64)
        ctx.close()

    if not args.no_learned:
        result["learned"] = learned_arm(w, levels, local, timed_solves, dev)
    if not args.no_c3 and world == 1:
        result["c3"] = precision_record(inputs.C3, local, dev, flush, stream, result["fma32"])
    if world == 1 and args.workload == inputs.C2.name:
        result["c2_geometry_bf16"] = precision_record(w, local, dev, flush, stream, result["fma32"])["geometry_bf16"]

    head = result["mixed"]
    t_step = sum(head["ms"]) / len(head["ms"])
    t_max, value = aggregate(t_step, w.n_free, dist)
    achieved = head["sweep_flops"] / head["t_sweep"]
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "DoFs/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_max,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 (patch smoother, local p-MG, GMG levels) + f64 (CG, residual, dots, coarse solve)",
        "data": "synthetic (seeded perturbed hex mesh, manufactured right-hand side)",
        "config": {
            "workload": w.name, "dim": w.dim, "cells_per_dir": w.N, "p": w.p, "n_free": w.n_free,
            "h_levels": levels, "p_levels": [w.p >> k for k in range(8) if w.p >> k >= 1],
            "smoother": "Chebyshev degree 3 on D^-1 A, Lanczos (16-step) bounds, N_MG = 1",
            "rtol": 1e-8, "step": "one GMG-PCG solve from u = 0",
            "l2": "flushed (512 MB write) before every timed step",
            "replicas": world,
            "patch_kernel_launch": {"variant": head["tuning"][0], "threads_per_cta": head["tuning"][1],
                                    "patches_per_cta": head["tuning"][2],
                                    "autotune_ms_per_variant": [round(x, 4) for x in head["tuning"][3]],
                                    "variant_per_mesh_level": head["level_variants"],
                                    "persistent_levels": head["persistent"],
                                    "tabulated_local_solve_levels": head["dense_local"]},
        },
        "time_to_solution_ms": t_max,
        "cg_iterations": [i for i, _ in head["its"]],
        "final_relres": max(r for _, r in head["its"]),
        "sweep": {"dofs_per_s": w.n_free / head["t_sweep"], "ms": head["t_sweep"] * 1e3,
                  "flops": head["sweep_flops"]},
        "setup_s": head["setup_s"],
        "roofline": {
            "bound": "alu", "achieved": achieved / 1e12,
            "peak": FP32_PEAK_DERIVED / 1e12, "unit": "TFLOP/s",
            "frac": achieved / FP32_PEAK_DERIVED,
            "traffic": (PATCH_LAUNCH_TRAFFIC["bytes"] if w.name == "c2_3d_q4_n32_perturbed"
                        and head["tuning"][0] == PATCH_LAUNCH_TRAFFIC["variant"] else None),
            "traffic_note": ("DRAM bytes per colour launch of the finest-level sweep; null: the kernel changed after "
                             "its last full ncu capture (degree-4 FP32 sweep under profiles/: 118.3 MB per colour-0 "
                             "launch, 130.5 MB per average launch, the algorithmic bytes)"),
            "kernel": "k_patch<3,4,float,SWEEP,variant> (finest-level patch sweep, 8 colour launches)",
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
            "measured_fma_peak": result["fma32"] / 1e12,
            "frac_of_measured_fma": achieved / result["fma32"],
        },
        "e2e": {"value": world * w.n_free / (statistics.mean(head["e2e_ms"]) * 1e-3), "unit": "DoFs/s",
                "ms": statistics.mean(head["e2e_ms"]), "h2d_bytes_per_step": nd * 8, "d2h_bytes_per_step": nd * 8,
                "api": "pmg_solve_cg_host"},
        "gpu_launches": head["launches"],
        "clocks": clk,
    }
    if "fp64" in result:
        f = result["fp64"]
        t64 = sum(f["ms"]) / len(f["ms"])
        a64 = f["sweep_flops"] / f["t_sweep"]
        out["fp64_plain"] = {
            "value": world * w.n_free / (t64 * 1e-3), "ms_per_step": t64,
            "cg_iterations": [i for i, _ in f["its"]], "final_relres": max(r for _, r in f["its"]),
            "sweep_ms": f["t_sweep"] * 1e3, "sweep_dofs_per_s": w.n_free / f["t_sweep"],
            "roofline": {"bound": "alu", "achieved": a64 / 1e12, "peak": FP64_PEAK_NOMINAL / 1e12,
                         "unit": "TFLOP/s", "frac": a64 / FP64_PEAK_NOMINAL,
                         "peak_source": "nominal GB300 FP64 rate", "measured_fma_peak": result["fma64"] / 1e12},
            "speedup_mixed_vs_fp64": t64 / t_max,
            "max_abs_diff_mixed_vs_fp64_solution": None,
        }
    if "learned" in result:
        L = result["learned"]
        tl = sum(L["ms"]) / len(L["ms"])
        out["learned"] = {
            "value": world * w.n_free / (tl * 1e-3), "ms_per_step": tl,
            "cg_iterations": [i for i, _ in L["its"]], "final_relres": max(r for _, r in L["its"]),
            "bounds_s_mlp": L["bounds_mlp"], "bounds_s_lanczos": L["bounds_lanczos"],
            "iterations_with_lanczos_bounds": L["its_lanczos"],
            "train": {"problems": L["train_problems"], "samples": L["samples"], "s": L["train_s"],
                      "loss_first_last": L["loss"]},
            "note": "mixed precision; Chebyshev intervals from the BF16 MLP (16-64-64-2) trained in this run on "
                    "Lanczos estimates of three small problems of the same degree",
        }
    if "c3" in result:
        out["workloads"] = {"c3": result["c3"]}
    if "c2_geometry_bf16" in result:
        out["geometry_bf16"] = {"c2": result["c2_geometry_bf16"],
                                "c3": result["c3"]["geometry_bf16"] if "c3" in result else None}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, levels)
    if dist:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


# -------------------------------------------------------------- reference
def run_reference(args):
    """The oracle on the host cores, on the workload of our arm.  Its CG
    iteration count is the oracle's own (GMG-PCG on the same kind of problem
    at twice the coarsest mesh size: the GPU path is never consulted); every step
    times a bounded sample of patch visits on all cores and extrapolates the
    solve's patch work from it (labelled)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2510_17785_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    levels = int(round(math.log2(w.N // w.coarse_N))) + 1
    first = oracle_cpu_sample(w.name, 1, 40, iterations_N=2 * w.coarse_N)
    iters = first["oracle_cg"]["iterations"]
    vals = []
    for i in range(args.warmup + args.steps):
        t = oracle_cpu_sample(w.name, 1, 40, seed=i + 1)
        v = w.n_free / (iters * solve_visits(w, levels) / t["visit_rate"])
        if i >= args.warmup:
            vals.append((v, t))
    v = statistics.mean(x for x, _ in vals)
    t = vals[-1][1]
    ms = w.n_free / v * 1e3
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "DoFs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "dim": w.dim, "cells_per_dir": w.N, "p": w.p, "n_free": w.n_free},
        "cpu_baseline": {"value": v, "unit": "DoFs/s", "cores": t["cores"], "kind": "oracle", "cpu": t["cpu"],
                         "sample": (f"per step: {t['patches']} seeded finest-level patches on {t['cores']} cores, "
                                    f"40 Evaluate + V-cycle visits each; extrapolated (labelled) to {iters} CG "
                                    f"iterations x 2 sweeps x all patches of levels 1..{levels - 1}, patch work only; "
                                    f"the iteration count is the oracle's own GMG-PCG on the same kind of problem "
                                    f"with {first['oracle_cg']['N']} cells per direction (relres "
                                    f"{first['oracle_cg']['relres']:.1e})"),
                         "extrapolated": True},
        "e2e": {"value": v, "unit": "DoFs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


if __name__ == "__main__":
    if len(sys.argv) == 3 and sys.argv[1] == "--cpu-child":
        print(json.dumps(_cpu_child(json.loads(sys.argv[2]))))
        sys.exit(0)
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.sweep_only:
        run_sweep_only(a)
    elif a.batch > 0:
        run_batch(a)
    else:
        run_ours(a)
