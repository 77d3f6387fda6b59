"""Small driver for kernel captures: set up one 3D problem and run a few
finest-level patch sweeps and one operator apply, nothing else.

    python -m paper_2510_17785_gb300.profile_sweep --N 16 --p 4 --precision mixed --sweeps 3

Meant for ``ncu --nvtx --nvtx-include "sweeps/" -k regex:k_patch ...`` (the sweeps
run inside the NVTX range "sweeps", so set-up launches are not captured) on a case far smaller than the
benchmark (a few hundred MB on the device), so that every replay pass of a
full capture saves and restores little memory.
"""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=16)
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--dim", type=int, default=3)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--sweeps", type=int, default=3)
    ap.add_argument("--levels", type=int, default=0, help="h-levels (default: down to 2 cells per direction)")
    ap.add_argument("--variant", type=int, default=-1,
                    help="launch-shape variant without set-up timing (default: time them all and keep the fastest)")
    args = ap.parse_args()
    if args.levels <= 0:                  # halve while the cell count stays even and >= 2
        args.levels, n = 1, args.N
        while n % 2 == 0 and n // 2 >= 2:
            args.levels, n = args.levels + 1, n // 2

    import torch
    from paper_2510_17785_gb300 import inputs, pmg

    w = inputs.Workload(f"prof_{args.dim}d_q{args.p}_n{args.N}", args.dim, args.N, args.p, 0.25, "uniform",
                        ("const", 1.0), "uniform", 77)
    prob = inputs.make_problem(w)
    prec = pmg.PREC_MIXED if args.precision == "mixed" else pmg.PREC_FP64
    tune = dict(autotune=0, variant=args.variant) if args.variant >= 0 else {}
    ctx = pmg.Context(0, precision=prec, **tune)
    ctx.mesh_structured(w.dim, w.N, w.p, args.levels, prob.coords, prob.kappa)
    ctx.setup()
    b = torch.tensor(prob.rhs, device="cuda")
    u = torch.zeros_like(b)
    lf = args.levels - 1
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("sweeps")       # ncu --nvtx --nvtx-include "sweeps/" selects these launches
    for _ in range(args.sweeps):
        ctx.patch_smooth(lf, b, u, 1, False)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    Au = torch.zeros_like(b)
    ctx.apply(lf, u, Au)
    torch.cuda.synchronize()
    print(f"ok: {w.name} sweeps={args.sweeps} tuning={ctx.tuning()} |u|_inf={float(u.abs().max()):.6e}")
    for lv in range(args.levels):
        v, ms = ctx.tuning_level(lv)
        print(f"  level {lv}: variant {v}, ms per variant {[round(x, 4) for x in ms]}")
    ctx.close()


if __name__ == "__main__":
    main()
