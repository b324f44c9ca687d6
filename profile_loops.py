"""Run selected loops of the library repeatedly on a lattice (for profilers).

    python profile_loops.py --n 60 --loops flux2,adjoint --reps 3

Builds the n^3 lattice with RCM numbering, autotunes every loop once, then
runs each requested loop `reps` times with a device synchronisation after
each repetition, and prints one line per loop with its mean time (CUDA
events).  Loops: gg, flux2, gg32, flux2_32, adjoint (flux adjoint +
scaling adjoint + Green-Gauss adjoint), stage (the FP64 RK stage), stage32
(the FP32-mixed stage of separate loops), fused (the fused FP32-mixed stage,
op2b_stage_mixed), visc and
visc32 (viscous node pass + edge loop, FP64 / FP32; not with adjoint),
gg_ff, flux2_ff and ffstage (the float-float Green-Gauss + scaling, flux,
and RK stage), adjoint_ff (the float-float flux adjoint with the FP64
scaling and Green-Gauss adjoints), jacobi (the factored block-Jacobi blocks
and their inverses).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=60)
    ap.add_argument("--loops", default="flux2")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--tune-cache", default="")
    ap.add_argument("--numbering", default="rcm", choices=["rcm", "rcb", "random", "none"])
    ap.add_argument("--force", action="append", default=[],
                    help="fix a strategy instead of tuning: loop:prec:strategy:block:part:staged "
                         "(loop and strategy as numbers of include/op2b.h)")
    args = ap.parse_args()
    import torch
    from paper_1403_7209_gb300 import meshgen, op2b as L
    from paper_1403_7209_gb300.solver import EdgeSolver
    L.load(build_if_missing=False)
    m = meshgen.lattice(args.n)
    q = meshgen.flow_state(m)
    names = args.loops.split(",")
    visc = any(nm.startswith("visc") for nm in names)
    s = EdgeSolver(m.edge, m.normal, m.dx, m.volume, q, renumber=args.numbering, mixed=True,
                   coords=m.coords,
                   adjoint=not visc, viscous=(1e-3, 0.72, 1e-3) if visc else None,
                   ff=not visc, precond="jacobi" in names)
    if args.tune_cache and os.path.exists(args.tune_cache):
        L.op2b_load_tuning(s.ctx, args.tune_cache)
    for loop in range(L.NUM_LOOPS):
        for prec in range(L.NUM_PREC):
            s.set_strategy(loop, prec, L.STRAT_AUTO)
    for f in args.force:
        s.set_strategy(*[int(x) for x in f.split(":")])
    s.time_step(0.5)
    L.op2b_dat_copy(s.ctx, s.d["q0"], s.d["q"])
    if not visc:
        s.t["lam"].normal_()
    run = {
        "gg": lambda: s.green_gauss(),
        "flux2": lambda: s.flux(2),
        "gg32": lambda: s.green_gauss(mixed=True),
        "flux2_32": lambda: s.flux(2, mixed=True),
        "adjoint": lambda: s.adjoint(2, recompute_gradient=False),
        "adjoint_ff": lambda: s.adjoint(2, recompute_gradient=False, ff=True),
        "jacobi": lambda: s.precondition(),
        "stage": lambda: s.stage(0.25),
        "visc": lambda: s.viscous_flux(zero=True),
        "visc32": lambda: s.viscous_flux(mixed=True, zero=True),
        "gg_ff": lambda: s.green_gauss(ff=True),
        "flux2_ff": lambda: s.flux(2, ff=True),
        "ffstage": lambda: s.stage(0.25, ff=True),
        "stage32": lambda: s.stage(0.25, mixed=True),
        "fused": lambda: s.stage_fused(0.25, residual=False),
        "fused_staged": lambda: s.stage_fused(0.25, residual=False, staged=True),
    }
    if visc:
        s.green_gauss()
        s.sync_shadow()
        s.green_gauss(mixed=True)
    if "fused" in names:
        s.stage_fused(0.25, sync=True, residual=False)
    for nm in names:  # warm-up: tunes and builds plans
        run[nm]()
    torch.cuda.synchronize()
    if args.tune_cache:
        L.op2b_save_tuning(s.ctx, args.tune_cache)
    out = {}
    for nm in names:
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ms = 0.0
        for _ in range(args.reps):
            ev[0].record()
            run[nm]()
            ev[1].record()
            torch.cuda.synchronize()
            ms += ev[0].elapsed_time(ev[1])
        out[nm] = ms / args.reps
    print(json.dumps({"n": args.n, "edges": m.num_edges, "ms": out}))
    s.close()


if __name__ == "__main__":
    main()
