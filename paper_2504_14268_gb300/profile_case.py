"""One small, deterministic launch of a library kernel, for a profiler to capture.

    python -m paper_2504_14268_gb300.profile_case solve --grid 128 --fmt 3,4,4,4 --iters 20
    python -m paper_2504_14268_gb300.profile_case spmv --grid 128 --fmt 0 --sched 2 --lanes 1

`solve`: a fixed-format solve of the Q1-FEM 27-point anisotropic matrix on grid^3 (the
bench's matrix family) for exactly `--iters` iterations (tolerance 1e-30), one launch of the
persistent kernel, autotuned product schedules; `--precond 2` runs the IC(0)
instantiation (the factor is computed before the solve). `spmv`: one product of the same matrix in
the given value format with the given schedule (two launches of the product kernel: a
warm-up and a timed one; no other launch of that kernel).
Prints the launch's iteration count and per-phase times (solve) or milliseconds (spmv).
"""
from __future__ import annotations

import argparse

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["solve", "spmv"])
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--aniso", type=float, default=1e-3)
    ap.add_argument("--fmt", default="3,4,4,4")
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--sched", type=int, default=2)
    ap.add_argument("--lanes", type=int, default=1)
    ap.add_argument("--precond", type=int, default=0, help="solve: 0 none, 1 Jacobi, 2 fp32 IC(0)")
    args = ap.parse_args()

    import torch

    from paper_2504_14268_gb300 import build
    from paper_2504_14268_gb300 import inputs as I

    build.build()
    from paper_2504_14268_gb300 import mpcg as M

    A = I.fem27_aniso(args.grid, args.aniso)
    n, rp, ci, val = A
    ctx = M.Context(0, M.Options(min_k=0, precond=args.precond if args.what == "solve" else 0))
    mat = ctx.matrix((n, torch.as_tensor(rp).cuda(), torch.as_tensor(ci).cuda(), torch.as_tensor(val).cuda()))
    fm = tuple(int(v) for v in args.fmt.split(","))
    b = torch.as_tensor(I.rhs_from_xstar(A, np.random.default_rng(0))[1]).cuda()
    if args.what == "solve":
        mat.autotune(3)
        if args.precond == 2:
            mat.ic0()
        pol = ctx.policy_fixed(fm if len(fm) == 4 else fm * 4)
        x = torch.zeros_like(b)
        res, h = ctx.solve(mat, b, x, 1e-30, args.iters, pol, history_cap=args.iters + 1)
        k = res["iters"]
        print(f"iterations {k}; mean phase times A {h['ns_a'][:k].mean() / 1e3:.1f} B {h['ns_b'][:k].mean() / 1e3:.1f} "
              f"C {h['ns_c'][:k].mean() / 1e3:.1f} us; schedules {mat.info()['spmv_sched']}")
    else:
        mat.set_schedule(fm[0], args.sched, args.lanes)
        y = torch.empty_like(b)
        ms = ctx.spmv(mat, fm[0], b, y, reps=1)
        print(f"product format {fm[0]}: {ms:.3f} ms; schedule {mat.info()['spmv_sched'][fm[0]]} "
              f"lanes {mat.info()['spmv_lanes'][fm[0]]}")


if __name__ == "__main__":
    main()
