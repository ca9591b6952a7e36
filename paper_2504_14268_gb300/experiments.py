"""The paper's experiment protocol (Section 5) on the GPU library.

    python -m paper_2504_14268_gb300.experiments --family synth --cost C1
    python -m paper_2504_14268_gb300.experiments --family poisson --cost C2 --precond 2
    python -m paper_2504_14268_gb300.experiments --family diffusion --cost C1 --train 64 --test 64

Ten training systems, 200 episodes per training system (Algorithm 1, run as batched
rounds: one episode of every training system per round), then the greedy policy
(Algorithm 2) on 100 test systems against fp64 CG with the same preconditioner; stopping at
rho < 1e-6 with k >= 10, or after 1000 iterations, or at a breakdown. Families: `synth`
(Section 5.1, A = B B^T + beta I, n = 5000, test systems with the pair count scaled by
U[0.8, 1.2]), `poisson` (Section 5.2, random subdomains, n = 6400), and `diffusion` (the
variable-coefficient 3D 7-point training family, edge 16..40, log-normal coefficients with sigma
in [0.5, 3]; test systems from another seed; by default tau = 1e-8 and M = I). Reports the
statistics of Tables 2-4: the share of each format over all operations, and the relative
error to the direct solution and the iteration count (mean, standard deviation, maximum,
25th and 75th percentiles) of both solvers. Systems on which the fp32 IC(0) factorization
breaks down are replaced by the next seed (the count is reported).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

COSTS = {"C1": (0.8, 0.6, 0.8, 1.0, 2.0), "C2": (0.5, 0.4, 0.5, 1.5, 3.0)}  # fp16, bf16, tf32, fp32, fp64
NAMES = ("fp16", "bf16", "tf32", "fp32", "fp64")


def _stats(v) -> dict:
    v = np.asarray(v, dtype=np.float64)
    return {"mean": float(v.mean()), "std": float(v.std()), "max": float(v.max()),
            "p25": float(np.percentile(v, 25)), "p75": float(np.percentile(v, 75))}


def format_shares(action_hists) -> dict:
    """Share of each format over every operation of every iteration (Table 2)."""
    tot = np.zeros(5)
    for h in action_hists:
        tot += np.asarray(h)[:, :5].sum(axis=0)
    return {NAMES[f]: float(tot[f] / max(tot.sum(), 1.0)) for f in range(5)}


def _systems(family: str, first_seed: int, count: int, ood: bool, ctx, precond: int, torch, I, M, skipped: list):
    out, seed = [], first_seed
    pool = I.cfg_train_set(count=count + 16, seed=2 if first_seed == 0 else 3) if family == "diffusion" else None
    while len(out) < count:
        xs = None
        if family == "diffusion":
            A, b, xs = pool[seed - first_seed]
        else:
            A, b = I.synth_bbt(seed, ood=ood) if family == "synth" else I.poisson_subdomain(seed)
        seed += 1
        n, rp, ci, val = A
        mat = ctx.matrix((n, torch.as_tensor(rp).cuda(), torch.as_tensor(ci).cuda(), torch.as_tensor(val).cuda()))
        if precond == 2:
            try:
                mat.ic0()
            except M.MpcgError:
                skipped.append(seed - 1)
                mat.close()
                continue
        out.append((A, b, mat, xs))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--family", choices=["synth", "poisson", "diffusion"], default="synth")
    ap.add_argument("--cost", choices=["C1", "C2"], default="C1")
    ap.add_argument("--precond", type=int, default=None,
                    help="0 none, 1 Jacobi, 2 fp32 IC(0) (default: 2, or 0 for the diffusion family)")
    ap.add_argument("--tau", type=float, default=None, help="tolerance (default: 1e-6, or 1e-8 for diffusion)")
    ap.add_argument("--train", type=int, default=10)
    ap.add_argument("--test", type=int, default=100)
    ap.add_argument("--episodes", type=int, default=200)
    ap.add_argument("--on-breakdown", type=int, default=0,
                    help="0: a breakdown ends the solve (the paper); 1: greedy solves restart in fp64")
    ap.add_argument("--out", default=None, help="also write the report (one JSON object) to this file")
    args = ap.parse_args()

    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    import torch

    from paper_2504_14268_gb300 import build
    from paper_2504_14268_gb300 import inputs as I

    build.build()
    from paper_2504_14268_gb300 import mpcg as M

    if args.precond is None:
        args.precond = 0 if args.family == "diffusion" else 2
    tau = args.tau if args.tau is not None else (1e-8 if args.family == "diffusion" else 1e-6)
    t_max = 1000
    opts = M.Options(cost=COSTS[args.cost], precond=args.precond, min_k=10, t_bin=t_max,
                     on_breakdown=args.on_breakdown)
    ctx = M.Context(0, opts)
    skipped: list = []
    t0 = time.time()
    train = _systems(args.family, 0, args.train, False, ctx, args.precond, torch, I, M, skipped)
    test = _systems(args.family, 100000, args.test, args.family == "synth", ctx, args.precond, torch, I, M, skipped)
    t_setup = time.time() - t0

    S = opts.b_bins * opts.r_bins
    pol = ctx.policy_qtable(np.zeros((4, S, 5)), np.zeros((4, S), dtype=np.int32))
    tb = [torch.as_tensor(b).cuda() for _, b, _, _ in train]
    torch.cuda.synchronize()
    t0 = time.time()
    its = ctx.train_qtable([m for _, _, m, _ in train], tb, tau, t_max, args.episodes, pol, want_iters=True)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    its = np.asarray(its, dtype=np.float64)

    mats = [m for _, _, m, _ in test]
    bs = [torch.as_tensor(b).cuda() for _, b, _, _ in test]
    xtrue = []
    for A, b, _, xs in test:
        n, rp, ci, val = A
        xtrue.append(xs if xs is not None else sla.spsolve(sp.csc_matrix(sp.csr_matrix((val, ci, rp), shape=(n, n))), b))
    report = {"family": args.family, "cost": args.cost, "precond": args.precond, "train": args.train,
              "test": args.test, "episodes": args.episodes, "on_breakdown": args.on_breakdown,
              "tau": tau, "skipped_seeds": skipped,
              "setup_s": round(t_setup, 2), "train_s": round(t_train, 2),
              "train_mean_iters_first_last_round": [float(its[0].mean()), float(its[-1].mean())]}
    for label, policy in (("rl", pol), ("fp64", ctx.policy_fixed((4, 4, 4, 4)))):
        xs = [torch.zeros_like(b) for b in bs]
        torch.cuda.synchronize()
        t0 = time.time()
        res = ctx.solve_batched(mats, bs, xs, [tau] * len(mats), [t_max] * len(mats), policy)
        torch.cuda.synchronize()
        dt = time.time() - t0
        err = [float(np.linalg.norm(x.cpu().numpy() - xt) / np.linalg.norm(xt)) for x, xt in zip(xs, xtrue)]
        ok = [r["outcome"] == 0 for r in res]
        report[label] = {"solve_s": round(dt, 3), "rel_err": _stats(err), "iters": _stats([r["iters"] for r in res]),
                         "converged": float(np.mean(ok)),
                         "breakdowns": int(sum(r["outcome"] == 2 for r in res)),
                         "restarts": int(sum(r["n_restarts"] for r in res)),
                         "rel_err_converged": _stats([e for e, c in zip(err, ok) if c]) if any(ok) else None,
                         "format_share": format_shares([r["action_hist"] for r in res])}
    line = json.dumps(report)
    print(line)
    if args.out:
        with open(args.out, "w") as f:
            f.write(line + "\n")


if __name__ == "__main__":
    main()
