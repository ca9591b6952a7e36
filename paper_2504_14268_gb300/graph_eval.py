"""The learned Q-function out of sample: shifted graph Laplacians of power-law graphs.

    python -m paper_2504_14268_gb300.graph_eval --sizes 65536 262144 1048576 4000000

Trains the tabular policy (Algorithm 1, batched rounds on the GPU) on the 32 x 32 Poisson
matrix and four small systems of the 27-point anisotropic FEM family, every operation in
{fp32, fp64}, tau = 1e-8; collects epsilon-greedy trajectories of those systems around the
table and fits the MLP Q-function to them (fitted-Q regression, the library's own forward,
backward and Adam kernels). Then solves L + 1e-4 I of preferential-attachment graphs (m = 6
edges per new node, mean degree 12) to tau = 1e-8 (true residual at convergence, cap 20000)
with all-fp64 CG, the table and the network: iterations, outcome, relative error to x*,
device time of one solve (CUDA events, after one warm-up solve) and mean precision cost per
operation (cost setting C1). One JSON object on stdout (and in --out).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

COST_C1 = (0.8, 0.6, 0.8, 1.0, 2.0)  # fp16, bf16, tf32, fp32, fp64 (Section 5)


def _mean_cost(res) -> float:
    ah = np.asarray(res["action_hist"])[:, :5]
    return float(sum(COST_C1[f] * ah[:, f].sum() for f in range(5)) / max(1, ah.sum()))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", type=int, nargs="+", default=[1 << 16, 1 << 18, 1 << 20, 4_000_000])
    ap.add_argument("--rounds", type=int, default=100, help="batched Algorithm 1 rounds of the table")
    ap.add_argument("--mlp-steps", type=int, default=4000)
    ap.add_argument("--cap", type=int, default=20000)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()

    import torch

    from paper_2504_14268_gb300 import build
    from paper_2504_14268_gb300 import inputs as I

    build.build()
    from paper_2504_14268_gb300 import mpcg as M

    def dev(A):
        n, rp, ci, val = A
        return (n, torch.as_tensor(rp).cuda(), torch.as_tensor(ci).cuda(), torch.as_tensor(val).cuda())

    H, tau = 64, 1e-8
    opts = M.Options(true_res_at_conv=1, on_breakdown=1, op_mask=(0b11000,) * 4, mlp_hidden=H, seed=5)
    ctx = M.Context(0, opts)
    train = [I.cfg_poisson32()[:2]]
    for i, (m, an) in enumerate([(24, 1e-3), (32, 1e-3), (40, 1e-2), (48, 3e-3)]):
        At = I.fem27_aniso(m, an)
        train.append((At, I.rhs_from_xstar(At, np.random.default_rng(100 + i))[1]))
    mats = [ctx.matrix(dev(A)) for A, _ in train]
    bs = [torch.as_tensor(b).cuda() for _, b in train]
    qs, vs = ctx.qtable_shapes()
    tab = ctx.policy_qtable(np.zeros(qs), np.zeros(vs, dtype=np.int32))
    t0 = time.time()
    ctx.train_qtable(mats, bs, tau, 1000, args.rounds, tab)
    data = np.concatenate([ctx.collect(mats, bs, tau, 1000, tab, eps=0.3, episode=1000 + e) for e in range(1, 13)])
    rng = np.random.default_rng(0)
    nparam = M.lib().mpcg_mlp_nparams(H, len(opts.precs))
    mlp = ctx.policy_mlp((rng.standard_normal(nparam) * 0.1).astype(np.float32))
    torch.cuda.synchronize()
    t1 = time.time()
    losses = ctx.mlp_train(mlp, data, steps=args.mlp_steps, batch=1024, lr=1e-3, target_sync=500, seed=3)
    torch.cuda.synchronize()
    t_mlp = time.time() - t1
    report = {"train": {"systems": len(train), "rounds": args.rounds, "transitions": int(len(data)),
                        "mlp_loss_first_last": [float(np.mean(losses[:100])), float(np.mean(losses[-100:]))],
                        "seconds": round(time.time() - t0, 2),
                        "mlp_train": {"steps": args.mlp_steps, "batch": 1024, "seconds": round(t_mlp, 3),
                                      "samples_per_s": round(args.mlp_steps * 1024 / max(t_mlp, 1e-9))}},
              "tau": tau, "cap": args.cap, "graphs": []}
    for n in args.sizes:
        t0 = time.time()
        A = I.ba_laplacian(n, 6, 1e-4, np.random.default_rng(n))
        xs, b = I.rhs_from_xstar(A, np.random.default_rng(n + 1))
        t_gen = time.time() - t0
        mat = ctx.matrix(dev(A))
        mat.autotune(2)
        bd = torch.as_tensor(b).cuda()
        row = {"n": int(n), "nnz": int(A[1][-1]), "max_row": int(np.max(np.diff(A[1]))), "generate_s": round(t_gen, 1)}
        for name, pol in (("fp64", ctx.policy_fixed((4, 4, 4, 4))), ("tabular", tab), ("mlp", mlp)):
            x = torch.zeros_like(bd)
            ctx.solve(mat, bd, x, tau, args.cap, pol)
            x.zero_()
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record()
            res, _ = ctx.solve(mat, bd, x, tau, args.cap, pol)
            ev[1].record()
            torch.cuda.synchronize()
            err = float(np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs))
            row[name] = {"outcome": int(res["outcome"]), "iters": int(res["iters"]), "rel_err": err,
                         "rel_res_true": float(res["rel_res_true"]), "ms": round(ev[0].elapsed_time(ev[1]), 2),
                         "mean_cost": round(_mean_cost(res), 3)}
        report["graphs"].append(row)
        mat.close()
        print(json.dumps(row), flush=True)
    line = json.dumps(report)
    print(line)
    if args.out:
        with open(args.out, "w") as f:
            f.write(line + "\n")


if __name__ == "__main__":
    main()
