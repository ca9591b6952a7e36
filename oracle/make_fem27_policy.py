"""Writes oracle/policy_fem27_c1.txt with the CPU oracle alone (test infrastructure).

1. A Q-table trained by Algorithm 1 (Section 4.1 update, epsilon-greedy with the Section 5
   schedule), in sequence on eight small systems of the Q1-FEM 27-point anisotropic family
   (edges 10..20, anisotropy 1e-3 .. 1e-2), 40 episodes each, tau = 1e-8, cost setting C1,
   every operation choosing from {fp32, fp64}, iteration bins over T_max = 5000, the true
   residual confirming a claimed convergence -- the options of the single-large-solve
   benchmark.
2. The oracle's own iteration counts on the benchmark's workload (grid^3, anisotropy 1e-3,
   b = A x* with x* ~ U[-1, 1] from seed 0, tau = 1e-8): the greedy solve with that table
   (Algorithm 2) and plain fp64 CG. The CPU arms of bench.py time a bounded number of
   iterations and extrapolate to these counts, so both arms share one basis.

    python oracle/make_fem27_policy.py [--grid 256] [--table-only]

No GPU output enters the file.
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

OUT = os.path.join(HERE, "policy_fem27_c1.txt")
TRAIN = [(10, 1e-3), (12, 1e-3), (14, 1e-2), (16, 1e-3), (18, 3e-3), (20, 1e-3), (16, 1e-2), (12, 3e-3)]
EPISODES, T_BIN, TAU, MASK, SEED = 40, 5000, 1e-8, (0b11000,) * 4, 3


def options():
    import oracle as O

    return O.Options(t_bin=T_BIN, op_mask=MASK, true_res_at_conv=1, on_breakdown=1, seed=SEED)


def train():
    import oracle as O
    from paper_2504_14268_gb300 import inputs as I

    o = options()
    qt = O.QTable.zeros(o)
    for i, (m, an) in enumerate(TRAIN):
        A = I.fem27_aniso(m, an)
        _, b = I.rhs_from_xstar(A, np.random.default_rng(100 + i))
        it = O.train_sequential(o, A, b, TAU, T_BIN, EPISODES, qt, ep_base=i * EPISODES)
        print(f"train {m}^3 aniso {an}: mean iterations {it.mean():.1f}, last {list(it[-5:])}", flush=True)
    return qt


def _solve(args):
    kind, grid, Q, visits = args
    import oracle as O
    from paper_2504_14268_gb300 import inputs as I

    A = I.fem27_aniso(grid, 1e-3)
    _, b = I.rhs_from_xstar(A, np.random.default_rng(0))
    o = options()
    t0 = time.time()
    if kind == "rl":
        out = O.solve(o, A, b, TAU, 20000, qtable=O.QTable(Q, visits))
    else:
        out = O.solve(o, A, b, TAU, 20000, fixed=(4, 4, 4, 4))
    return kind, out.iters, out.outcome, out.rho_true, time.time() - t0


def write(qt, counts):
    o = options()
    with open(OUT, "w") as f:
        f.write("# Q-table and iteration counts written by oracle/make_fem27_policy.py (CPU oracle only).\n")
        f.write(f"# options: b_bins=10 r_bins=10 t_bin={T_BIN} eps_min=1e-16 precs=fp16,bf16,tf32,fp32,fp64 cost=C1 "
                f"op_mask=fp32,fp64 (every operation) true_res_at_conv=1 tau={TAU}\n")
        f.write(f"# training: Algorithm 1 in sequence, {EPISODES} episodes per system, systems (edge, anisotropy) "
                f"{TRAIN}\n")
        for key, val in counts.items():
            f.write(f"# {key}: {val}\n")
        f.write("# rows: op j (4) x state s (100); columns: Q_j(s, p) for the 5 precisions, then the update count\n")
        for j in range(4):
            for s in range(o.n_states):
                f.write(" ".join(f"{v:.17g}" for v in qt.Q[j, s]) + f" {int(qt.visits[j, s])}\n")
    print("wrote", OUT)


def load(path: str = OUT):
    """(Q [4][100][5], visits [4][100], {key: value} of the header's counts)."""
    counts = {}
    with open(path) as f:
        for line in f:
            if line.startswith("# iters_") or line.startswith("# outcome_") or line.startswith("# rho_true_"):
                k, v = line[2:].split(":", 1)
                counts[k.strip()] = float(v)
    rows = np.loadtxt(path, comments="#")
    Q = rows[:, :5].reshape(4, 100, 5).copy()
    visits = rows[:, 5].astype(np.int32).reshape(4, 100).copy()
    return Q, visits, counts


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=256)
    ap.add_argument("--table-only", action="store_true")
    args = ap.parse_args()
    qt = train()
    counts = {}
    if not args.table_only:
        ctx = mp.get_context("spawn")
        with ctx.Pool(2) as pool:
            for kind, it, outc, rt, dt in pool.map(_solve, [(k, args.grid, qt.Q, qt.visits) for k in ("rl", "fp64")]):
                counts[f"iters_{kind}_{args.grid}"] = it
                counts[f"outcome_{kind}_{args.grid}"] = outc
                counts[f"rho_true_{kind}_{args.grid}"] = rt
                print(f"{kind} solve on {args.grid}^3: {it} iterations, outcome {outc}, true residual {rt:.3g}, "
                      f"{dt:.0f} s", flush=True)
    write(qt, counts)


if __name__ == "__main__":
    main()
