"""Writes qtable_diffusion3d_c1.txt: a Q-table trained by the CPU oracle alone.

Algorithm 1 (Section 4.1 update, epsilon-greedy with the Section 5 schedule) run in
sequence on 8 variable-coefficient 3D 7-point diffusion matrices (edge 10..14, log-normal
coefficients with sigma in [0.5, 3]), 200 episodes per matrix (Section 5), T_max = 1000,
tau = 1e-8, cost setting C1, and the true residual confirming a claimed convergence.
Used by bench.py (both arms) as the tabular policy; no GPU output enters it.

    python tests/golden/make_qtable.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2504_14268_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "qtable_diffusion3d_c1.txt")
COUNT, M_LO, M_HI, SEED, EPISODES, TMAX, TAU = 8, 10, 14, 7, 200, 1000, 1e-8


def options():
    return O.Options(seed=1, true_res_at_conv=1)


def main():
    o = options()
    qt = O.QTable.zeros(o)
    sets = I.cfg_train_set(count=COUNT, m_lo=M_LO, m_hi=M_HI, seed=SEED)
    for i, (A, b, _) in enumerate(sets):
        t0 = time.time()
        it = O.train_sequential(o, A, b, TAU, TMAX, EPISODES, qt, ep_base=i * EPISODES)
        print(f"matrix {i}: n={A[0]} mean iters {it.mean():.1f} last {it[-10:]} {time.time() - t0:.1f}s", flush=True)
    with open(OUT, "w") as f:
        f.write("# Q-table written by tests/golden/make_qtable.py (CPU oracle only).\n")
        f.write(f"# b_bins=10 r_bins=10 t_bin=1000 eps_min=1e-16 precs=fp16,bf16,tf32,fp32,fp64 cost=C1 "
                f"tau={TAU} tmax={TMAX} episodes={EPISODES} matrices={COUNT} edge={M_LO}..{M_HI} seed={SEED}\n")
        f.write("# rows: op j (4) x state s (100); columns: Q_j(s, p) for the 5 precisions, then the update count\n")
        for j in range(4):
            for s in range(o.n_states):
                f.write(" ".join(f"{v:.17g}" for v in qt.Q[j, s]) + f" {int(qt.visits[j, s])}\n")
    print("wrote", OUT)


def load(path=OUT):
    rows = np.loadtxt(path, comments="#")
    Q = rows[:, :5].reshape(4, 100, 5).copy()
    visits = rows[:, 5].astype(np.int32).reshape(4, 100).copy()
    return Q, visits


if __name__ == "__main__":
    main()
