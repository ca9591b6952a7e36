"""Benchmark: RL-mixed-precision CG on one GB300 versus all-FP64 CG.

Workload (default): Q1-FEM 27-point anisotropic diffusion on a 256^3 grid (n = 16.8M,
Z = 449M, K = diag(1, 1, 1e-3)), b = A x* with x* ~ U[-1, 1], solved to a true relative
residual of 1e-8. The policy is the paper's tabular Q-learning (Algorithm 1), trained at set-up
on the GPU (batched episodes, one persistent launch per round) on 16 smaller systems of the
same family (24^3 to 48^3, anisotropy 1e-3 to 1e-2), cost setting C1, every operation choosing
from {fp32, fp64} (the formats whose unit roundoff is at most sqrt(tau)), then applied greedily
(Algorithm 2). One step = one complete solve (every row of the hot path: the mixed-precision
SpMV, the fused dot/axpy passes, the fp64 scalars and residual recomputation, the policy)
through the C ABI, inputs resident in HBM. The matrix and its value copies exceed the 129 MB
L2 many times over, so no L2 flush is needed between steps.

Prints one JSON line (see the fields below). `--impl reference` runs the CPU oracle arm on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0
TAU = 1e-8
GRID = 256
ANISO = 1e-3
MAX_ITER = 20000
BYTES = {0: 2, 1: 2, 2: 4, 3: 4, 4: 8, 5: 2, 6: 2}
# policy training: formats with u <= sqrt(tau) for every operation (fp32, fp64), iteration
# bins over the training horizon T_max = 5000 (so the state is in effect the residual bin),
# 16 systems of the workload's family, 150 rounds of batched episodes
OP_MASK = (0b11000,) * 4
T_BIN = 5000
TRAIN_SET = [(24, 1e-3), (28, 1e-3), (32, 1e-3), (36, 1e-3), (40, 1e-3), (44, 1e-3), (48, 1e-3), (32, 1e-2),
             (40, 1e-2), (48, 3e-3), (30, 3e-3), (36, 1e-2), (26, 1e-3), (34, 3e-3), (42, 1e-3), (46, 1e-2)]
TRAIN_ROUNDS = 150
TRAIN_SEED = 3


def solver_options(M):
    return M.Options(true_res_at_conv=1, on_breakdown=1, op_mask=OP_MASK, t_bin=T_BIN, seed=TRAIN_SEED)


def train_policy(M, ctx):
    """Algorithm 1, batched on the GPU, on the training family. Returns (policy, seconds,
    mean iterations of the first and last three rounds)."""
    import torch

    from paper_2504_14268_gb300 import inputs as I

    mats, bs = [], []
    for i, (m, an) in enumerate(TRAIN_SET):
        At = I.fem27_aniso(m, an)
        _, bt = I.rhs_from_xstar(At, np.random.default_rng(100 + i))
        mats.append(ctx.matrix((At[0], torch.as_tensor(At[1]).cuda(), torch.as_tensor(At[2]).cuda(),
                                torch.as_tensor(At[3]).cuda())))
        bs.append(torch.as_tensor(bt).cuda())
    nprec = 5
    pol = ctx.policy_qtable(np.zeros((4, 100, nprec)), np.zeros((4, 100), dtype=np.int32))
    torch.cuda.synchronize()
    t0 = time.time()
    its = ctx.train_qtable(mats, bs, TAU, T_BIN, TRAIN_ROUNDS, pol, want_iters=True)
    torch.cuda.synchronize()
    dt = time.time() - t0
    for m in mats:
        m.close()
    return pol, dt, (float(its[:3].mean()), float(its[-3:].mean()))


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_cg_persistent_fem27_256.md")


def sources_sha256() -> str:
    """Hash of the kernel sources and the C header (the build the ncu counters belong to)."""
    import glob
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2504_14268_gb300", "csrc")
    for f in sorted(glob.glob(os.path.join(csrc, "*"))) + [os.path.join(ROOT, "include", "mpcg.h")]:
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode())
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic():
    """DRAM bytes per launch of the solver kernel on this workload from the committed ncu
    summary, or None when that summary was taken on other kernel sources."""
    try:
        vals = {}
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if ":" in line and line.strip().startswith(("traffic_bytes_per_launch", "sources_sha256")):
                    k, v = line.strip().split(":", 1)
                    vals[k.strip()] = v.strip().strip("`")
        if vals.get("sources_sha256") == sources_sha256():
            return float(vals["traffic_bytes_per_launch"])
    except Exception:
        pass
    return None


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


def workload(grid: int):
    from paper_2504_14268_gb300 import inputs as I

    A = I.fem27_aniso(grid, ANISO)
    xs, b = I.rhs_from_xstar(A, np.random.default_rng(0))
    return A, b, xs


def load_policy():
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    from make_qtable import load

    return load()


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([s.strip() for s in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, nm in enumerate(names):
                if len(s) > 5 + k and s[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def iter_bytes(n: int, Z: int, fmt: tuple, flags: int, next_p1: int) -> float:
    """Algorithmic HBM bytes of one iteration of the persistent kernel (each array touched
    once): phase A reads the p1 value copy and the columns (Z (v + 4)), row_ptr (4n), p once
    in its p1 copy (n v) and in fp64 for nu (8n, shared with the gather when p1 = fp64), and
    writes q (n v); phase B reads q (plus the fp32 row scale for row-scaled formats) and r,
    writes r; phase C reads p, x, r and writes x, p and p's copy in the next format; a
    residual recomputation reads the fp64 values, columns, row_ptr, x, b and writes r."""
    p1 = fmt[0]
    v = BYTES[p1]
    a = Z * (v + 4) + 4 * (n + 1) + n * v + (0 if p1 == 4 else 8 * n) + n * v
    bb = n * v + (4 * n if p1 in (5, 6) else 0) + 16 * n
    c = 48 * n + (0 if next_p1 == 4 else BYTES[next_p1] * n)
    t = (Z * 12 + 4 * (n + 1) + 24 * n) if flags & 4 else 0
    return a + bb + c + t


def launch_bytes(n: int, Z: int, hist) -> float:
    """Bytes of one persistent launch: initialisation (b read, x, r, p written), every
    iteration of the history, and the closing fp64 residual."""
    total = 8 * n + 24 * n
    for k in range(len(hist)):
        nxt = int(hist["fmt"][k + 1][0]) if k + 1 < len(hist) else 4
        total += iter_bytes(n, Z, tuple(int(f) for f in hist["fmt"][k]), int(hist["flags"][k]), nxt)
    total += Z * 12 + 4 * (n + 1) + 16 * n
    return total


def cpu_sample(A, b, Q, visits, gpu_iters: int, budget_s: float = 15.0):
    """The oracle, as it stands, on the first iterations of the same solve. Returns
    (solves/s extrapolated to the GPU's iteration count, iterations sampled, seconds)."""
    import oracle as O

    o = O.Options(true_res_at_conv=1, on_breakdown=1, op_mask=OP_MASK, t_bin=T_BIN)
    qt = O.QTable(Q.copy(), visits.copy())
    t0 = time.time()
    O.solve(o, A, b, TAU, 1, qtable=qt)
    t1 = time.time() - t0
    its = max(1, min(50, int(budget_s / max(t1, 1e-3))))
    t0 = time.time()
    out = O.solve(o, A, b, TAU, its, qtable=qt)
    dt = time.time() - t0
    per_it = dt / max(1, len(out.hist))
    return 1.0 / (per_it * max(gpu_iters, 1)), len(out.hist), dt


def run_reference(args):
    """CPU oracle arm: each step is a bounded sample of the workload's solve."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    A, b, xs = workload(args.grid)
    Q, visits = load_policy()
    # iterations of the full solve are taken from the oracle's own fp64 convergence bound
    # (square root of the closed-form condition number), not from the GPU
    from paper_2504_14268_gb300 import inputs as I

    lo, hi = I.fem27_spectrum(args.grid, ANISO)
    est_iters = int(math.ceil(0.5 * math.sqrt(hi / lo) * math.log(2 / TAU)))
    for _ in range(args.warmup):
        cpu_sample(A, b, Q, visits, est_iters, budget_s=2.0)
    vals = []
    t0 = time.time()
    for _ in range(args.steps):
        v, its, dt = cpu_sample(A, b, Q, visits, est_iters, budget_s=args.ref_budget)
        vals.append(v)
    T = time.time() - t0
    value = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": "solves/s to true relative residual 1e-8 (RL-mixed CG)",
        "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+mixed", "data": "synthetic",
        "config": {"workload": f"fem27_aniso_{args.grid}^3 (n={A[0]}, nnz={len(A[3])}), tau=1e-8, tabular policy"},
        "cpu_baseline": {"kind": "oracle", "value": value, "unit": "solves/s", "cores": 1,
                         "sample": f"first iterations of the solve per step (about {args.ref_budget:.0f} s of "
                                   f"single-thread oracle time), extrapolated to {est_iters} iterations"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def max_over_ranks(t_local: float, dist, device) -> float:
    """The job's time: the slowest rank's (every rank solves its own replica)."""
    if dist is None:
        return t_local
    import torch

    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, steps: int, t_job: float) -> float:
    """Solves per second of the whole job: every rank's solves over the slowest rank's time."""
    return world * steps / t_job


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=GRID)
    ap.add_argument("--ref-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2504_14268_gb300 import mpcg as M

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()

    t_gen = time.time()
    A, b, xs = workload(args.grid)
    n, rp, ci, val = A
    Z = len(val)
    t_gen = time.time() - t_gen
    ctx = M.Context(local, solver_options(M))
    pol, t_train, train_its = train_policy(M, ctx)
    t0 = time.time()
    mat = ctx.matrix((n, torch.as_tensor(rp).cuda(), torch.as_tensor(ci).cuda(), torch.as_tensor(val).cuda()))
    torch.cuda.synchronize()
    t_setup = time.time() - t0
    t0 = time.time()
    mat.autotune(5)
    t_tune = time.time() - t0
    pol64 = ctx.policy_fixed((4, 4, 4, 4))
    bd = torch.as_tensor(b).cuda()
    x = torch.zeros_like(bd)
    hist = np.zeros(MAX_ITER, dtype=M.REC_DTYPE)

    for _ in range(args.warmup):
        res, _ = ctx.solve(mat, bd, x, TAU, MAX_ITER, pol, stream=stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    results = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for s in range(args.steps):
            ev[s][0].record(stream)
            res, h = ctx.solve(mat, bd, x, TAU, MAX_ITER, pol, history=hist if s == 0 else None, stream=stream)
            ev[s][1].record(stream)
            results.append(res)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(c) for a, c in ev]
    T = max_over_ranks(sum(step_ms) / 1e3, dist, "cuda")
    r0 = results[0]
    h0 = hist[: r0["iters"] + 1][: len(hist)]
    h0 = hist[: min(MAX_ITER, max(1, r0["iters"]))]
    xerr = float(np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs))

    # all-FP64 CG on the same GPU (same kernel, every operation in fp64)
    x64 = torch.zeros_like(bd)
    res64, _ = ctx.solve(mat, bd, x64, TAU, MAX_ITER, pol64, stream=stream)
    e64 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e64[0].record(stream)
    res64, _ = ctx.solve(mat, bd, x64, TAU, MAX_ITER, pol64, stream=stream)
    e64[1].record(stream)
    torch.cuda.synchronize()
    t64 = e64[0].elapsed_time(e64[1]) / 1e3
    xerr64 = float(np.linalg.norm(x64.cpu().numpy() - xs) / np.linalg.norm(xs))

    # SpMV bandwidth per value format (standalone product, autotuned schedule)
    hbm, peak_kind = peaks()
    xr = torch.rand(n, dtype=torch.float64, device="cuda")
    yr = torch.empty_like(xr)
    spmv = {}
    for fmt, name in enumerate(M.FORMAT_NAMES):
        ms = ctx.spmv(mat, fmt, xr, yr, reps=10, stream=stream)
        v = BYTES[fmt]
        byts = Z * (v + 4) + 4 * (n + 1) + 2 * n * v + (4 * n if fmt in (5, 6) else 0)
        spmv[name] = {"ms": round(ms, 4), "gbs": round(byts / ms / 1e6, 1), "frac": round(byts / ms / 1e6 / hbm, 3)}

    # roofline of the persistent kernel (the only kernel of a step)
    lb = launch_bytes(n, Z, h0)
    achieved = lb / (statistics.mean(step_ms) / 1e3) / 1e9

    # end to end through the C ABI with pinned host buffers (H2D of b, D2H of x inside)
    bh = torch.as_tensor(b).pin_memory()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()
    ctx.solve(mat, bh, xh, TAU, MAX_ITER, pol, stream=stream)
    ee = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ee[0].record(stream)
    for _ in range(args.steps):
        ctx.solve(mat, bh, xh, TAU, MAX_ITER, pol, stream=stream)
    ee[1].record(stream)
    torch.cuda.synchronize()
    e2e_T = ee[0].elapsed_time(ee[1]) / 1e3

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        Q, visits = load_policy()
        v, its, dt = cpu_sample(A, b, Q, visits, r0["iters"])
        cpu = {"kind": "oracle", "value": v, "unit": "solves/s", "cores": 1,
               "sample": f"first {its} iterations of the same solve ({dt:.1f} s single-thread; policy: the "
                         f"oracle-trained table tests/golden/qtable_diffusion3d_c1.txt under the same operation "
                         f"sets), extrapolated to the GPU's {r0['iters']} iterations"}

    if rank == 0:
        ah = np.array(r0["action_hist"])[:, :7]
        line = {
            "metric": "solves/s to true relative residual 1e-8 (RL-mixed CG), with time vs all-FP64 CG and SpMV % HBM",
            "value": whole_job_rate(world, args.steps, T), "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+mixed", "data": "synthetic",
            "config": {"workload": f"fem27_aniso_{args.grid}^3", "n": n, "nnz": Z, "anisotropy": ANISO, "tau": TAU,
                       "policy": f"tabular Q (Algorithm 1) trained on the GPU at set-up: {len(TRAIN_SET)} systems "
                                 f"24^3-48^3 of the same family, {TRAIN_ROUNDS} batched rounds, cost C1, every "
                                 f"operation in {{fp32, fp64}}, T_max {T_BIN}; greedy (Algorithm 2)",
                       "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas" if world > 1 else "1 GPU"},
            "time_to_tol_s": 1e-3 * statistics.mean(step_ms), "iters": r0["iters"], "outcome": r0["outcome"],
            "rel_res_true": r0["rel_res_true"], "rel_err_xstar": xerr,
            "fp64": {"time_to_tol_s": t64, "iters": res64["iters"], "rel_res_true": res64["rel_res_true"],
                     "rel_err_xstar": xerr64},
            "speedup_vs_fp64": t64 / (1e-3 * statistics.mean(step_ms)),
            "action_mix": {M.FORMAT_NAMES[f]: int(ah[:, f].sum()) for f in range(7)},
            "spmv": spmv,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(achieved / hbm, 3), "traffic": measured_traffic(), "peak_source": peak_kind,
                         "kernel": "cg_persistent", "bytes_per_launch": lb, "sources_sha256": sources_sha256()},
            "e2e": {"value": args.steps / e2e_T, "unit": "solves/s", "h2d_bytes_per_step": 8 * n,
                    "d2h_bytes_per_step": 8 * n + 288},
            "cpu_baseline": cpu,
            "gpu_launches": args.steps,
            "clocks": clk.summary(),
            "setup_s": {"generate": round(t_gen, 1), "matrix_create": round(t_setup, 2), "autotune": round(t_tune, 2),
                        "train_policy": round(t_train, 2)},
            "training": {"rounds": TRAIN_ROUNDS, "systems": len(TRAIN_SET),
                         "mean_iters_first_last": [round(train_its[0], 1), round(train_its[1], 1)]},
        }
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
