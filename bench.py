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

Besides the timed solve the line reports: all-FP64 CG on the same GPU, the standalone SpMV
bandwidth per value format, the roofline of the solver kernel, the end-to-end rate with host
buffers, a policy allowed every format of the paper's precision set, the 512-system uneven
batch under a CUDA graph, and the CPU oracle's rates (one core and all cores).

Prints one JSON line. `--impl reference` runs the CPU oracle arm (all host cores) on bounded
samples of the same workload instead. Sections of the run carry NVTX ranges (solve_rl,
solve_fp64, spmv_<format>, batch_<policy>) so that a profiler can select one launch.
"""
from __future__ import annotations

import argparse
import contextlib
import json
import math
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-8 residual & solves/s: RL-mixed vs FP64 CG; SpMV % HBM peak"
UNIT = "solves/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM = 6800.0
TAU = 1e-8
GRID = 256
ANISO = 1e-3
MAX_ITER = 20000
BYTES = {0: 2, 1: 2, 2: 4, 3: 4, 4: 8, 5: 2, 6: 2, 7: 1}
# policy training: formats with u <= sqrt(tau) for every operation (fp32, fp64), iteration
# bins over the training horizon T_max = 5000 (so the state is in effect the residual bin),
# 16 systems of the workload's family, 150 rounds of batched episodes
OP_MASK = (0b11000,) * 4
T_BIN = 5000
TRAIN_SET = [(24, 1e-3), (28, 1e-3), (32, 1e-3), (36, 1e-3), (40, 1e-3), (44, 1e-3), (48, 1e-3), (32, 1e-2),
             (40, 1e-2), (48, 3e-3), (30, 3e-3), (36, 1e-2), (26, 1e-3), (34, 3e-3), (42, 1e-3), (46, 1e-2)]
TRAIN_ROUNDS = 150
TRAIN_SEED = 3
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_solve_fem27_128.md")


@contextlib.contextmanager
def nvtx(name: str):
    import torch

    torch.cuda.nvtx.range_push(name)
    try:
        yield
    finally:
        torch.cuda.nvtx.range_pop()


STEPPED = 0  # single solves: automatic (the stepped graph at this size); --stepped overrides


def solver_options(M, op_mask=OP_MASK):
    return M.Options(true_res_at_conv=1, on_breakdown=1, op_mask=op_mask, t_bin=T_BIN, seed=TRAIN_SEED,
                     stepped=STEPPED)


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


def traffic_ratio():
    """DRAM bytes per algorithmic byte of the solver kernel, from the committed ncu summary of a
    small case of the same family (the ratio does not depend on the grid: both grow with the
    iterations times the bytes per iteration); None when that summary was taken on other
    kernel sources."""
    try:
        vals = {}
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if ":" in line and line.strip().startswith(("traffic_per_algorithmic_byte", "sources_sha256")):
                    k, v = line.strip().split(":", 1)
                    vals[k.strip()] = v.strip().strip("`")
        if vals.get("sources_sha256") == sources_sha256():
            return float(vals["traffic_per_algorithmic_byte"])
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
    """Algorithmic HBM bytes of one iteration of the solver (each array touched once): phase A
    reads the p1 value copy and the columns (Z (v + 4)), row_ptr (4n), p once in its p1 copy
    (n v) and in fp64 for nu (8n; none when p1 = fp64 or when nu's format is p1's, whose
    rounding of p is the low copy itself), and writes q (n v); phase B reads q (plus the fp32 row scale for row-scaled formats) and r,
    writes r; phase C reads p, x, r and writes x, p and p's copy in the next format; a
    residual recomputation reads the fp64 values, columns, row_ptr, x, b and writes r."""
    p1, p3 = fmt[0], fmt[2]
    v = BYTES[p1]
    base = {5: 1, 6: 0}
    # nu reads p in fp64 unless the product is fp64 (the gather reads it) or nu's format is the
    # product's (then fl_p3(p) is p's low copy, which the gather reads)
    nu_from_low = p3 != 4 and base.get(p3, p3) == base.get(p1, p1) and p1 not in (5, 6)
    a = Z * (v + 4) + 4 * (n + 1) + n * v + (0 if p1 == 4 or nu_from_low else 8 * n) + n * v
    bb = n * v + (4 * n if p1 in (5, 6) else 0) + 16 * n
    c = 48 * n + (0 if next_p1 == 4 else BYTES[next_p1] * n)
    t = (Z * 12 + 4 * (n + 1) + 24 * n) if flags & 4 else 0
    return a + bb + c + t


def product_bytes(n: int, Z: int, fmt: tuple) -> float:
    """Algorithmic bytes of phase A alone (the product kernel): values and columns, row_ptr,
    p's low copy, p in fp64 for nu when needed, q written."""
    p1, p3 = fmt[0], fmt[2]
    v = BYTES[p1]
    base = {5: 1, 6: 0}
    nu_from_low = p3 != 4 and base.get(p3, p3) == base.get(p1, p1) and p1 not in (5, 6)
    return Z * (v + 4) + 4 * (n + 1) + n * v + (0 if p1 == 4 or nu_from_low else 8 * n) + n * v


def launch_bytes(n: int, Z: int, hist) -> float:
    """Bytes of one persistent launch: initialisation (b read, x, r, p written), every
    iteration of the history, and the closing fp64 residual."""
    total = 8 * n + 24 * n
    for k in range(len(hist)):
        nxt = int(hist["fmt"][k + 1][0]) if k + 1 < len(hist) else 4
        total += iter_bytes(n, Z, tuple(int(f) for f in hist["fmt"][k]), int(hist["flags"][k]), nxt)
    total += Z * 12 + 4 * (n + 1) + 16 * n
    return total


# ---------------------------------------------------------------------------------------
# CPU oracle (the cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------------------

def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_policy(grid: int):
    """The oracle-trained Q-table of the benchmark's options and the oracle's own iteration
    counts on this workload (oracle/policy_fem27_c1.txt, written by the oracle alone), or a
    closed-form CG bound when the file has no count for this grid."""
    from oracle import make_fem27_policy as P
    from paper_2504_14268_gb300 import inputs as I

    Q, visits, counts = P.load()
    lo, hi = I.fem27_spectrum(grid, ANISO)
    bound = int(math.ceil(0.5 * math.sqrt(hi / lo) * math.log(2 / TAU)))
    basis = {}
    for kind in ("rl", "fp64"):
        key = f"iters_{kind}_{grid}"
        if key in counts:
            basis[kind] = (int(counts[key]), f"the oracle's own {kind} solve of this workload ({int(counts[key])} "
                                             f"iterations, oracle/policy_fem27_c1.txt)")
        else:
            basis[kind] = (bound, f"the closed-form CG bound 0.5 sqrt(kappa) ln(2/tau) = {bound} iterations")
    return Q, visits, basis


def _oracle_options():
    import oracle as O

    return O.Options(true_res_at_conv=1, on_breakdown=1, op_mask=OP_MASK, t_bin=T_BIN)


def _oracle_iters(A, b, kind, Q, visits, k):
    """k iterations of the oracle's solve from x_0 = 0 (RL-mixed with the table, or fp64)."""
    import oracle as O

    o = _oracle_options()
    if kind == "rl":
        out = O.solve(o, A, b, TAU, k, qtable=O.QTable(Q.copy(), visits.copy()))
    else:
        out = O.solve(o, A, b, TAU, k, fixed=(4, 4, 4, 4))
    return len(out.hist) if k > 0 else 0


def _timed_iters(A, b, kind, Q, visits, k):
    """(seconds of a solve with no iteration -- the initial and closing fp64 residuals --,
    seconds of a solve with k iterations, iterations done)."""
    t0 = time.time()
    _oracle_iters(A, b, kind, Q, visits, 0)
    t1 = time.time()
    done = _oracle_iters(A, b, kind, Q, visits, k)
    return t1 - t0, time.time() - t1, done


def _oracle_worker(args):
    """Spawned worker: maps the staged workload and times k oracle iterations."""
    d, kind, k = args
    A = (int(np.load(os.path.join(d, "n.npy"))[0]), np.load(os.path.join(d, "rp.npy"), mmap_mode="r"),
         np.load(os.path.join(d, "ci.npy"), mmap_mode="r"), np.load(os.path.join(d, "val.npy"), mmap_mode="r"))
    b = np.load(os.path.join(d, "b.npy"), mmap_mode="r")
    Q = np.load(os.path.join(d, "Q.npy"))
    visits = np.load(os.path.join(d, "visits.npy"))
    return _timed_iters(A, b, kind, Q, visits, k)


class OracleBench:
    """Times the oracle, as it stands, on bounded samples of the workload: in this process
    (one core) or as one process per host core, each running the same sample concurrently
    (the whole CPU's throughput; the workload is staged once in files that the processes
    map). A sample's iteration time is the time of k iterations minus that of a solve with
    none (the initial and closing fp64 residuals, which a solve pays once). Rates are
    solves/s: iterations per second over the basis iteration count."""

    def __init__(self, A, b, Q, visits):
        self.A, self.b, self.Q, self.visits = A, b, Q, visits
        self.dir = None
        self.pool = None
        self.t_iter = {}

    def probe(self, kind):
        """Seconds per iteration from a one-iteration single-core run (first call also builds)."""
        if kind not in self.t_iter:
            t0, t1, done = _timed_iters(self.A, self.b, kind, self.Q, self.visits, 1)
            self.t_iter[kind] = max(t1 - t0, 1e-3) / max(done, 1)
        return self.t_iter[kind]

    def single(self, kind, budget_s, basis):
        k = max(1, min(200, int(budget_s / self.probe(kind))))
        t0, tk, done = _timed_iters(self.A, self.b, kind, self.Q, self.visits, k)
        per_it = max(tk - t0, 1e-6) / max(done, 1)
        return {"value": 1.0 / (per_it * basis), "cores": 1, "iters": done, "seconds": round(tk, 2),
                "fixed_s": round(t0, 2)}

    def _stage(self):
        if self.dir is None:
            import multiprocessing as mp

            self.dir = tempfile.mkdtemp(prefix="mpcg_oracle_")
            n, rp, ci, val = self.A
            for name, arr in (("n", np.array([n])), ("rp", rp), ("ci", ci), ("val", val), ("b", self.b),
                              ("Q", self.Q), ("visits", self.visits)):
                np.save(os.path.join(self.dir, name + ".npy"), np.ascontiguousarray(arr))
            self.pool = mp.get_context("spawn").Pool(host_cores())

    def all_cores(self, kind, budget_s, basis):
        self._stage()
        P = host_cores()
        # concurrent runs share the memory system: size the sample below the single-core budget
        k = max(1, min(200, int(budget_s / (2.0 * self.probe(kind)))))
        t0 = time.time()
        out = self.pool.map(_oracle_worker, [(self.dir, kind, k)] * P)
        dt = time.time() - t0
        per_it = max(max(o[1] - o[0], 1e-6) / max(o[2], 1) for o in out)  # the slowest process
        done = min(o[2] for o in out)
        return {"value": P / (per_it * basis), "cores": P, "iters": done, "seconds": round(dt, 2)}

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None
        if self.dir is not None:
            shutil.rmtree(self.dir, ignore_errors=True)
            self.dir = None


def cpu_baseline(A, b, grid, budget_s=8.0):
    """The oracle on one core (the line's cpu_baseline) plus all cores and plain fp64 CG."""
    Q, visits, basis = oracle_policy(grid)
    ob = OracleBench(A, b, Q, visits)
    try:
        rl1 = ob.single("rl", budget_s, basis["rl"][0])
        rlP = ob.all_cores("rl", budget_s, basis["rl"][0])
        f1 = ob.single("fp64", budget_s / 2, basis["fp64"][0])
        fP = ob.all_cores("fp64", budget_s / 2, basis["fp64"][0])
    finally:
        ob.close()
    return {
        "kind": "oracle", "value": rl1["value"], "unit": UNIT, "cores": 1,
        "sample": (f"the first {rl1['iters']} iterations of the same RL-mixed solve ({rl1['seconds']} s, one thread, "
                   f"less {rl1['fixed_s']} s of a solve with no iteration; policy: the oracle-trained table "
                   f"oracle/policy_fem27_c1.txt, same options), extrapolated to {basis['rl'][1]}"),
        "all_cores": {"value": rlP["value"], "cores": rlP["cores"],
                      "sample": f"{rlP['cores']} concurrent processes, {rlP['iters']} iterations each, {rlP['seconds']} s"},
        "fp64_cg": {"value_1core": f1["value"], "value_all_cores": fP["value"], "cores": fP["cores"],
                    "sample": f"plain fp64 CG (oracle, no rounding), {f1['iters']} / {fP['iters']} iterations, "
                              f"extrapolated to {basis['fp64'][1]}"},
    }


def run_reference(args):
    """CPU oracle arm: each step runs a bounded sample of the workload's RL-mixed solve on every
    host core (one process per core, the same sample each); solves/s on the oracle's own
    iteration basis."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    A, b, xs = workload(args.grid)
    Q, visits, basis = oracle_policy(args.grid)
    ob = OracleBench(A, b, Q, visits)
    try:
        for _ in range(args.warmup):
            ob.all_cores("rl", 0.5, basis["rl"][0])
        vals, secs = [], []
        for _ in range(args.steps):
            r = ob.all_cores("rl", args.ref_budget, basis["rl"][0])
            vals.append(r["value"])
            secs.append(r["seconds"])
    finally:
        ob.close()
    value = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+mixed", "data": "synthetic",
        "config": {"workload": f"fem27_aniso_{args.grid}^3", "n": A[0], "nnz": len(A[3]), "anisotropy": ANISO,
                   "tau": TAU, "policy": "tabular Q (Algorithm 1) trained by the oracle on the same family, "
                                         "operations in {fp32, fp64}; greedy (Algorithm 2)"},
        "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": r["cores"],
                         "sample": f"per step {r['cores']} concurrent oracle processes (one per host core), "
                                   f"{r['iters']} iterations of the RL-mixed solve each, extrapolated to "
                                   f"{basis['rl'][1]}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------

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


def timed_solve(ctx, mat, bd, x, pol, stream, reps=1):
    import torch

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(reps):
        res, _ = ctx.solve(mat, bd, x, TAU, MAX_ITER, pol, stream=stream)
    ev[1].record(stream)
    torch.cuda.synchronize()
    return res, ev[0].elapsed_time(ev[1]) / 1e3 / reps


def fp16_capable_policy(M, ctx_all, mat, bd, x, xs, stream, t64):
    """A policy trained with every operation free to choose any format of the paper's set
    (fp16, bf16, tf32, fp32, fp64), same training set and rounds: its greedy solve of the
    workload, against all-FP64 CG."""
    pol, t_train, its = train_policy(M, ctx_all)
    with nvtx("solve_rl_fullset"):
        ctx_all.solve(mat, bd, x, TAU, MAX_ITER, pol, stream=stream)
        res, t = timed_solve(ctx_all, mat, bd, x, pol, stream)
    ah = np.array(res["action_hist"])[:, :8]
    err = float(np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs))
    return {"policy": "tabular Q, every operation in {fp16, bf16, tf32, fp32, fp64}, same training",
            "time_to_tol_s": t, "iters": res["iters"], "outcome": res["outcome"],
            "rel_res_true": res["rel_res_true"], "rel_err_xstar": err, "speedup_vs_fp64": t64 / t,
            "action_mix": {M.FORMAT_NAMES[f]: int(ah[:, f].sum()) for f in range(8)},
            "train_s": round(t_train, 2), "restarts": res["n_restarts"]}


def batch512(M, pol_rl, stream):
    """The uneven batch: 512 SPD systems (n log-uniform on [1e3, 2e5]; 2D and 3D variable-
    coefficient diffusion and banded matrices), one persistent lockstep launch per batch captured
    in a CUDA graph, tau = 1e-8, cap 5000; fp64 CG and the benchmark's tabular policy."""
    import torch

    from paper_2504_14268_gb300 import inputs as I

    t0 = time.time()
    sets = I.cfg_batched()
    t_gen = time.time() - t0
    out = {"systems": len(sets), "rows": int(sum(s[0][0] for s in sets)),
           "nnz": int(sum(len(s[0][3]) for s in sets)), "generate_s": round(t_gen, 1)}
    for name, pol_of in (("fp64", lambda c: c.policy_fixed((4, 4, 4, 4))), ("rl", None)):
        ctx = M.Context(0, solver_options(M))
        mats = [ctx.matrix((A[0], torch.as_tensor(A[1]).cuda(), torch.as_tensor(A[2]).cuda(),
                            torch.as_tensor(A[3]).cuda())) for A, _, _ in sets]
        bs = [torch.as_tensor(b).cuda() for _, b, _ in sets]
        xs = [torch.zeros_like(b) for b in bs]
        pol = pol_of(ctx) if pol_of else ctx.policy_load(pol_rl.save())
        g = ctx.graph(mats, bs, xs, [TAU] * len(sets), [5000] * len(sets), pol)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        with nvtx(f"batch_{name}"):
            ev[0].record(stream)
            g.launch(stream)
            ev[1].record(stream)
        res = g.results(stream)
        t = ev[0].elapsed_time(ev[1]) / 1e3
        conv = sum(r["outcome"] == M.CONVERGED for r in res)
        out[name] = {"batch_s": round(t, 3), "solves_per_s": len(sets) / t, "fraction_converged": conv / len(sets),
                     "median_iters": float(np.median([r["iters"] for r in res]))}
        g.close()
        del mats, bs, xs
        ctx.close()
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", type=int, default=GRID)
    ap.add_argument("--ref-budget", type=float, default=4.0, help="seconds of oracle work per reference step")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the full-precision-set policy, the 512-system batch and the SpMV table")
    ap.add_argument("--stepped", type=int, default=0,
                    help="single-solve launch form: 0 automatic, 1 persistent kernel, 2 stepped graph, 3 stepped "
                         "passes launched by the host (profilers see each phase kernel)")
    ap.add_argument("--history-out", default=None,
                    help="write the first timed solve's per-iteration records (numpy .npy) to this path")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    global STEPPED
    STEPPED = args.stepped

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
    with Clocks(local) as clk, nvtx("solve_rl"):
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
    h0 = hist[: min(MAX_ITER, max(1, r0["iters"]))]
    xerr = float(np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs))

    # all-FP64 CG on the same GPU (same kernel, every operation in fp64)
    x64 = torch.zeros_like(bd)
    with nvtx("solve_fp64"):
        ctx.solve(mat, bd, x64, TAU, MAX_ITER, pol64, stream=stream)
        res64, t64 = timed_solve(ctx, mat, bd, x64, pol64, stream)
    xerr64 = float(np.linalg.norm(x64.cpu().numpy() - xs) / np.linalg.norm(xs))

    # roofline of the persistent kernel (the only kernel of a step)
    hbm, peak_kind = peaks()
    lb = launch_bytes(n, Z, h0)
    achieved = lb / (statistics.mean(step_ms) / 1e3) / 1e9
    ratio = traffic_ratio()
    if args.history_out:
        np.save(args.history_out, h0)
    # the product kernel alone (phase A of every iteration): its algorithmic bytes over its
    # device time, the globaltimer span from the previous phase's end to the product's end
    # (launch gap included) recorded in the history of the first timed solve
    pa_bytes = sum(product_bytes(n, Z, tuple(int(f) for f in h0["fmt"][k])) for k in range(len(h0)))
    pa_s = float(np.sum(h0["ns_a"].astype(np.float64))) / 1e9
    prod = {"kernel": "cg_phase<A> (product and nu)", "achieved": round(pa_bytes / pa_s / 1e9, 1), "peak": hbm,
            "unit": "GB/s", "frac": round(pa_bytes / pa_s / 1e9 / hbm, 3), "share_of_step":
            round(pa_s / (step_ms[0] / 1e3), 3), "source": "per-phase device time (globaltimer) of the first timed "
                                                          "solve's iteration records"}

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

    extras = {}
    if not args.no_extras and rank == 0:
        # SpMV bandwidth per value format (standalone product, autotuned schedule)
        xr = torch.rand(n, dtype=torch.float64, device="cuda")
        yr = torch.empty_like(xr)
        spmv = {}
        for fmt, name in enumerate(M.FORMAT_NAMES):
            with nvtx(f"spmv_{name}"):
                ms = ctx.spmv(mat, fmt, xr, yr, reps=10, stream=stream)
            v = BYTES[fmt]
            byts = Z * (v + 4) + 4 * (n + 1) + 2 * n * v + (4 * n if fmt in (5, 6) else 0)
            spmv[name] = {"ms": round(ms, 4), "gbs": round(byts / ms / 1e6, 1),
                          "frac": round(byts / ms / 1e6 / hbm, 3)}
        extras["spmv"] = spmv
        del xr, yr
        ctx_all = M.Context(local, solver_options(M, op_mask=(0, 0, 0, 0)))
        mat_all = ctx_all.matrix((n, torch.as_tensor(rp).cuda(), torch.as_tensor(ci).cuda(),
                                  torch.as_tensor(val).cuda()))
        mat_all.autotune(3)
        extras["fullset_policy"] = fp16_capable_policy(M, ctx_all, mat_all, bd, torch.zeros_like(bd), xs, stream, t64)
        mat_all.close()
        ctx_all.close()
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(A, b, args.grid)

    if not args.no_extras and rank == 0:
        mat.close()
        del bd, x, x64
        torch.cuda.empty_cache()
        extras["batch512"] = batch512(M, pol, stream)

    if rank == 0:
        ah = np.array(r0["action_hist"])[:, :8]
        line = {
            "metric": METRIC, "value": whole_job_rate(world, args.steps, T), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+mixed",
            "data": "synthetic",
            "config": {"workload": f"fem27_aniso_{args.grid}^3", "n": n, "nnz": Z, "anisotropy": ANISO, "tau": TAU,
                       "policy": f"tabular Q (Algorithm 1) trained on the GPU at set-up: {len(TRAIN_SET)} systems "
                                 f"24^3-48^3 of the same family, {TRAIN_ROUNDS} batched rounds, cost C1, every "
                                 f"operation in {{fp32, fp64}}, T_max {T_BIN}; greedy (Algorithm 2)",
                       "l2": "inputs larger than L2 (no flush)", "parallelism": "replicas" if world > 1 else "1 GPU"},
            "time_to_tol_s": 1e-3 * statistics.mean(step_ms), "iters": r0["iters"], "outcome": r0["outcome"],
            "rel_res_true": r0["rel_res_true"], "rel_err_xstar": xerr, "near_edge_count": r0["near_edge_count"],
            "fp64": {"time_to_tol_s": t64, "iters": res64["iters"], "rel_res_true": res64["rel_res_true"],
                     "rel_err_xstar": xerr64},
            "speedup_vs_fp64": t64 / (1e-3 * statistics.mean(step_ms)),
            "action_mix": {M.FORMAT_NAMES[f]: int(ah[:, f].sum()) for f in range(8)},
            **extras,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(achieved / hbm, 3), "traffic": None if ratio is None else round(ratio * lb),
                         "peak_source": peak_kind, "kernel": "solve step", "bytes_per_launch": lb,
                         "kernel_note": "the whole step: one launch of the solve (the stepped graph's phase "
                                        "kernels, or the persistent kernel), CUDA events around it",
                         "traffic_note": "DRAM bytes per algorithmic byte from an ncu capture of the same kernels "
                                         "on the 128^3 case, times this launch's algorithmic bytes"},
            "roofline_product": prod,
            "e2e": {"value": args.steps / e2e_T, "unit": UNIT, "h2d_bytes_per_step": 8 * n,
                    "d2h_bytes_per_step": 8 * n + 296},
            "cpu_baseline": cpu,
            "gpu_launches": int(sum(r["kernel_launches"] for r in results)),
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
