"""CPU oracle for the mixed-precision CG method -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference arms may import this package. The CUDA library does not depend on it, and
it shares no code with that library.

The numerics live in ``mpcg_oracle.c`` (plain C, fp64, single-threaded); this module
compiles it with gcc on first use and wraps it with ctypes. Every function cites the
paper passage it follows (arXiv 2504.14268): Table 1 (formats), Section 3 Eq. (1)-(4)
(CG), Section 4.1 (MDP, reward, Q-learning), Section 4.2 (operation precisions),
Algorithm 1 (training) and Algorithm 2 (inference).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpcg_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liborc.so")
_lock = threading.Lock()
_lib = None

# Format codes (same numeric order as the paper's precision set in Section 5, then extensions).
FP16, BF16, TF32, FP32, FP64, BF16R, FP16R, Q52 = range(8)
FORMAT_NAMES = ["fp16", "bf16", "tf32", "fp32", "fp64", "bf16r", "fp16r", "q52"]

CONVERGED, MAX_ITER, BREAKDOWN = 0, 1, 2
POL_FIXED, POL_SCHEDULE, POL_QTABLE, POL_MLP = 0, 1, 2, 3
MODE_INFER, MODE_TRAIN = 0, 1
NFEAT = 16


def build(force: bool = False) -> str:
    """Compiles the oracle into ``oracle/_build/liborc.so`` (gcc, no FMA contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _OUT)
    return _OUT


class Opts(C.Structure):
    _fields_ = [
        ("b_bins", C.c_int), ("r_bins", C.c_int), ("t_bin", C.c_int), ("min_k", C.c_int),
        ("eps_min", C.c_double), ("nprec", C.c_int), ("precs", C.c_int * 8), ("cost", C.c_double * 8),
        ("w1", C.c_double), ("w2", C.c_double), ("w3", C.c_double), ("lr", C.c_double),
        ("gamma", C.c_double), ("eps0", C.c_double), ("eps_floor", C.c_double), ("seed", C.c_uint64),
        ("unvisited_fallback", C.c_int), ("true_res_every", C.c_int), ("true_res_at_conv", C.c_int),
        ("op_mask", C.c_int * 4), ("on_breakdown", C.c_int), ("mlp_hidden", C.c_int), ("precond", C.c_int),
        ("variant", C.c_int), ("joint", C.c_int),
    ]


class Policy(C.Structure):
    _fields_ = [
        ("kind", C.c_int), ("fixed", C.c_int * 4), ("sched", C.c_void_p), ("sched_len", C.c_int),
        ("Q", C.c_void_p), ("visits", C.c_void_p), ("mlp", C.c_void_p), ("feat_static", C.c_void_p),
    ]


class Result(C.Structure):
    _fields_ = [("outcome", C.c_int32), ("iters", C.c_int32), ("nrec", C.c_int32), ("pad", C.c_int32),
                ("rho_rec", C.c_double), ("rho_true", C.c_double)]


REC_DTYPE = np.dtype([
    ("k", np.int32), ("state", np.int32), ("fmt", np.int32, 4), ("act", np.int32, 4),
    ("rho", np.float64), ("nu", np.float64), ("alpha", np.float64), ("sigma", np.float64),
    ("beta", np.float64), ("reward", np.float64), ("flags", np.int32), ("pad", np.int32),
])
TRANS_DTYPE = np.dtype([
    ("s", np.int32), ("s_next", np.int32), ("act", np.int32, 4), ("reward", np.float64),
    ("terminal", np.int32), ("pad", np.int32),
])


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, i, i64, d, u64 = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_uint64
            L.orc_chop.restype = d
            L.orc_chop.argtypes = [d, i]
            L.orc_chop_tee.restype = d
            L.orc_chop_tee.argtypes = [d, i, i, i]
            L.orc_chop_vec.argtypes = [vp, vp, i64, i]
            L.orc_philox4x64.argtypes = [vp, vp, vp]
            L.orc_row_scale.restype = d
            L.orc_row_scale.argtypes = [vp, vp, i]
            L.orc_state.restype = i
            L.orc_state.argtypes = [C.POINTER(Opts), i, d]
            L.orc_reward.restype = d
            L.orc_reward.argtypes = [C.POINTER(Opts), d, vp, d]
            L.orc_epsilon.restype = d
            L.orc_epsilon.argtypes = [C.POINTER(Opts), i, i]
            L.orc_draw.argtypes = [u64, u64, u64, u64, u64, C.POINTER(d), C.POINTER(C.c_uint32)]
            L.orc_spmv.argtypes = [i, vp, vp, vp, i, vp, vp]
            L.orc_dot.restype = d
            L.orc_dot.argtypes = [i64, vp, vp, i]
            L.orc_true_residual.restype = d
            L.orc_true_residual.argtypes = [i, vp, vp, vp, vp, vp, vp]
            L.orc_q_update.argtypes = [C.POINTER(Opts), vp, vp, vp]
            L.orc_greedy_action.restype = i
            L.orc_greedy_action.argtypes = [C.POINTER(Opts), vp, vp, i, d, vp]
            L.orc_run.restype = i
            L.orc_run.argtypes = [C.POINTER(Opts), i, vp, vp, vp, vp, vp, d, i, C.POINTER(Policy), i,
                                  u64, u64, d, vp, vp, vp, vp, C.POINTER(Result)]
            L.orc_train_sequential.restype = i
            L.orc_train_sequential.argtypes = [C.POINTER(Opts), i, vp, vp, vp, vp, d, i, i, u64, vp, vp, vp]
            L.orc_train_round.restype = i
            L.orc_train_round.argtypes = [C.POINTER(Opts), i, vp, vp, vp, vp, vp, d, i, i, i, vp, vp, vp]
            L.orc_mlp_nparams.restype = i64
            L.orc_mlp_nparams.argtypes = [i, i]
            L.orc_mlp_forward.argtypes = [vp, i, i, vp, vp, vp, vp]
            L.orc_mlp_loss_grad.restype = d
            L.orc_mlp_loss_grad.argtypes = [vp, i, i, i, vp, vp, vp, vp]
            L.orc_mlp_targets.argtypes = [vp, i, i, i, vp, vp, vp, d, vp, vp]
            L.orc_adam.argtypes = [vp, vp, vp, vp, i64, i, d, d, d, d]
            L.orc_static_features.argtypes = [i, vp, vp, vp, vp]
            L.orc_ic0.restype = i
            L.orc_ic0.argtypes = [i, vp, vp, vp, vp]
            L.orc_ic0_apply.argtypes = [i, vp, vp, vp, vp, vp]
            _lib = L
    return _lib


# Cost settings of Section 5 (C1, C2) for fp16, bf16, tf32, fp32, fp64. READING: the
# row-scaled extensions cost their base format plus 0.05; q52 (Table 1's quarter precision,
# outside Section 5's set, so without a published cost) half of fp16's.
COST_C1 = {FP16: 0.8, BF16: 0.6, TF32: 0.8, FP32: 1.0, FP64: 2.0, BF16R: 0.65, FP16R: 0.85, Q52: 0.4}
COST_C2 = {FP16: 0.5, BF16: 0.4, TF32: 0.5, FP32: 1.5, FP64: 3.0, BF16R: 0.45, FP16R: 0.55, Q52: 0.25}
PAPER_PRECS = (FP16, BF16, TF32, FP32, FP64)


@dataclass
class Options:
    """Hyper-parameters; defaults are Section 4.1 / Section 5 values."""
    b_bins: int = 10
    r_bins: int = 10
    t_bin: int = 1000
    min_k: int = 10
    eps_min: float = 1e-16
    precs: tuple = PAPER_PRECS
    cost: dict = field(default_factory=lambda: dict(COST_C1))
    w1: float = 1.0
    w2: float = 0.1
    w3: float = 10.0
    lr: float = 0.1
    gamma: float = 0.9
    eps0: float = 1.0
    eps_floor: float = 0.1
    seed: int = 0
    unvisited_fallback: int = FP64
    true_res_every: int = 0
    true_res_at_conv: int = 0
    op_mask: tuple = (0, 0, 0, 0)
    on_breakdown: int = 0
    mlp_hidden: int = 64
    precond: int = 0
    variant: int = 0  # 0: the CG of Section 3; 1: the single-reduction iteration (orc_run_sr)
    joint: int = 0  # 0: a Q-table per operation (Section 4.1); 1: one table over the joint actions

    def c(self) -> Opts:
        o = Opts()
        for name in ("b_bins", "r_bins", "t_bin", "min_k", "eps_min", "w1", "w2", "w3", "lr", "gamma",
                     "eps0", "eps_floor", "seed", "unvisited_fallback", "true_res_every",
                     "true_res_at_conv", "on_breakdown", "mlp_hidden", "precond", "variant", "joint"):
            setattr(o, name, getattr(self, name))
        for j in range(4):
            o.op_mask[j] = int(self.op_mask[j])
        o.nprec = len(self.precs)
        for a, f in enumerate(self.precs):
            o.precs[a] = f
            o.cost[a] = self.cost[f]
        return o

    @property
    def n_states(self) -> int:
        return self.b_bins * self.r_bins


# ---------------------------------------------------------------------------
# Elementary operations
# ---------------------------------------------------------------------------

def chop(x, fmt: int) -> np.ndarray:
    """fl_p(x) elementwise (Section 4 rounding model, Table 1 parameters), RNE, subnormals on."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    lib().orc_chop_vec(_p(x), _p(y), x.size, fmt)
    return y


def chop_tee(x: float, t: int, emin: int, emax: int) -> float:
    return lib().orc_chop_tee(float(x), t, emin, emax)


def philox4x64(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64(_p(c), _p(k), _p(out))
    return out


def draw(seed: int, e: int, lane: int, k: int, j: int):
    u = C.c_double()
    pick = C.c_uint32()
    lib().orc_draw(seed, e, lane, k, j, C.byref(u), C.byref(pick))
    return u.value, pick.value


def state(opts: Options, k: int, rho: float) -> int:
    o = opts.c()
    return lib().orc_state(C.byref(o), k, rho)


def reward(opts: Options, rho: float, act, tau: float) -> float:
    o = opts.c()
    a = np.ascontiguousarray(act, dtype=np.int32)
    return lib().orc_reward(C.byref(o), rho, _p(a), tau)


def epsilon(opts: Options, e: int, E: int) -> float:
    o = opts.c()
    return lib().orc_epsilon(C.byref(o), e, E)


def _csr(A):
    n, rp, ci, val = A
    return (int(n), np.ascontiguousarray(rp, dtype=np.int32), np.ascontiguousarray(ci, dtype=np.int32),
            np.ascontiguousarray(val, dtype=np.float64))


def spmv(A, fmt: int, p) -> np.ndarray:
    """q = fl_p1(A fl_p1(p)) with fp64 sums (Section 4.2 op 1)."""
    n, rp, ci, val = _csr(A)
    p = np.ascontiguousarray(p, dtype=np.float64)
    q = np.empty(n, dtype=np.float64)
    lib().orc_spmv(n, _p(rp), _p(ci), _p(val), fmt, _p(p), _p(q))
    return q


def dot(x, y, fmt: int) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    return lib().orc_dot(x.size, _p(x), _p(y), fmt)


def true_residual(A, b, x):
    n, rp, ci, val = _csr(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    rt = np.empty(n, dtype=np.float64)
    nn = lib().orc_true_residual(n, _p(rp), _p(ci), _p(val), _p(b), _p(x), _p(rt))
    return rt, nn


def row_scale(A, i: int) -> float:
    n, rp, ci, val = _csr(A)
    return lib().orc_row_scale(_p(rp), _p(val), i)


# ---------------------------------------------------------------------------
# Policies and solves
# ---------------------------------------------------------------------------

@dataclass
class QTable:
    """Q_j(s, p) for the four operations (Section 4.1) plus per-(op, state) update counts."""
    Q: np.ndarray       # [4, S, nprec] float64
    visits: np.ndarray  # [4, S] int32

    @staticmethod
    def zeros(opts: Options) -> "QTable":
        S = opts.n_states
        if opts.joint:  # one table over the joint actions: [S][|P|^4], counts per state
            return QTable(np.zeros((S, len(opts.precs) ** 4)), np.zeros(S, dtype=np.int32))
        return QTable(np.zeros((4, S, len(opts.precs))), np.zeros((4, S), dtype=np.int32))

    def copy(self) -> "QTable":
        return QTable(self.Q.copy(), self.visits.copy())


def _policy(kind, fixed=None, sched=None, qt=None, mlp=None, feat_static=None):
    P = Policy()
    P.kind = kind
    keep = []
    if fixed is not None:
        for j in range(4):
            P.fixed[j] = int(fixed[j])
    if sched is not None:
        s = np.ascontiguousarray(sched, dtype=np.int32).reshape(-1, 4)
        keep.append(s)
        P.sched = _p(s)
        P.sched_len = s.shape[0]
    if qt is not None:
        assert qt.Q.flags.c_contiguous and qt.Q.dtype == np.float64
        assert qt.visits.flags.c_contiguous and qt.visits.dtype == np.int32
        P.Q = _p(qt.Q)
        P.visits = _p(qt.visits)
    if mlp is not None:
        m = np.ascontiguousarray(mlp, dtype=np.float64)
        keep.append(m)
        P.mlp = _p(m)
    if feat_static is not None:
        f = np.ascontiguousarray(feat_static, dtype=np.float64)
        keep.append(f)
        P.feat_static = _p(f)
    return P, keep


@dataclass
class SolveOut:
    x: np.ndarray
    outcome: int
    iters: int
    rho_rec: float
    rho_true: float
    hist: np.ndarray
    feats: np.ndarray | None = None
    trans: np.ndarray | None = None


def solve(opts: Options, A, b, tau: float, max_iter: int, *, fixed=None, sched=None, qtable=None,
          mlp=None, feat_static=None, x0=None, train: bool = False, episode: int = 0, lane: int = 0,
          eps: float = 0.0, want_feats: bool = False, want_trans: bool = False) -> SolveOut:
    """Algorithm 2 (or, with train=True, one episode of Algorithm 1's loop)."""
    n, rp, ci, val = _csr(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    if fixed is not None:
        P, keep = _policy(POL_FIXED, fixed=fixed)
    elif sched is not None:
        P, keep = _policy(POL_SCHEDULE, sched=sched)
    elif qtable is not None:
        P, keep = _policy(POL_QTABLE, qt=qtable, feat_static=feat_static)
    elif mlp is not None:
        P, keep = _policy(POL_MLP, mlp=mlp, feat_static=feat_static)
    else:
        raise ValueError("no policy")
    o = opts.c()
    hist = np.zeros(max(max_iter, 1), dtype=REC_DTYPE)
    feats = np.zeros((max_iter + 1, NFEAT)) if want_feats else None
    trans = np.zeros(max(max_iter, 1), dtype=TRANS_DTYPE) if want_trans else None
    ntrans = np.zeros(1, dtype=np.int32)
    res = Result()
    rc = lib().orc_run(C.byref(o), n, _p(rp), _p(ci), _p(val), _p(b), _p(x), tau, max_iter, C.byref(P),
                       MODE_TRAIN if train else MODE_INFER, episode, lane, eps, _p(trans), _p(ntrans),
                       _p(hist), _p(feats), C.byref(res))
    del keep
    if rc < 0:
        raise ValueError(_PRECOND_ERRORS.get(rc, f"solve refused ({rc})"))
    hist = hist[: res.nrec]
    return SolveOut(x, res.outcome, res.iters, res.rho_rec, res.rho_true, hist,
                    feats[: len(hist) + 1] if feats is not None else None,
                    trans[: int(ntrans[0])] if trans is not None else None)


_PRECOND_ERRORS = {
    -1: "Jacobi preconditioning needs a positive diagonal entry in every row",
    -2: "incomplete Cholesky breaks down (a non-positive pivot)",
    -3: "incomplete Cholesky needs a diagonal entry in every row, strictly increasing columns "
        "and a symmetric pattern",
    -4: "the single-reduction iteration runs with M = I or Jacobi",
}


def ic0(A) -> np.ndarray:
    """IC(0) factor in fp32 (orc_ic0): one value per stored entry, l_ij at (i, j) for j <= i
    and l_ji at (i, j) for j > i. Raises ValueError on breakdown or an unusable pattern."""
    n, rp, ci, val = _csr(A)
    L = np.zeros(max(len(ci), 1), dtype=np.float32)
    rc = lib().orc_ic0(n, _p(rp), _p(ci), _p(val), _p(L))
    if rc < 0:
        raise ValueError(_PRECOND_ERRORS[rc])
    return L[: len(ci)]


def ic0_apply(A, L, r) -> np.ndarray:
    """M^-1 r for M = L L^T in fp32 (forward then backward substitution), returned in fp64."""
    n, rp, ci, _ = _csr(A)
    L = np.ascontiguousarray(L, dtype=np.float32)
    r = np.ascontiguousarray(r, dtype=np.float64)
    w = np.zeros(n)
    lib().orc_ic0_apply(n, _p(rp), _p(ci), _p(L), _p(r), _p(w))
    return w


def train_sequential(opts: Options, A, b, tau: float, t_max: int, E: int, qt: QTable, ep_base: int = 0):
    """Algorithm 1 on one matrix: E episodes with online Q updates. Returns iterations per episode."""
    n, rp, ci, val = _csr(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    o = opts.c()
    iters = np.zeros(E, dtype=np.int32)
    lib().orc_train_sequential(C.byref(o), n, _p(rp), _p(ci), _p(val), _p(b), tau, t_max, E, ep_base,
                               _p(qt.Q), _p(qt.visits), _p(iters))
    return iters


def train_round(opts: Options, mats, bs, tau: float, t_max: int, e: int, E: int, qt: QTable):
    """One round of the batched reading of Algorithm 1 (lane-private episodes, ordered replay)."""
    B = len(mats)
    cs = [_csr(A) for A in mats]
    bs = [np.ascontiguousarray(b, dtype=np.float64) for b in bs]
    ns = np.array([c[0] for c in cs], dtype=np.int32)
    arr = lambda xs: (C.c_void_p * B)(*[x.ctypes.data for x in xs])
    o = opts.c()
    iters = np.zeros(B, dtype=np.int32)
    lib().orc_train_round(C.byref(o), B, _p(ns), arr([c[1] for c in cs]), arr([c[2] for c in cs]),
                          arr([c[3] for c in cs]), arr(bs), tau, t_max, e, E, _p(qt.Q), _p(qt.visits),
                          _p(iters))
    return iters


def greedy_action(opts: Options, qt: QTable, k: int, rho: float):
    """Algorithm 2's decision at iteration k with residual rho: (state, formats of ops 1-4)."""
    o = opts.c()
    act = np.zeros(4, dtype=np.int32)
    s = lib().orc_greedy_action(C.byref(o), _p(qt.Q), _p(qt.visits), int(k), float(rho), _p(act))
    return s, tuple(int(opts.precs[a]) for a in act)


def q_update(opts: Options, qt: QTable, trans: np.ndarray):
    o = opts.c()
    for t in np.atleast_1d(trans):
        tt = np.array([t], dtype=TRANS_DTYPE)
        lib().orc_q_update(C.byref(o), _p(qt.Q), _p(qt.visits), _p(tt))


# ---------------------------------------------------------------------------
# MLP Q-function (extension)
# ---------------------------------------------------------------------------

def mlp_nparams(H: int, nout: int) -> int:
    return lib().orc_mlp_nparams(H, nout)


def mlp_forward(w, H: int, nout: int, f):
    w = np.ascontiguousarray(w, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    h1, h2, out = np.zeros(H), np.zeros(H), np.zeros(nout)
    lib().orc_mlp_forward(_p(w), H, nout, _p(f), _p(h1), _p(h2), _p(out))
    return out, h1, h2


def mlp_loss_grad(w, H: int, nprec: int, feats, acts, y):
    w = np.ascontiguousarray(w, dtype=np.float64)
    feats = np.ascontiguousarray(feats, dtype=np.float64)
    acts = np.ascontiguousarray(acts, dtype=np.int32)
    y = np.ascontiguousarray(y, dtype=np.float64)
    g = np.zeros_like(w)
    B = feats.shape[0]
    loss = lib().orc_mlp_loss_grad(_p(w), H, nprec, B, _p(feats), _p(acts), _p(y), _p(g))
    return loss, g


def mlp_targets(wt, H: int, nprec: int, feats_next, rew, done, gamma: float, op_mask=(0, 0, 0, 0)):
    """Fitted-Q targets y[B][4] = r + gamma (1 - done) max over allowed p of Q_target(f_next)[j, p]."""
    wt = np.ascontiguousarray(wt, dtype=np.float64)
    fn = np.ascontiguousarray(feats_next, dtype=np.float64)
    rew = np.ascontiguousarray(rew, dtype=np.float64)
    done = np.ascontiguousarray(done, dtype=np.int32)
    mask = np.ascontiguousarray(op_mask, dtype=np.int32)
    B = fn.shape[0]
    y = np.zeros((B, 4))
    lib().orc_mlp_targets(_p(wt), H, nprec, B, _p(fn), _p(rew), _p(done), float(gamma), _p(mask), _p(y))
    return y


def adam(w, m, v, g, t: int, lr: float = 1e-3, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    for a in (w, m, v):
        assert a.flags.c_contiguous and a.dtype == np.float64
    g = np.ascontiguousarray(g, dtype=np.float64)
    lib().orc_adam(_p(w), _p(m), _p(v), _p(g), w.size, t, lr, b1, b2, eps)


def static_features(A) -> np.ndarray:
    n, rp, ci, val = _csr(A)
    f = np.zeros(5)
    lib().orc_static_features(n, _p(rp), _p(ci), _p(val), _p(f))
    return f
