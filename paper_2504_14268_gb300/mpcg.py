"""Thin Python binding of the C ABI in include/mpcg.h (argument marshalling only).

Every numerical step runs in the CUDA library libmpcg.so; this module only converts
numpy arrays / torch tensors to pointers, fills the C structs and checks status codes.
It raises if the library has not been built: there is no fallback.

Raw functions keep the C names (``mpcg_create``, ``mpcg_solve``, ...); the classes
``Context``, ``Matrix``, ``Policy`` and ``Graph`` wrap the handles.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field, fields

import numpy as np

from . import build as _build

FP16, BF16, TF32, FP32, FP64, BF16R, FP16R, Q52 = range(8)
FORMAT_NAMES = ["fp16", "bf16", "tf32", "fp32", "fp64", "bf16r", "fp16r", "q52"]
CONVERGED, MAX_ITER, BREAKDOWN = 0, 1, 2
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "BAD_POLICY", 5: "TIMEOUT", 6: "INTERNAL"}
SCHED_VECTOR, SCHED_STREAM, SCHED_VLOAD, SCHED_MERGE, SCHED_XSTAGE = 0, 1, 2, 3, 4


class MpcgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mpcg status {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p)]


class COptions(C.Structure):
    _fields_ = [
        ("b_bins", C.c_int32), ("r_bins", C.c_int32), ("t_bin", C.c_int32), ("min_k", C.c_int32),
        ("eps_min", C.c_double), ("nprec", C.c_int32), ("precs", C.c_int32 * 8), ("cost", C.c_double * 8),
        ("w1", C.c_double), ("w2", C.c_double), ("w3", C.c_double), ("lr", C.c_double), ("gamma", C.c_double),
        ("eps0", C.c_double), ("eps_floor", C.c_double), ("seed", C.c_uint64),
        ("unvisited_fallback", C.c_int32), ("true_res_every", C.c_int32), ("true_res_at_conv", C.c_int32),
        ("warm_start", C.c_int32), ("op_mask", C.c_int32 * 4), ("on_breakdown", C.c_int32),
        ("mlp_hidden", C.c_int32),
        ("batch_mode", C.c_int32),
        ("precond", C.c_int32),
        ("edge_tol", C.c_double),
        ("stepped", C.c_int32), ("variant", C.c_int32),
        ("joint", C.c_int32), ("reserved_joint", C.c_int32),
    ]


class CResult(C.Structure):
    _fields_ = [("outcome", C.c_int32), ("iters", C.c_int32), ("rel_res_rec", C.c_double),
                ("rel_res_true", C.c_double), ("n_true_checks", C.c_int32), ("n_restarts", C.c_int32),
                ("action_hist", (C.c_int64 * 8) * 4), ("near_edge_count", C.c_int32),
                ("kernel_launches", C.c_int32)]


class CStats(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("mean_row_nnz", C.c_double), ("max_row_nnz", C.c_double),
                ("cv_row_nnz", C.c_double), ("spmv_sched", C.c_int32 * 8), ("spmv_lanes", C.c_int32 * 8),
                ("device_bytes", C.c_int64), ("static_features", C.c_double * 5)]


TRANS_DTYPE = np.dtype([
    ("f", np.float32, 16), ("f_next", np.float32, 16), ("act", np.int32, 4), ("reward", np.float32),
    ("done", np.int32),
])
assert TRANS_DTYPE.itemsize == 152

REC_DTYPE = np.dtype([
    ("k", np.int32), ("state", np.int32), ("fmt", np.int8, 4), ("act", np.int8, 4),
    ("rho", np.float64), ("nu", np.float64), ("alpha", np.float64), ("sigma", np.float64),
    ("beta", np.float64), ("reward", np.float64), ("flags", np.int32), ("ns_a", np.uint32),
    ("ns_b", np.uint32), ("ns_c", np.uint32),
])
assert REC_DTYPE.itemsize == 80

# Every entry point declared in include/mpcg.h, with (restype, argtypes).
_vp, _i32, _i64, _d, _sz = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_size_t
_st = C.c_int
SIGNATURES = {
    "mpcg_options_default": (None, [C.POINTER(COptions)]),
    "mpcg_create": (_st, [C.POINTER(_vp), C.c_int, C.POINTER(COptions)]),
    "mpcg_destroy": (_st, [_vp]),
    "mpcg_last_error": (C.c_char_p, [_vp]),
    "mpcg_device_info": (_st, [_vp, C.POINTER(_i32), C.POINTER(_i32)]),
    "mpcg_matrix_create": (_st, [_vp, C.POINTER(Csr), C.POINTER(_vp), _vp]),
    "mpcg_matrix_destroy": (_st, [_vp]),
    "mpcg_matrix_info": (_st, [_vp, C.POINTER(CStats)]),
    "mpcg_matrix_autotune": (_st, [_vp, _vp, _i32, _vp]),
    "mpcg_matrix_set_schedule": (_st, [_vp, _i32, _i32, _i32]),
    "mpcg_matrix_ic0": (_st, [_vp, _vp, _vp, _vp]),
    "mpcg_csr_levels": (_st, [_i32, _vp, _vp, _vp, _vp, _vp]),
    "mpcg_spmv": (_st, [_vp, _vp, _i32, _vp, _vp, _i32, C.POINTER(_d), _vp]),
    "mpcg_policy_fixed": (_st, [_vp, C.POINTER(_i32), C.POINTER(_vp)]),
    "mpcg_policy_schedule": (_st, [_vp, _vp, _i32, C.POINTER(_vp)]),
    "mpcg_policy_qtable": (_st, [_vp, _vp, _vp, C.POINTER(_vp)]),
    "mpcg_policy_mlp": (_st, [_vp, _vp, C.POINTER(_vp)]),
    "mpcg_mlp_nparams": (_i64, [_i32, _i32]),
    "mpcg_policy_get_qtable": (_st, [_vp, _vp, _vp]),
    "mpcg_policy_get_mlp": (_st, [_vp, _vp]),
    "mpcg_policy_save": (_st, [_vp, _vp, C.POINTER(_sz)]),
    "mpcg_policy_load": (_st, [_vp, _vp, _sz, C.POINTER(_vp)]),
    "mpcg_policy_destroy": (_st, [_vp]),
    "mpcg_solve": (_st, [_vp, _vp, _vp, _vp, _d, _i32, _vp, C.POINTER(CResult), _vp, _i32, _vp]),
    "mpcg_solve_batched": (_st, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "mpcg_solve_noalloc": (_st, [_vp, _vp, _vp, _vp, _d, _i32, _vp, C.POINTER(CResult), _vp]),
    "mpcg_graph_create": (_st, [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.POINTER(_vp)]),
    "mpcg_graph_launch": (_st, [_vp, _vp]),
    "mpcg_graph_results": (_st, [_vp, _vp, _vp]),
    "mpcg_graph_destroy": (_st, [_vp]),
    "mpcg_train_qtable": (_st, [_vp, _i32, _vp, _vp, _d, _i32, _i32, _vp, _vp, _vp]),
    "mpcg_collect": (_st, [_vp, _i32, _vp, _vp, _d, _i32, _vp, _d, C.c_uint64, _vp, _i64, C.POINTER(_i64), _vp]),
    "mpcg_mlp_loss_grad": (_st, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, C.POINTER(_d), _vp]),
    "mpcg_mlp_train": (_st, [_vp, _vp, _vp, _i64, _i32, _i32, C.c_float, _i32, C.c_uint64, _vp, _vp]),
    "mpcg_mlp_targets": (_st, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp]),
    "mpcg_mlp_adam": (_st, [_vp, _vp, _vp, _vp, _vp, _i32, C.c_float, _vp]),
}

_LIB = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Loads libmpcg.so (built by __graft_entry__.build() / paper_2504_14268_gb300.build)."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise ImportError(f"libmpcg.so is not built ({path}); run python -m paper_2504_14268_gb300.build")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _ptr(a):
    """Pointer of a contiguous numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(a)}")


def _dtype_name(a):
    return str(a.dtype).replace("torch.", "")


def _check_dtype(a, name, want):
    if a is not None and _dtype_name(a) != want:
        raise TypeError(f"{name} must be {want}, got {_dtype_name(a)}")


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


@dataclass
class Options:
    """Mirror of mpcg_options (defaults: Sections 4.1 and 5 of the paper, cost setting C1)."""
    b_bins: int = 10
    r_bins: int = 10
    t_bin: int = 1000
    min_k: int = 10
    eps_min: float = 1e-16
    precs: tuple = (FP16, BF16, TF32, FP32, FP64)
    cost: tuple = (0.8, 0.6, 0.8, 1.0, 2.0)
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
    warm_start: int = 0
    op_mask: tuple = (0, 0, 0, 0)
    on_breakdown: int = 0
    mlp_hidden: int = 64
    batch_mode: int = 0
    precond: int = 0  # 0: M = I; 1: Jacobi; 2: fp32 IC(0) (factor kept with the matrix)
    edge_tol: float = 5e-3  # greedy decisions this close (relative) to a residual-bin edge are counted
    stepped: int = 0  # single solves: 0 automatic, 1 persistent launch, 2 one kernel per phase in a graph loop
    variant: int = 0  # 0: the CG of Section 3; 1: the single-reduction iteration (lockstep / stepped kernels)
    joint: int = 0  # tabular policies: 1 = one table over the joint actions, Q[S][nprec^4], visits[S]

    def c(self) -> COptions:
        o = COptions()
        for f in fields(self):
            if f.name in ("precs", "cost", "op_mask", "reserved_joint"):
                continue
            setattr(o, f.name, getattr(self, f.name))
        if len(self.precs) != len(self.cost):
            raise ValueError("precs and cost must have the same length")
        for j in range(4):
            o.op_mask[j] = int(self.op_mask[j])
        o.nprec = len(self.precs)
        for a, (p, c) in enumerate(zip(self.precs, self.cost)):
            o.precs[a] = p
            o.cost[a] = c
        return o

    @property
    def n_states(self):
        return self.b_bins * self.r_bins


def result_dict(r: CResult) -> dict:
    return dict(outcome=r.outcome, iters=r.iters, rel_res_rec=r.rel_res_rec, rel_res_true=r.rel_res_true,
                n_true_checks=r.n_true_checks, n_restarts=r.n_restarts,
                action_hist=np.array([list(row) for row in r.action_hist]), near_edge_count=r.near_edge_count,
                kernel_launches=r.kernel_launches)


class Context:
    """mpcg_create / mpcg_destroy."""

    def __init__(self, device: int = 0, options: Options | None = None):
        self.options = options or Options()
        self._opts = self.options.c()
        h = C.c_void_p()
        self._check(lib().mpcg_create(C.byref(h), device, C.byref(self._opts)), ctx=False)
        self.handle = h

    def _check(self, status: int, ctx: bool = True):
        if status != 0:
            msg = lib().mpcg_last_error(self.handle).decode() if ctx else "mpcg_create failed"
            raise MpcgError(status, msg)

    def close(self):
        if getattr(self, "handle", None):
            lib().mpcg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_info(self):
        a, b = C.c_int32(), C.c_int32()
        self._check(lib().mpcg_device_info(self.handle, C.byref(a), C.byref(b)))
        return a.value, b.value

    # ---- matrices
    def matrix(self, A, stream=None) -> "Matrix":
        n, rp, ci, val = A
        _check_dtype(rp, "row_ptr", "int32")
        _check_dtype(ci, "col", "int32")
        _check_dtype(val, "val", "float64")
        csr = Csr(int(n), int(val.shape[0]) if hasattr(val, "shape") else len(val), _ptr(rp), _ptr(ci), _ptr(val))
        h = C.c_void_p()
        self._check(lib().mpcg_matrix_create(self.handle, C.byref(csr), C.byref(h), _stream(stream)))
        return Matrix(self, h, int(n))

    # ---- policies
    def policy_fixed(self, fmts) -> "Policy":
        arr = (C.c_int32 * 4)(*[int(f) for f in fmts])
        h = C.c_void_p()
        self._check(lib().mpcg_policy_fixed(self.handle, arr, C.byref(h)))
        return Policy(self, h, "fixed")

    def policy_schedule(self, fmts) -> "Policy":
        a = np.ascontiguousarray(np.asarray(fmts, dtype=np.int32).reshape(-1, 4))
        h = C.c_void_p()
        self._check(lib().mpcg_policy_schedule(self.handle, _ptr(a), a.shape[0], C.byref(h)))
        return Policy(self, h, "schedule")

    def qtable_shapes(self):
        """Shapes of a tabular policy's (Q, visits) under this context's options."""
        o = self.options
        P = len(o.precs)
        if o.joint:
            return (o.n_states, P ** 4), (o.n_states,)
        return (4, o.n_states, P), (4, o.n_states)

    def policy_qtable(self, Q, visits=None) -> "Policy":
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        v = None if visits is None else np.ascontiguousarray(visits, dtype=np.int32)
        qs, vs = self.qtable_shapes()
        if Q.size != int(np.prod(qs)) or (v is not None and v.size != int(np.prod(vs))):
            raise ValueError(f"Q-table must have {qs} entries and visits {vs}")
        h = C.c_void_p()
        self._check(lib().mpcg_policy_qtable(self.handle, _ptr(Q), _ptr(v), C.byref(h)))
        return Policy(self, h, "qtable")

    def policy_mlp(self, params) -> "Policy":
        p = np.ascontiguousarray(params, dtype=np.float32)
        need = lib().mpcg_mlp_nparams(self.options.mlp_hidden, len(self.options.precs))
        if p.size != need:
            raise ValueError(f"MLP needs {need} parameters, got {p.size}")
        h = C.c_void_p()
        self._check(lib().mpcg_policy_mlp(self.handle, _ptr(p), C.byref(h)))
        return Policy(self, h, "mlp")

    def policy_load(self, blob: bytes) -> "Policy":
        buf = C.create_string_buffer(blob, len(blob))
        h = C.c_void_p()
        self._check(lib().mpcg_policy_load(self.handle, buf, len(blob), C.byref(h)))
        return Policy(self, h, "loaded")

    # ---- solves
    def solve(self, A: "Matrix", b, x, tol: float, max_iter: int, policy: "Policy", history_cap: int = 0,
              history=None, stream=None):
        """mpcg_solve. b, x: float64 numpy arrays or torch tensors (host or device). Returns
        (result dict, history records or None)."""
        _check_dtype(b, "b", "float64")
        _check_dtype(x, "x", "float64")
        res = CResult()
        if history is None and history_cap > 0:
            history = np.zeros(history_cap, dtype=REC_DTYPE)
        cap = 0 if history is None else (history.shape[0] if hasattr(history, "shape") else len(history))
        self._check(lib().mpcg_solve(self.handle, A.handle, _ptr(b), _ptr(x), float(tol), int(max_iter),
                                     policy.handle, C.byref(res), _ptr(history), int(cap), _stream(stream)))
        return result_dict(res), history

    def solve_noalloc(self, A: "Matrix", b, x, tol: float, max_iter: int, policy: "Policy", stream=None) -> dict:
        """mpcg_solve_noalloc: the solve without device allocation (b, x device tensors)."""
        _check_dtype(b, "b", "float64")
        _check_dtype(x, "x", "float64")
        res = CResult()
        self._check(lib().mpcg_solve_noalloc(self.handle, A.handle, _ptr(b), _ptr(x), float(tol), int(max_iter),
                                             policy.handle, C.byref(res), _stream(stream)))
        return result_dict(res)

    def solve_batched(self, mats, bs, xs, tols, max_iters, policy: "Policy", stream=None):
        """mpcg_solve_batched with device tensors. Returns a list of result dicts."""
        nsys = len(mats)
        A = (C.c_void_p * nsys)(*[m.handle.value for m in mats])
        B = (C.c_void_p * nsys)(*[_ptr(b).value for b in bs])
        X = (C.c_void_p * nsys)(*[_ptr(x).value for x in xs])
        T = (C.c_double * nsys)(*[float(t) for t in tols])
        M = (C.c_int32 * nsys)(*[int(m) for m in max_iters])
        R = (CResult * nsys)()
        self._check(lib().mpcg_solve_batched(self.handle, nsys, A, B, X, T, M, policy.handle, R, _stream(stream)))
        return [result_dict(r) for r in R]

    def graph(self, mats, bs, xs, tols, max_iters, policy: "Policy", stream=None) -> "Graph":
        nsys = len(mats)
        A = (C.c_void_p * nsys)(*[m.handle.value for m in mats])
        B = (C.c_void_p * nsys)(*[_ptr(b).value for b in bs])
        X = (C.c_void_p * nsys)(*[_ptr(x).value for x in xs])
        T = (C.c_double * nsys)(*[float(t) for t in tols])
        M = (C.c_int32 * nsys)(*[int(m) for m in max_iters])
        h = C.c_void_p()
        self._check(lib().mpcg_graph_create(self.handle, nsys, A, B, X, T, M, policy.handle, _stream(stream),
                                            C.byref(h)))
        return Graph(self, h, nsys)

    def train_qtable(self, mats, bs, tol: float, t_max: int, episodes: int, policy: "Policy",
                     want_iters: bool = False, stream=None):
        nsys = len(mats)
        A = (C.c_void_p * nsys)(*[m.handle.value for m in mats])
        B = (C.c_void_p * nsys)(*[_ptr(b).value for b in bs])
        it = np.zeros((episodes, nsys), dtype=np.int32) if want_iters else None
        self._check(lib().mpcg_train_qtable(self.handle, nsys, A, B, float(tol), int(t_max), int(episodes),
                                            policy.handle, _ptr(it), _stream(stream)))
        return it

    def collect(self, mats, bs, tol: float, max_iter: int, behavior: "Policy", eps: float, episode: int,
                cap: int | None = None, stream=None) -> np.ndarray:
        """mpcg_collect: one epsilon-greedy episode per system; returns TRANS_DTYPE records."""
        nsys = len(mats)
        cap = cap if cap is not None else nsys * max_iter
        out = np.zeros(cap, dtype=TRANS_DTYPE)
        A = (C.c_void_p * nsys)(*[m.handle.value for m in mats])
        B = (C.c_void_p * nsys)(*[_ptr(b).value for b in bs])
        cnt = C.c_int64()
        self._check(lib().mpcg_collect(self.handle, nsys, A, B, float(tol), int(max_iter), behavior.handle, float(eps),
                                       int(episode), _ptr(out), int(cap), C.byref(cnt), _stream(stream)))
        return out[: cnt.value]

    def mlp_loss_grad(self, params, feats, acts, y, stream=None):
        p = np.ascontiguousarray(params, dtype=np.float32)
        f = np.ascontiguousarray(feats, dtype=np.float32)
        a = np.ascontiguousarray(acts, dtype=np.int32)
        yy = np.ascontiguousarray(y, dtype=np.float32)
        g = np.zeros_like(p)
        loss = C.c_double()
        self._check(lib().mpcg_mlp_loss_grad(self.handle, _ptr(p), f.shape[0], _ptr(f), _ptr(a), _ptr(yy), _ptr(g),
                                             C.byref(loss), _stream(stream)))
        return loss.value, g

    def mlp_targets(self, target_params, feats_next, rew, done, stream=None) -> np.ndarray:
        """mpcg_mlp_targets: fitted-Q targets y[B][4] (host arrays in and out)."""
        w = np.ascontiguousarray(target_params, dtype=np.float32)
        fn = np.ascontiguousarray(feats_next, dtype=np.float32)
        r = np.ascontiguousarray(rew, dtype=np.float32)
        dn = np.ascontiguousarray(done, dtype=np.int32)
        y = np.zeros((fn.shape[0], 4), dtype=np.float32)
        self._check(lib().mpcg_mlp_targets(self.handle, _ptr(w), fn.shape[0], _ptr(fn), _ptr(r), _ptr(dn), _ptr(y),
                                           _stream(stream)))
        return y

    def mlp_train(self, policy: "Policy", data, steps: int, batch: int = 4096, lr: float = 1e-3,
                  target_sync: int = 200, seed: int = 0, stream=None) -> np.ndarray:
        d = np.ascontiguousarray(data, dtype=TRANS_DTYPE)
        losses = np.zeros(steps, dtype=np.float32)
        self._check(lib().mpcg_mlp_train(self.handle, policy.handle, _ptr(d), d.shape[0], int(steps), int(batch),
                                         float(lr), int(target_sync), int(seed), _ptr(losses), _stream(stream)))
        return losses

    def mlp_adam(self, params, m, v, grad, t: int, lr: float = 1e-3, stream=None):
        """mpcg_mlp_adam: one Adam step; params, m, v (float32 host arrays) updated in place."""
        for a in (params, m, v):
            if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags.c_contiguous):
                raise TypeError("params, m and v must be C-contiguous float32 numpy arrays")
        g = np.ascontiguousarray(grad, dtype=np.float32)
        self._check(lib().mpcg_mlp_adam(self.handle, _ptr(params), _ptr(m), _ptr(v), _ptr(g), int(t), float(lr),
                                        _stream(stream)))

    def spmv(self, A: "Matrix", fmt: int, x, y, reps: int = 1, stream=None) -> float:
        ms = C.c_double()
        self._check(lib().mpcg_spmv(self.handle, A.handle, int(fmt), _ptr(x), _ptr(y), int(reps), C.byref(ms),
                                    _stream(stream)))
        return ms.value


class Matrix:
    def __init__(self, ctx: Context, handle, n: int):
        self.ctx, self.handle, self.n = ctx, handle, n

    def info(self) -> dict:
        s = CStats()
        self.ctx._check(lib().mpcg_matrix_info(self.handle, C.byref(s)))
        return dict(n=s.n, nnz=s.nnz, mean_row_nnz=s.mean_row_nnz, max_row_nnz=s.max_row_nnz,
                    cv_row_nnz=s.cv_row_nnz, spmv_sched=list(s.spmv_sched), spmv_lanes=list(s.spmv_lanes),
                    device_bytes=s.device_bytes, static_features=list(s.static_features))

    def autotune(self, reps: int = 5, stream=None):
        self.ctx._check(lib().mpcg_matrix_autotune(self.ctx.handle, self.handle, int(reps), _stream(stream)))

    def set_schedule(self, fmt: int, sched: int, lanes: int):
        self.ctx._check(lib().mpcg_matrix_set_schedule(self.handle, int(fmt), int(sched), int(lanes)))

    def ic0(self, out=None, stream=None):
        """IC(0) factor in fp32 (mpcg_matrix_ic0); `out`: a float32 device tensor of nnz
        elements that receives it, or None to only compute and keep it with the matrix."""
        _check_dtype(out, "out", "float32")
        self.ctx._check(lib().mpcg_matrix_ic0(self.ctx.handle, self.handle, _ptr(out), _stream(stream)))
        return out

    def close(self):
        if getattr(self, "handle", None):
            lib().mpcg_matrix_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Policy:
    def __init__(self, ctx: Context, handle, kind: str):
        self.ctx, self.handle, self.kind = ctx, handle, kind

    def qtable(self):
        qs, vs = self.ctx.qtable_shapes()
        Q = np.zeros(qs)
        v = np.zeros(vs, dtype=np.int32)
        self.ctx._check(lib().mpcg_policy_get_qtable(self.handle, _ptr(Q), _ptr(v)))
        return Q, v

    def mlp_params(self):
        o = self.ctx.options
        p = np.zeros(lib().mpcg_mlp_nparams(o.mlp_hidden, len(o.precs)), dtype=np.float32)
        self.ctx._check(lib().mpcg_policy_get_mlp(self.handle, _ptr(p)))
        return p

    def save(self) -> bytes:
        n = C.c_size_t(0)
        self.ctx._check(lib().mpcg_policy_save(self.handle, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self.ctx._check(lib().mpcg_policy_save(self.handle, buf, C.byref(n)))
        return buf.raw[: n.value]

    def close(self):
        if getattr(self, "handle", None):
            lib().mpcg_policy_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    def __init__(self, ctx: Context, handle, nsys: int):
        self.ctx, self.handle, self.nsys = ctx, handle, nsys

    def launch(self, stream=None):
        self.ctx._check(lib().mpcg_graph_launch(self.handle, _stream(stream)))

    def results(self, stream=None):
        R = (CResult * self.nsys)()
        self.ctx._check(lib().mpcg_graph_results(self.handle, R, _stream(stream)))
        return [result_dict(r) for r in R]

    def close(self):
        if getattr(self, "handle", None):
            lib().mpcg_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlp_nparams(hidden: int, nprec: int) -> int:
    return int(lib().mpcg_mlp_nparams(hidden, nprec))


def csr_levels(A):
    """mpcg_csr_levels on a host CSR (n, row_ptr, col, ...): the dependency levels of the
    substitutions L y = r and L^T w = y over its pattern, and their depths."""
    n, rp, ci = int(A[0]), np.ascontiguousarray(A[1], dtype=np.int32), np.ascontiguousarray(A[2], dtype=np.int32)
    lo = np.zeros(max(n, 1), dtype=np.int32)
    up = np.zeros(max(n, 1), dtype=np.int32)
    depth = np.zeros(2, dtype=np.int32)
    st = lib().mpcg_csr_levels(n, _ptr(rp), _ptr(ci), _ptr(lo), _ptr(up), _ptr(depth))
    if st != 0:
        raise MpcgError(st, "mpcg_csr_levels: invalid CSR")
    return lo[:n], up[:n], (int(depth[0]), int(depth[1]))
