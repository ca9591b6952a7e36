"""Full-size checks on the 256^3 anisotropic 27-point workload (n = 16.8M, Z = 449M), in the
launch configuration the benchmark times (autotuned schedules).

The oracle cannot run this size end to end, so the product is checked on sampled rows
(the oracle computes each sampled row of q = fl_p1(A fl_p1(x)) exactly as it would in a
full product) and the solve through properties that hold at any size."""
import numpy as np
import pytest

import oracle as O
from paper_2504_14268_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 256
T_BITS = {0: 11, 1: 8, 2: 11, 3: 24, 5: 8, 6: 11}


@pytest.fixture(scope="module")
def big():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2504_14268_gb300 import mpcg as M

    A = I.fem27_aniso(N, 1e-3)
    xs, b = I.rhs_from_xstar(A, np.random.default_rng(0))
    ctx = M.Context(0, M.Options(true_res_at_conv=1, on_breakdown=1))
    n, rp, ci, val = A
    mat = ctx.matrix((n, torch.as_tensor(rp).cuda(), torch.as_tensor(ci).cuda(), torch.as_tensor(val).cuda()))
    return M, A, xs, b, ctx, mat


def _sample_rows(A, count=3000, seed=0):
    n, rp, ci, val = A
    rng = np.random.default_rng(seed)
    rows = set(rng.integers(0, n, count).tolist())
    rows |= set(range(0, 300)) | set(range(n - 300, n))
    # rows whose nonzeros sit past byte offset 2^31 of the fp64 values and 2^32 of any copy
    for e in (2 ** 28, 2 ** 29, 2 ** 30 // 2 * 3):
        if e < rp[-1]:
            r = int(np.searchsorted(rp, e, side="right") - 1)
            rows |= set(range(max(0, r - 50), min(n, r + 50)))
    return np.array(sorted(rows), dtype=np.int64)


def _sub_csr(A, rows):
    n, rp, ci, val = A
    lens = rp[rows + 1] - rp[rows]
    srp = np.zeros(len(rows) + 1, dtype=np.int32)
    np.cumsum(lens, out=srp[1:])
    idx = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows])
    return (len(rows), srp, ci[idx].astype(np.int32), val[idx])


def _check_rows(fmt, y, ref, absref):
    if fmt == 4:
        assert np.all(np.abs(y - ref) <= 1e-14 * absref + 1e-300)
    elif fmt == 3:
        assert np.all(np.abs(y - ref) <= 64 * 2.0 ** -24 * absref)
    else:
        # correctly rounded row sums: equal to the oracle's fp64-sum rounding
        assert np.mean(y == ref) >= 0.9999, (fmt, np.flatnonzero(y != ref)[:5])
        assert np.all(np.abs(y - ref) <= np.abs(ref) * 2.0 ** (1 - T_BITS[fmt]) + 1e-300)


@pytest.mark.parametrize("sched,lanes", [(0, 1), (0, 2), (2, 1), (1, 2), (1, 4)])
def test_fullsize_spmv_sampled_rows(big, sched, lanes):
    M, A, xs, b, ctx, mat = big
    n = A[0]
    rows = _sample_rows(A)
    sub = _sub_csr(A, rows)
    absub = (sub[0], sub[1], sub[2], np.abs(sub[3]))
    x = np.random.default_rng(1).uniform(-1, 1, n)
    xd = torch.as_tensor(x).cuda()
    yd = torch.empty_like(xd)
    # orc_spmv over the sampled rows reads the full vector through their column indices
    for fmt in range(8):
        try:
            mat.set_schedule(fmt, sched, lanes)
        except M.MpcgError:
            continue  # this tile size does not fit the stream schedule's stage
        ctx.spmv(mat, fmt, xd, yd)
        y = yd.cpu().numpy()[rows]
        ref = _oracle_rows(sub, fmt, x)
        base = fmt if fmt < 5 or fmt == 7 else (1 if fmt == 5 else 0)
        absref = _oracle_rows(absub, 4, np.abs(O.chop(x, base)))
        _check_rows(fmt, y, ref, absref)
        mat.set_schedule(fmt, 0, 1)


def _oracle_rows(sub, fmt, x):
    m, srp, sci, sval = sub
    q = np.empty(m)
    # the oracle's product on a row subset: orc_spmv loops over the m rows and gathers x
    L = O.lib()
    import ctypes as C

    L.orc_spmv(m, srp.ctypes.data_as(C.c_void_p), sci.ctypes.data_as(C.c_void_p), sval.ctypes.data_as(C.c_void_p),
               fmt, np.ascontiguousarray(x).ctypes.data_as(C.c_void_p), q.ctypes.data_as(C.c_void_p))
    return q


def test_fullsize_solve_properties(big):
    """Autotuned all-fp64 and mixed solves at full size: the reported true residual equals
    ||b - A x|| / ||b|| recomputed by scipy, the fp64 solve reaches 1e-8, and the mixed
    schedule with residual confirmation reaches it too."""
    import scipy.sparse as sp

    M, A, xs, b, ctx, mat = big
    n, rp, ci, val = A
    mat.autotune(3)
    S = sp.csr_matrix((val, ci, rp), shape=(n, n))
    bd = torch.as_tensor(b).cuda()
    for fmts in ((4, 4, 4, 4), None):
        pol = ctx.policy_fixed(fmts) if fmts else ctx.policy_schedule([(0, 0, 3, 3)] * 60 + [(3, 3, 3, 3)] * 120 +
                                                                       [(4, 4, 4, 4)] * 5000)
        x = torch.zeros_like(bd)
        res, hist = ctx.solve(mat, bd, x, 1e-8, 6000, pol, history_cap=6000)
        xh = x.cpu().numpy()
        true = np.linalg.norm(b - S @ xh) / np.linalg.norm(b)
        assert res["outcome"] == M.CONVERGED
        assert true < 1e-8
        assert res["rel_res_true"] == pytest.approx(true, rel=1e-6)
        rho = hist["rho"][: res["iters"]]
        assert np.all(np.isfinite(rho)) and rho[-1] < 1e-8
