"""The stepped single solve (one kernel per phase of the iteration, repeated on the device by a
conditional while-loop CUDA graph) against the CPU oracle and against the persistent launch,
through the C ABI.

Tolerances as in the other parity tests: residual histories within 1e-6 relative on all-fp64
iterations and 5e-3 otherwise, final error to x* within 10x the oracle's. Against the
persistent launch (same arithmetic, other CTA partition of the sums): fp64 histories within
1e-9 relative and the same iteration count."""
import numpy as np
import pytest

import oracle as O
from paper_2504_14268_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALL64 = (4, 4, 4, 4)
TOL64, TOL_LOW = 1e-6, 5e-3


@pytest.fixture(scope="module")
def M():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2504_14268_gb300 import mpcg

    return mpcg


def _dev(A):
    n, rp, ci, val = A
    return (n, torch.as_tensor(rp).cuda(), torch.as_tensor(ci).cuda(), torch.as_tensor(val).cuda())


def _solve(M, A, b, fmts, tol, cap, stepped, sched=None, **kw):
    kw.setdefault("min_k", 0)
    ctx = M.Context(0, M.Options(stepped=stepped, **kw))
    mat = ctx.matrix(_dev(A))
    if sched is not None:
        for f in sched[0]:
            mat.set_schedule(f, *sched[1])
    pol = ctx.policy_fixed(fmts)
    bd = torch.as_tensor(b).cuda()
    x = torch.zeros_like(bd)
    res, hist = ctx.solve(mat, bd, x, tol, cap, pol, history_cap=cap)
    return res, hist, x.cpu().numpy()


@pytest.mark.parametrize("case", ["poisson32", "fem24"])
@pytest.mark.parametrize("fmts,tol", [(ALL64, 1e-10), ((3, 3, 3, 3), 1e-6), ((0, 0, 3, 3), 1e-3),
                                      ((6, 4, 3, 4), 1e-3)])
def test_stepped_fixed_policy_matches_oracle_and_persistent(M, case, fmts, tol):
    if case == "poisson32":
        A, b, xs = I.cfg_poisson32()
    else:
        A = I.fem27_aniso(24, 1e-2)
        xs, b = I.rhs_from_xstar(A, np.random.default_rng(5))
    cap = 600
    res, hist, x = _solve(M, A, b, fmts, tol, cap, stepped=2)
    ref = O.solve(O.Options(min_k=0), A, b, tol, cap, fixed=fmts)
    assert res["outcome"] == ref.outcome
    n = min(res["iters"], ref.iters)
    err = np.abs(hist["rho"][:n] - ref.hist["rho"][:n]) / np.abs(ref.hist["rho"][:n])
    assert np.all(err <= (TOL64 if fmts == ALL64 else TOL_LOW)), (float(err.max()), int(np.argmax(err)))
    assert abs(res["iters"] - ref.iters) <= max(1, ref.iters // 50)
    eg = np.linalg.norm(x - xs) / np.linalg.norm(xs)
    eo = np.linalg.norm(ref.x - xs) / np.linalg.norm(xs)
    assert eg <= 10 * eo + 1e-15
    # the persistent launch: same iterations; fp64 histories agree to the reduction order
    rp_, hp, xp = _solve(M, A, b, fmts, tol, cap, stepped=1)
    if fmts == ALL64:
        assert rp_["iters"] == res["iters"]
        m = res["iters"]
        assert np.all(np.abs(hp["rho"][:m] - hist["rho"][:m]) <= 1e-9 * hist["rho"][:m])
    assert np.all(hist["ns_a"][:n] > 0) and np.all(hist["ns_b"][:n] > 0)
    # launches: one persistent kernel; the graph runs four phase kernels and the control
    # kernel per pass, at least one pass per iteration plus the initialisation
    assert rp_["kernel_launches"] == 1
    assert res["kernel_launches"] % 5 == 0 and res["kernel_launches"] >= 5 * (res["iters"] + 1)


def test_stepped_greedy_qtable_with_replacement_and_restart(M):
    """A Q-table policy with the benchmark's options (true residual at a claimed convergence,
    fp64 restart after a breakdown): the stepped and the persistent launch take the same
    decisions and reach the same iteration count."""
    A = I.fem27_aniso(32, 1e-3)
    xs, b = I.rhs_from_xstar(A, np.random.default_rng(0))
    oo = O.Options(t_bin=5000, op_mask=(0b11000,) * 4, true_res_at_conv=1, on_breakdown=1, seed=3)
    qt = O.QTable.zeros(oo)
    for i, m in enumerate((10, 12)):
        At = I.fem27_aniso(m, 1e-3)
        _, bt = I.rhs_from_xstar(At, np.random.default_rng(100 + i))
        O.train_sequential(oo, At, bt, 1e-8, 5000, 10, qt, ep_base=i * 10)
    out = {}
    for stepped in (1, 2):
        ctx = M.Context(0, M.Options(t_bin=5000, op_mask=(0b11000,) * 4, true_res_at_conv=1, on_breakdown=1, seed=3,
                                     stepped=stepped))
        mat = ctx.matrix(_dev(A))
        pol = ctx.policy_qtable(qt.Q, qt.visits)
        bd = torch.as_tensor(b).cuda()
        x = torch.zeros_like(bd)
        res, hist = ctx.solve(mat, bd, x, 1e-8, 3000, pol, history_cap=3000)
        out[stepped] = (res, hist, x.cpu().numpy())
    (r1, h1, x1), (r2, h2, x2) = out[1], out[2]
    assert r1["outcome"] == r2["outcome"] == O.CONVERGED
    assert r1["iters"] == r2["iters"] and r2["rel_res_true"] < 1e-8
    k = r2["iters"]
    same = np.all(h1["fmt"][:k] == h2["fmt"][:k], axis=1)
    assert np.mean(same) > 0.98
    assert np.all(np.flatnonzero(h2["flags"][:k] & 4) == np.flatnonzero(h1["flags"][:k] & 4))
    assert np.linalg.norm(x2 - xs) <= 10 * np.linalg.norm(x1 - xs)


def test_stepped_edge_cases(M):
    ctx = M.Context(0, M.Options(min_k=0, stepped=2))
    pol = ctx.policy_fixed(ALL64)
    E = (0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    res, _ = ctx.solve(ctx.matrix(E), np.zeros(0), np.zeros(0), 1e-8, 10, pol)
    assert res["outcome"] == O.CONVERGED and res["iters"] == 0
    A, b, _ = I.cfg_poisson32()
    mat = ctx.matrix(A)
    x = np.full(A[0], 7.0)
    res, _ = ctx.solve(mat, np.zeros(A[0]), x, 1e-8, 10, pol)
    assert res["outcome"] == O.CONVERGED and res["iters"] == 0 and not x.any()
    x = np.zeros(A[0])
    res, _ = ctx.solve(mat, b, x, 1e-8, 0, pol)
    assert res["outcome"] == O.MAX_ITER and res["iters"] == 0
    x = np.zeros(A[0])
    res, _ = ctx.solve(mat, b, x, 1e-30, 25, pol)
    assert res["outcome"] == O.MAX_ITER and res["iters"] == 25
    ind = (2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32), np.array([1.0, 2.0, 2.0, 1.0]))
    x = np.zeros(2)
    res, _ = ctx.solve(ctx.matrix(ind), np.array([1.0, -1.0]), x, 1e-8, 10, pol)
    assert res["outcome"] == O.BREAKDOWN and res["iters"] == 0 and not x.any()
    # fp16 overflow of the values: breakdown, and with the fp64 restart option a converged solve
    big = (A[0], A[1], A[2], A[3] * 1e5)
    x = np.zeros(A[0])
    res, _ = ctx.solve(ctx.matrix(big), b, x, 1e-8, 50, ctx.policy_fixed((0, 4, 4, 4)))
    assert res["outcome"] == O.BREAKDOWN
    ctx2 = M.Context(0, M.Options(min_k=0, stepped=2, on_breakdown=1))
    x = np.zeros(A[0])
    res, h = ctx2.solve(ctx2.matrix(big), b, x, 1e-8, 500, ctx2.policy_fixed((0, 4, 4, 4)), history_cap=500)
    ref = O.solve(O.Options(min_k=0, on_breakdown=1), big, b, 1e-8, 500, fixed=(0, 4, 4, 4))
    assert res["outcome"] == ref.outcome == O.CONVERGED and res["n_restarts"] == 1
    assert abs(res["iters"] - ref.iters) <= 1


def test_stepped_replacement_stream_schedule_and_jacobi(M):
    A, b, xs = I.cfg_poisson32()
    sched = [(0, 0, 3, 3)] * 60 + [(3, 3, 3, 3)] * 40 + [ALL64] * 1000
    ctx = M.Context(0, M.Options(min_k=0, true_res_at_conv=1, true_res_every=25, stepped=2))
    mat = ctx.matrix(_dev(A))
    pol = ctx.policy_schedule(sched)
    bd = torch.as_tensor(b).cuda()
    x = torch.zeros_like(bd)
    res, hist = ctx.solve(mat, bd, x, 1e-8, 1000, pol, history_cap=1000)
    ref = O.solve(O.Options(min_k=0, true_res_at_conv=1, true_res_every=25), A, b, 1e-8, 1000, sched=sched)
    assert res["outcome"] == O.CONVERGED == ref.outcome and res["rel_res_true"] < 1e-8
    err = np.abs(hist["rho"][:24] - ref.hist["rho"][:24]) / ref.hist["rho"][:24]
    assert np.all(err <= TOL_LOW)
    k = min(res["iters"], ref.iters)
    periodic = np.arange(24, k, 25)  # r replaced by b - A x after every 25th iteration
    assert np.all(hist["flags"][periodic] & 4) and np.all(ref.hist["flags"][periodic] & 4)
    # the staged stream product (dynamic shared memory ring) in the stepped product kernel
    Af = I.fem27_aniso(20, 1e-2)
    xf, bf = I.rhs_from_xstar(Af, np.random.default_rng(8))
    r1, h1, x1 = _solve(M, Af, bf, (3, 4, 3, 4), 1e-6, 400, stepped=2, sched=((3, 4), (1, 4)))
    ref = O.solve(O.Options(min_k=0), Af, bf, 1e-6, 400, fixed=(3, 4, 3, 4))
    n = min(r1["iters"], ref.iters)
    assert np.all(np.abs(h1["rho"][:n] - ref.hist["rho"][:n]) <= TOL_LOW * ref.hist["rho"][:n])
    # Jacobi
    rng = np.random.default_rng(4)
    Aj = I.diffusion_varcoef((14, 12, 10), 1.5, rng)
    _, bj = I.rhs_from_xstar(Aj, rng)
    r2, h2, _ = _solve(M, Aj, bj, ALL64, 1e-8, 3000, stepped=2, precond=1)
    ref = O.solve(O.Options(min_k=0, precond=1), Aj, bj, 1e-8, 3000, fixed=ALL64)
    assert r2["iters"] == ref.iters
    n = min(r2["iters"], 60)
    assert np.all(np.abs(h2["rho"][:n] - ref.hist["rho"][:n]) <= TOL64 * ref.hist["rho"][:n])
