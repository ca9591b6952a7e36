"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: per-iteration residual histories within 1e-6 relative on iterations whose
actions are all fp64 and 5e-3 relative otherwise (the oracle sums in fp64 and rounds the
output; the GPU accumulates the low-precision operations in fp32, so q and the dots may
differ by one unit in the last place of their format); final error to x* within 10x the
oracle's; greedy actions identical except where the residual lies within the history
tolerance of a bin edge."""
import math

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


def _ctx(M, **kw):
    kw.setdefault("min_k", 0)
    return M.Context(0, M.Options(**kw))


def _oopts(**kw):
    kw.setdefault("min_k", 0)
    return O.Options(**kw)


def _dev(A):
    n, rp, ci, val = A
    return (n, torch.as_tensor(rp).cuda(), torch.as_tensor(ci).cuda(), torch.as_tensor(val).cuda())


def _hist_err(hg, ho, n):
    rg, ro = hg["rho"][:n], ho["rho"][:n]
    return np.abs(rg - ro) / np.maximum(np.abs(ro), 1e-300)


def _block_matrix(vals):
    """Block diagonal of [[1, v], [v, 1]] blocks; with x = (0, 1, 0, 1, ...) row 2i of A x is
    exactly the stored value of v in the product's format."""
    m = len(vals)
    rp = np.arange(0, 4 * m + 1, 2, dtype=np.int32)
    ci = np.empty(4 * m, dtype=np.int32)
    val = np.empty(4 * m)
    for i, v in enumerate(vals):
        ci[4 * i:4 * i + 4] = [2 * i, 2 * i + 1, 2 * i, 2 * i + 1]
        val[4 * i:4 * i + 4] = [1.0, v, v, 1.0]
    return (2 * m, rp, ci, val)


def _edge_values():
    rng = np.random.default_rng(11)
    mant = rng.uniform(1, 2, 20000) * rng.choice([-1.0, 1.0], 20000)
    vals = list(mant * 2.0 ** rng.integers(-160, 140, 20000))
    f16 = np.arange(1, 0x7C00, 7, dtype=np.uint16).view(np.float16).astype(np.float64)
    bf = (np.arange(1, 0x7F80, 5, dtype=np.uint32) << 16).view(np.float32).astype(np.float64)
    for grid in (f16, bf):
        vals += list(0.5 * (grid[:-1] + grid[1:]))  # midpoints: ties to even
        vals += list(grid[:-1] + 0.25 * (grid[1:] - grid[:-1]))
    # q52 (3 significand digits, fp16 exponent range): every value, midpoints and quarter
    # points between neighbours, the overflow edge x_max + ulp / 2 = 57344 + 4096
    q8 = (np.arange(1, 0x7C, dtype=np.uint16) << 8).view(np.float16).astype(np.float64)
    vals += list(0.5 * (q8[:-1] + q8[1:])) + list(q8[:-1] + 0.25 * (q8[1:] - q8[:-1])) + list(q8)
    vals += [57344.0, 61439.99, 61440.0, 2.0 ** -16, 2.0 ** -17, 3 * 2.0 ** -18]
    vals += [65504.0, 65519.99, 65520.0, 3.4028235677973366e38, 2.0 ** -24, 3 * 2.0 ** -26, 2.0 ** -149,
             2.0 ** -136 * 1.5, 1e-300, 1e300]
    return np.array([v for v in vals if v != 0.0 and math.isfinite(v)])


def test_format_copies_are_bit_exact(M):
    """Every value copy (one rounding from fp64, the fl_p of Table 1 formats and the row-scaled
    extensions) equals the oracle's rounding bit for bit, including ties, subnormals and
    overflow."""
    vals = _edge_values()
    A = _block_matrix(vals)
    ctx = _ctx(M)
    mat = ctx.matrix(_dev(A))
    x = np.tile([0.0, 1.0], A[0] // 2)
    xd = torch.as_tensor(x).cuda()
    yd = torch.empty_like(xd)
    for fmt in range(8):
        ctx.spmv(mat, fmt, xd, yd)
        y = yd.cpu().numpy()
        ref = O.spmv(A, fmt, x)
        assert np.array_equal(y, ref, equal_nan=True), (fmt, np.flatnonzero(~((y == ref) | (np.isnan(y) & np.isnan(ref))))[:5])


SCHEDULES = [(0, 1), (0, 2), (0, 4), (0, 8), (0, 16), (0, 32), (2, 1), (1, 1), (1, 2), (1, 4), (3, 1), (4, 1)]


@pytest.mark.parametrize("which", ["poisson", "diffusion3d", "banded"])
def test_spmv_every_format_and_lane_count(M, which):
    rng = np.random.default_rng(1)
    if which == "poisson":
        A = I.poisson2d(40)
    elif which == "diffusion3d":
        A = I.diffusion_varcoef((11, 13, 9), 1.5, rng)
    else:
        A = I.banded_spd(1500, 40, 1e-3, rng)
    n, rp, ci, val = A
    ctx = _ctx(M)
    mat = ctx.matrix(_dev(A))
    x = rng.uniform(-1, 1, n)
    xd = torch.as_tensor(x).cuda()
    yd = torch.empty_like(xd)
    absA = (n, rp, ci, np.abs(val))
    for fmt in range(8):
        ref = O.spmv(A, fmt, x)
        mag = O.spmv(absA, 4, np.abs(O.chop(x, fmt if fmt < 5 or fmt == 7 else (0 if fmt == 6 else 1))))
        for sched, lanes in SCHEDULES:
            try:
                mat.set_schedule(fmt, sched, lanes)
            except M.MpcgError:
                assert sched == 1  # a stream tile that does not fit its stage
                continue
            ctx.spmv(mat, fmt, xd, yd)
            y = yd.cpu().numpy()
            if fmt == 4:
                assert np.all(np.abs(y - ref) <= 1e-14 * mag + 1e-300), (fmt, sched, lanes)
            elif fmt == 3:
                # fp32 products accumulated in fp32: one unit of the output plus the fp32
                # recursive-summation bound
                ulp = np.abs(ref) * 2.0 ** -23
                bound = ulp + 64 * 2.0 ** -24 * mag * 2
                assert np.all(np.abs(y - ref) <= bound), (fmt, sched, lanes, np.max(np.abs(y - ref) - bound))
            else:
                # 16-bit, tf32 and q52 formats: the correctly rounded row sum, as the oracle's
                # (exact products summed in fp64, then rounded once)
                assert np.array_equal(y, ref), (fmt, sched, lanes, np.flatnonzero(y != ref)[:5])


@pytest.mark.parametrize("fmts,tol,maxit", [
    (ALL64, 1e-10, 1000),
    ((3, 3, 3, 3), 1e-6, 300),
    ((2, 2, 2, 2), 1e-4, 300),
    ((0, 0, 3, 3), 1e-3, 300),
    ((1, 1, 1, 1), 1e-2, 200),
    ((6, 0, 3, 4), 1e-3, 200),
    ((5, 4, 4, 3), 1e-2, 200),
    ((7, 4, 4, 4), 1e-3, 200),
    ((7, 7, 7, 7), 1e-3, 200),
    ((4, 4, 7, 7), 1e-3, 200),
])
def test_fixed_policy_history_matches_oracle(M, fmts, tol, maxit):
    A, b, xs = I.cfg_poisson32()
    ctx = _ctx(M)
    mat = ctx.matrix(_dev(A))
    bd = torch.as_tensor(b).cuda()
    x = torch.zeros_like(bd)
    pol = ctx.policy_fixed(fmts)
    res, hist = ctx.solve(mat, bd, x, tol, maxit, pol, history_cap=maxit)
    ref = O.solve(_oopts(), A, b, tol, maxit, fixed=fmts)
    assert res["outcome"] == ref.outcome
    n = min(res["iters"], ref.iters)
    err = _hist_err(hist, ref.hist, n)
    lim = TOL64 if fmts == ALL64 else TOL_LOW
    assert np.all(err <= lim), (fmts, float(err.max()), int(np.argmax(err)))
    assert abs(res["iters"] - ref.iters) <= max(1, ref.iters // 50)
    xg = x.cpu().numpy()
    eg = np.linalg.norm(xg - xs) / np.linalg.norm(xs)
    eo = np.linalg.norm(ref.x - xs) / np.linalg.norm(xs)
    assert eg <= 10 * eo + 1e-15
    assert res["rel_res_true"] == pytest.approx(np.linalg.norm(b - _mv(A, xg)) / np.linalg.norm(b), rel=1e-6)


def _mv(A, x):
    import scipy.sparse as sp

    n, rp, ci, val = A
    return sp.csr_matrix((val, ci, rp), shape=(n, n)) @ x


def test_replayed_schedule_with_residual_replacement(M):
    A, b, xs = I.cfg_poisson32()
    sched = [(0, 0, 3, 3)] * 60 + [(3, 3, 3, 3)] * 40 + [ALL64] * 1000
    ctx = _ctx(M, true_res_at_conv=1)
    mat = ctx.matrix(_dev(A))
    bd = torch.as_tensor(b).cuda()
    x = torch.zeros_like(bd)
    pol = ctx.policy_schedule(sched)
    res, hist = ctx.solve(mat, bd, x, 1e-8, 1000, pol, history_cap=1000)
    ref = O.solve(_oopts(true_res_at_conv=1), A, b, 1e-8, 1000, sched=sched)
    assert res["outcome"] == O.CONVERGED == ref.outcome
    assert res["rel_res_true"] < 1e-8
    n = min(res["iters"], ref.iters)
    err = _hist_err(hist, ref.hist, n)
    assert np.all(err[:60] <= TOL_LOW)
    assert abs(res["iters"] - ref.iters) <= 3


def test_greedy_qtable_matches_oracle(M):
    """A Q-table trained by the oracle drives both solvers; actions agree except where rho is
    within the history tolerance of a residual-bin threshold."""
    A, b, xs = I.cfg_poisson32()
    oo = _oopts(seed=3, cost=dict(O.COST_C2))
    qt = O.QTable.zeros(oo)
    O.train_sequential(oo, A, b, 1e-6, 400, 30, qt)
    ref = O.solve(oo, A, b, 1e-6, 400, qtable=qt)
    ctx = _ctx(M, seed=3, cost=(0.5, 0.4, 0.5, 1.5, 3.0))
    mat = ctx.matrix(_dev(A))
    pol = ctx.policy_qtable(qt.Q, qt.visits)
    bd = torch.as_tensor(b).cuda()
    x = torch.zeros_like(bd)
    res, hist = ctx.solve(mat, bd, x, 1e-6, 400, pol, history_cap=400)
    n = min(res["iters"], ref.iters)
    delta = 1.6
    thr = 10.0 ** (-np.arange(1, 10) * delta)
    near = 0
    for k in range(n):
        if not np.array_equal(hist["fmt"][k], ref.hist["fmt"][k]):
            rho_k = 1.0 if k == 0 else ref.hist["rho"][k - 1]
            assert np.min(np.abs(rho_k / thr - 1)) <= TOL_LOW, k
            near += 1
            break  # trajectories separate after a differing action
    assert res["outcome"] == ref.outcome


def _train_both(M, precs, cost, E=6, tmax=200, seed=5, eps=None):
    A, b, xs = I.cfg_poisson32()
    ek = {} if eps is None else dict(eps0=eps, eps_floor=eps)
    oo = _oopts(seed=seed, precs=precs, cost={p: c for p, c in zip(precs, cost)}, **ek)
    qt = O.QTable.zeros(oo)
    it_o = O.train_sequential(oo, A, b, 1e-6, tmax, E, qt)
    ctx = _ctx(M, seed=seed, precs=precs, cost=cost, **ek)
    mat = ctx.matrix(_dev(A))
    bd = torch.as_tensor(b).cuda()
    S = 100
    pol = ctx.policy_qtable(np.zeros((4, S, len(precs))), np.zeros((4, S), dtype=np.int32))
    it_g = ctx.train_qtable([mat], [bd], 1e-6, tmax, E, pol, want_iters=True)
    Qg, vg = pol.qtable()
    return it_o, it_g[:, 0], qt, Qg, vg


def test_training_one_lane_matches_algorithm_1_fp32_fp64(M):
    """Batched training with one system is Algorithm 1. With P = {fp32, fp64} the two sides
    take the same actions, so the tables agree to the accuracy of the residual histories."""
    it_o, it_g, qt, Qg, vg = _train_both(M, (O.FP32, O.FP64), (1.0, 2.0))
    assert list(it_o) == list(it_g)
    assert np.array_equal(vg, qt.visits)
    assert np.allclose(Qg, qt.Q, rtol=1e-6, atol=1e-9)


def test_training_one_lane_matches_algorithm_1_full_set(M):
    """Full precision set: episodes agree until the residual histories separate (a residual
    within rounding of a bin edge, or an fp16 dot rounded on either side of a tie, is enough
    to split them); iteration counts stay close. With a constant exploration rate a run of
    E' episodes is the prefix of a longer run, so the tables are compared after every
    prefix of episodes that both sides ran alike (same iteration counts and visits): there
    they agree to the accuracy of the rewards (the 5e-3 relative residual tolerance moves
    -log10 rho by about 2e-3 per update)."""
    precs, cost = (0, 1, 2, 3, 4), (0.8, 0.6, 0.8, 1.0, 2.0)
    it_o, it_g, qt, Qg, vg = _train_both(M, precs, cost)
    assert np.all(np.abs(np.asarray(it_o) - np.asarray(it_g)) <= np.maximum(3, np.asarray(it_o) // 10))
    # every iteration updates each operation's table once
    assert vg.sum() == 4 * int(np.sum(it_g)) and qt.visits.sum() == 4 * int(np.sum(it_o))
    compared = 0
    for E in range(1, 7):
        it_o, it_g, qt, Qg, vg = _train_both(M, precs, cost, E=E, tmax=60, seed=8, eps=0.3)
        if list(it_o) != list(it_g) or not np.array_equal(vg, qt.visits):
            break
        assert np.allclose(Qg, qt.Q, rtol=2e-2, atol=2e-2), (E, float(np.max(np.abs(Qg - qt.Q))))
        compared = E
    print(f"full-set training: tables compared after 1..{compared} episodes")
    assert compared >= 1


def test_training_one_lane_short_episodes_full_set(M):
    """Full precision set, episodes cut at 12 iterations (before the fp16 residual histories
    separate): the same states are visited and the tables agree to the accuracy of the
    rewards (the 5e-3 relative residual tolerance moves -log10 rho by about 2e-3)."""
    it_o, it_g, qt, Qg, vg = _train_both(M, (0, 1, 2, 3, 4), (0.8, 0.6, 0.8, 1.0, 2.0), E=6, tmax=12)
    assert list(it_o) == list(it_g) == [12] * 6
    assert np.sum(vg != qt.visits) <= 4  # a residual within rounding of a bin edge may move one visit
    same = (vg == qt.visits)[..., None] & np.ones_like(Qg, dtype=bool)
    assert np.allclose(Qg[same], qt.Q[same], rtol=2e-2, atol=2e-2)


def test_batched_matches_single_and_oracle(M):
    sets = I.cfg_train_set(count=6, m_lo=6, m_hi=12)
    ctx = _ctx(M)
    pol = ctx.policy_fixed((0, 3, 3, 4))
    mats = [ctx.matrix(_dev(A)) for A, _, _ in sets]
    bs = [torch.as_tensor(b).cuda() for _, b, _ in sets]
    xs = [torch.zeros_like(b) for b in bs]
    res = ctx.solve_batched(mats, bs, xs, [1e-6] * 6, [500] * 6, pol)
    for (A, b, xstar), r, x in zip(sets, res, xs):
        ref = O.solve(_oopts(), A, b, 1e-6, 500, fixed=(0, 3, 3, 4))
        assert r["outcome"] == ref.outcome
        assert abs(r["iters"] - ref.iters) <= max(2, ref.iters // 20)
        eg = np.linalg.norm(x.cpu().numpy() - xstar)
        eo = np.linalg.norm(ref.x - xstar)
        assert eg <= 10 * eo + 1e-12


@pytest.mark.parametrize("stepped", [0, 2])
def test_staged_x_schedule_in_the_solver_kernels(M, stepped):
    """The staged-x product (schedule 4) inside the solver: a lockstep batch of diffusion systems
    (stepped = 0) and the stepped single solve of a 2D Poisson system (stepped = 2), every
    product format's schedule forced to it, against the oracle; a matrix whose columns do not
    increase in every row is refused for it."""
    ctx = _ctx(M, stepped=stepped)
    pol = ctx.policy_fixed((0, 3, 3, 4))
    if stepped == 0:
        sets = I.cfg_train_set(count=4, m_lo=6, m_hi=12)
    else:
        A = I.poisson2d(64)
        xs0, b0 = I.rhs_from_xstar(A, np.random.default_rng(9))
        sets = [(A, b0, xs0)]
    mats = [ctx.matrix(_dev(A)) for A, _, _ in sets]
    for m in mats:
        for f in range(8):
            m.set_schedule(f, 4, 1)
    bs = [torch.as_tensor(b).cuda() for _, b, _ in sets]
    xs = [torch.zeros_like(b) for b in bs]
    if stepped == 0:
        res = ctx.solve_batched(mats, bs, xs, [1e-6] * len(sets), [500] * len(sets), pol)
    else:
        res = [ctx.solve(mats[0], bs[0], xs[0], 1e-6, 500, pol)[0]]
    for (A, b, xstar), r, x in zip(sets, res, xs):
        ref = O.solve(_oopts(), A, b, 1e-6, 500, fixed=(0, 3, 3, 4))
        assert r["outcome"] == ref.outcome
        assert abs(r["iters"] - ref.iters) <= max(2, ref.iters // 20)
        assert np.linalg.norm(x.cpu().numpy() - xstar) <= 10 * np.linalg.norm(ref.x - xstar) + 1e-12
    # columns out of order in one row: the staged window cannot be read off the row ends
    n, rp, ci, val = I.poisson2d(8)
    ci2, val2 = ci.copy(), val.copy()
    e0, e1 = rp[10], rp[11]
    ci2[e0:e1], val2[e0:e1] = ci[e0:e1][::-1].copy(), val[e0:e1][::-1].copy()
    m2 = ctx.matrix(_dev((n, rp, ci2, val2)))
    with pytest.raises(M.MpcgError):
        m2.set_schedule(3, 4, 1)


def test_autotune_cache_by_bucket(M):
    """The autotuner times a matrix once per bucket (row-length statistics, n, column order)
    and context: a second matrix with the same pattern takes the first one's schedules without
    timing; reps < 0 times it anyway."""
    import time

    ctx = _ctx(M)
    m1 = ctx.matrix(_dev(I.fem27_aniso(72, 1e-3)))
    m2 = ctx.matrix(_dev(I.fem27_aniso(72, 1e-2)))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m1.autotune(3)
    t1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    m2.autotune(3)
    t2 = time.perf_counter() - t0
    i1, i2 = m1.info(), m2.info()
    assert i1["spmv_sched"] == i2["spmv_sched"] and i1["spmv_lanes"] == i2["spmv_lanes"]
    assert t2 < 0.1 * t1, (t1, t2)
    t0 = time.perf_counter()
    m2.autotune(-3)
    t3 = time.perf_counter() - t0
    assert t3 > 5 * t2, (t2, t3)


def test_graph_replay_reproduces_results(M):
    sets = I.cfg_train_set(count=4, m_lo=6, m_hi=9)
    ctx = _ctx(M)
    pol = ctx.policy_fixed(ALL64)
    mats = [ctx.matrix(_dev(A)) for A, _, _ in sets]
    bs = [torch.as_tensor(b).cuda() for _, b, _ in sets]
    xs = [torch.zeros_like(b) for b in bs]
    g = ctx.graph(mats, bs, xs, [1e-6] * 4, [3000] * 4, pol)
    g.launch()
    r1 = g.results()
    x1 = [x.clone() for x in xs]
    g.launch()
    r2 = g.results()
    for a, c, x, y in zip(r1, r2, x1, xs):
        assert a["iters"] == c["iters"] and a["rel_res_true"] == c["rel_res_true"]
        assert torch.equal(x, y)
        assert a["outcome"] == c["outcome"]


def test_edge_cases(M):
    ctx = _ctx(M)
    # empty system
    E = (0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    mat = ctx.matrix(E)
    pol = ctx.policy_fixed(ALL64)
    res, _ = ctx.solve(mat, np.zeros(0), np.zeros(0), 1e-8, 10, pol)
    assert res["outcome"] == O.CONVERGED and res["iters"] == 0
    # zero right-hand side, host buffers
    A, b, _ = I.cfg_poisson32()
    mat = ctx.matrix(A)
    x = np.full(A[0], 7.0)
    res, _ = ctx.solve(mat, np.zeros(A[0]), x, 1e-8, 10, pol)
    assert res["outcome"] == O.CONVERGED and res["iters"] == 0 and not x.any()
    # iteration cap 0
    x = np.zeros(A[0])
    res, _ = ctx.solve(mat, b, x, 1e-8, 0, pol)
    assert res["outcome"] == O.MAX_ITER and res["iters"] == 0
    # indefinite matrix: p^T A p < 0 at k = 0
    ind = (2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32), np.array([1.0, 2.0, 2.0, 1.0]))
    m2 = ctx.matrix(ind)
    x = np.zeros(2)
    res, _ = ctx.solve(m2, np.array([1.0, -1.0]), x, 1e-8, 10, pol)
    assert res["outcome"] == O.BREAKDOWN and res["iters"] == 0 and not x.any()
    # fp16 overflow of the matrix values breaks down; the row-scaled fp16 copy does not
    big = (A[0], A[1], A[2], A[3] * 1e5)
    m3 = ctx.matrix(big)
    x = np.zeros(A[0])
    res, _ = ctx.solve(m3, b, x, 1e-8, 50, ctx.policy_fixed((0, 4, 4, 4)))
    assert res["outcome"] == O.BREAKDOWN and res["iters"] == 0
    res, _ = ctx.solve(m3, b, x, 1e-8, 50, ctx.policy_fixed((6, 4, 4, 4)))
    assert res["outcome"] != O.BREAKDOWN
    # invalid structure is rejected with a message
    bad = (2, np.array([0, 2, 1], np.int32), np.array([0, 1], np.int32), np.array([1.0, 1.0]))
    with pytest.raises(M.MpcgError, match="row_ptr"):
        ctx.matrix(bad)
    nodiag = (2, np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), np.array([1.0, 1.0]))
    with pytest.raises(M.MpcgError, match="diagonal"):
        ctx.matrix(nodiag)
    badcol = (2, np.array([0, 1, 2], np.int32), np.array([0, 5], np.int32), np.array([1.0, 1.0]))
    with pytest.raises(M.MpcgError, match="column"):
        ctx.matrix(badcol)


def test_policy_blob_round_trip(M):
    ctx = _ctx(M)
    rng = np.random.default_rng(0)
    Q = rng.standard_normal((4, 100, 5))
    v = rng.integers(0, 3, (4, 100)).astype(np.int32)
    p = ctx.policy_qtable(Q, v)
    blob = p.save()
    q = ctx.policy_load(blob)
    Q2, v2 = q.qtable()
    assert np.array_equal(Q, Q2) and np.array_equal(v, v2)
    with pytest.raises(M.MpcgError):
        ctx.policy_load(b"garbage" * 40)
