"""GPU parity of the learned-policy paths against the CPU oracle (through the C ABI).

* Greedy tabular decisions (Algorithm 2) on the 27-point FEM family with the options of the
  single-large-solve benchmark: the GPU solves greedily, the oracle replays the GPU's
  action sequence, and every GPU decision is checked against the oracle's own greedy
  decision on the replayed residual history. Decisions may differ only where the residual
  lies within the history tolerance of a residual-bin edge; such decisions are counted by
  the library (mpcg_result.near_edge_count) and the count must cover every difference.
* Batched training rounds with several lanes (the lane-private episodes and the ordered
  replay) and one-lane training under a per-operation precision mask (Algorithm 1 with the
  bootstrap max over the allowed set).
* The Adam step of the MLP Q-function's optimiser from identical gradients.

Tolerances: residual histories 1e-6 relative on all-fp64 iterations and 5e-3 otherwise;
final error to x* within 10x the oracle's; tables within 1e-6 relative where the two sides
take the same actions."""
import numpy as np
import pytest

import oracle as O
from paper_2504_14268_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL_LOW = 1e-6, 5e-3
MASK_32_64 = (0b11000,) * 4
T_BIN = 5000


@pytest.fixture(scope="module")
def M():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2504_14268_gb300 import mpcg

    return mpcg


def _dev(A):
    n, rp, ci, val = A
    return (n, torch.as_tensor(rp).cuda(), torch.as_tensor(ci).cuda(), torch.as_tensor(val).cuda())


def _bench_options(**kw):
    """The single-large-solve benchmark's solver options (oracle side)."""
    return O.Options(t_bin=T_BIN, op_mask=MASK_32_64, true_res_at_conv=1, on_breakdown=1, seed=3, **kw)


def _oracle_table(oo, sizes, episodes):
    """Algorithm 1 in sequence on small systems of the 27-point family (oracle only)."""
    qt = O.QTable.zeros(oo)
    for i, (m, an) in enumerate(sizes):
        A = I.fem27_aniso(m, an)
        _, b = I.rhs_from_xstar(A, np.random.default_rng(100 + i))
        O.train_sequential(oo, A, b, 1e-8, T_BIN, episodes, qt, ep_base=i * episodes)
    return qt


def _near_edge(rho, r_bins=10, eps_min=1e-16, tol=TOL_LOW):
    delta = -np.log10(eps_min) / r_bins
    thr = 10.0 ** (-np.arange(1, r_bins) * delta)
    return bool(np.min(np.abs(rho / thr - 1.0)) <= tol)


@pytest.mark.parametrize("grid", [48, 64])
def test_greedy_parity_on_the_benchmark_family(M, grid):
    """Histories are compared element-wise up to the first residual replacement (flag 4, the
    fp64 b - A x at a claimed convergence): from there on the replaced residual carries the
    rounding gap that each side's earlier fp32 products left between the recursive residual
    and b - A x, which differs between two correctly rounding implementations by a relative
    amount of order one once the residual is near tau. The replacement must happen at the
    same iteration on both sides, and both must converge in fp64 within a few iterations."""
    oo = _bench_options()
    qt = _oracle_table(oo, [(10, 1e-3), (12, 1e-3), (14, 1e-2), (12, 3e-3)], 15)
    A = I.fem27_aniso(grid, 1e-3)
    xs, b = I.rhs_from_xstar(A, np.random.default_rng(0))
    ctx = M.Context(0, M.Options(t_bin=T_BIN, op_mask=MASK_32_64, true_res_at_conv=1, on_breakdown=1, seed=3))
    mat = ctx.matrix(_dev(A))
    mat.autotune(3)
    pol = ctx.policy_qtable(qt.Q, qt.visits)
    bd = torch.as_tensor(b).cuda()
    x = torch.zeros_like(bd)
    cap = 4000
    res, hist = ctx.solve(mat, bd, x, 1e-8, cap, pol, history_cap=cap)
    assert res["outcome"] == O.CONVERGED and res["rel_res_true"] < 1e-8
    it = res["iters"]
    h = hist[:it]
    assert set(np.unique(h["fmt"])) <= {3, 4}
    # the oracle replays the GPU's action sequence
    sched = np.array(h["fmt"], dtype=np.int32)
    ref = O.solve(oo, A, b, 1e-8, cap, sched=sched)
    assert ref.outcome == O.CONVERGED and ref.rho_true < 1e-8
    n = min(it, ref.iters)
    repl_g = np.flatnonzero(h["flags"][:n] & 4)
    repl_o = np.flatnonzero(ref.hist["flags"][:n] & 4)
    first = int(repl_g[0]) if len(repl_g) else n
    assert (int(repl_o[0]) if len(repl_o) else n) == first
    all64 = np.all(sched[:first] == 4, axis=1)
    err = np.abs(h["rho"][:first] - ref.hist["rho"][:first]) / np.abs(ref.hist["rho"][:first])
    lim = np.where(all64, TOL64, TOL_LOW)
    assert np.all(err <= lim), (int(np.argmax(err > lim)), float(err.max()))
    assert abs(it - ref.iters) <= 10
    # GPU decisions against the oracle's greedy decision: on the replayed history up to the
    # first replacement, and on the GPU's own residuals at every iteration (the decision
    # function alone; log10 bins against thresholds can differ only at an edge)
    diffs = 0
    rho_o, rho_g = 1.0, 1.0
    for k in range(it):
        gk = tuple(int(f) for f in h["fmt"][k])
        s, fm = O.greedy_action(oo, qt, k, rho_g)
        if fm != gk or s != int(h["state"][k]):
            assert _near_edge(rho_g), (k, rho_g, fm, gk)
        if k <= first and k < n:
            s, fm = O.greedy_action(oo, qt, k, rho_o)
            if fm != gk or s != int(h["state"][k]):
                assert _near_edge(rho_o), (k, rho_o, fm, gk)
                diffs += 1
            rho_o = ref.hist["rho"][k]
        rho_g = h["rho"][k]
    assert diffs <= res["near_edge_count"], (diffs, res["near_edge_count"])
    eg = np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs)
    eo = np.linalg.norm(ref.x - xs) / np.linalg.norm(xs)
    assert eg <= 10 * eo
    print(f"grid {grid}: {it} iterations (oracle replay {ref.iters}), fp32 share {np.mean(sched == 3):.2f}, "
          f"first replacement at {first}, max history error before it {err.max():.2e}, decisions differing "
          f"{diffs}, near-edge decisions {res['near_edge_count']}, error to x* {eg:.3g} / {eo:.3g}")


def _train_lanes(M, oo, precs, cost, sets, E, tmax, **mopts):
    ctx = M.Context(0, M.Options(min_k=oo.min_k, seed=oo.seed, precs=precs, cost=cost, op_mask=oo.op_mask,
                                 eps0=oo.eps0, eps_floor=oo.eps_floor, **mopts))
    mats = [ctx.matrix(_dev(A)) for A, _, _ in sets]
    bs = [torch.as_tensor(b).cuda() for _, b, _ in sets]
    S = oo.n_states
    pol = ctx.policy_qtable(np.zeros((4, S, len(precs))), np.zeros((4, S), dtype=np.int32))
    its = ctx.train_qtable(mats, bs, 1e-6, tmax, E, pol, want_iters=True)
    Qg, vg = pol.qtable()
    return its, Qg, vg


def test_training_round_with_four_lanes_matches_oracle(M):
    """Batched reading of Algorithm 1 with B = 4 lanes: every lane's episode on its private
    copy, then the replay of all transitions in lane order onto the round-start table. With
    P = {fp32, fp64} both sides take the same actions, so iteration counts and visits are
    equal and the tables agree to the accuracy of the residual histories. The lanes are
    well-conditioned systems (2D Poisson 20^2, 26^2, 32^2 and a 10^3 27-point FEM system),
    whose oracle trajectories do not move when b is perturbed by 1e-12 (on high-contrast
    diffusion systems one fp32 rounding apart is enough to change an episode's length)."""
    sets = []
    for i, m in enumerate((20, 26, 32)):
        A = I.poisson2d(m)
        xs, b = I.rhs_from_xstar(A, np.random.default_rng(40 + i))
        sets.append((A, b, xs))
    A = I.fem27_aniso(10, 1e-2)
    xs, b = I.rhs_from_xstar(A, np.random.default_rng(43))
    sets.append((A, b, xs))
    precs, cost = (O.FP32, O.FP64), (1.0, 2.0)
    # the product stays in fp64 (its fp32 form accumulates in fp32 on the GPU, so histories
    # drift apart by about 1e-5 over an episode); z and the two dots choose from {fp32, fp64}
    # and round alike on both sides, so the replay order is checked to rounding accuracy
    oo = O.Options(seed=9, min_k=0, precs=precs, cost={O.FP32: 1.0, O.FP64: 2.0}, op_mask=(0b10, 0b11, 0b11, 0b11))
    E, tmax = 8, 300
    qt = O.QTable.zeros(oo)
    it_o = np.array([O.train_round(oo, [s[0] for s in sets], [s[1] for s in sets], 1e-6, tmax, e, E, qt)
                     for e in range(1, E + 1)])
    it_g, Qg, vg = _train_lanes(M, oo, precs, cost, sets, E, tmax)
    assert np.array_equal(it_g, it_o), (it_g, it_o)
    assert np.array_equal(vg, qt.visits)
    assert np.allclose(Qg, qt.Q, rtol=1e-6, atol=1e-9), float(np.max(np.abs(Qg - qt.Q)))


def test_training_one_lane_under_an_operation_mask(M):
    """Algorithm 1 with one lane, the full precision set and every operation restricted to
    {fp32, fp64}: greedy choice, exploration and the bootstrap max run over the allowed
    entries, and the entries outside the mask are never updated on either side."""
    A, b, _ = I.cfg_poisson32()
    precs, cost = (0, 1, 2, 3, 4), (0.8, 0.6, 0.8, 1.0, 2.0)
    oo = O.Options(seed=7, min_k=0, op_mask=MASK_32_64)
    E, tmax = 8, 250
    qt = O.QTable.zeros(oo)
    it_o = O.train_sequential(oo, A, b, 1e-6, tmax, E, qt)
    it_g, Qg, vg = _train_lanes(M, oo, precs, cost, [(A, b, None)], E, tmax)
    assert list(it_g[:, 0]) == list(it_o)
    assert np.array_equal(vg, qt.visits)
    assert not Qg[:, :, :3].any() and not qt.Q[:, :, :3].any()
    assert np.allclose(Qg, qt.Q, rtol=1e-6, atol=1e-9), float(np.max(np.abs(Qg - qt.Q)))


def test_joint_table_training_and_greedy_match_oracle(M):
    """One Q-table over the joint actions (the |P|^4 alternative that Section 4.1 weighs):
    four-lane training rounds as in the per-operation test (same systems, same mask, so both
    sides take the same actions), tables [S][|P|^4] and per-state visits compared; then a
    greedy solve with the trained table on each lane system, every decision equal to the
    oracle's unless the library counted it as lying within the history tolerance of a
    residual-bin edge."""
    sets = []
    for i, m in enumerate((20, 26, 32)):
        A = I.poisson2d(m)
        xs, b = I.rhs_from_xstar(A, np.random.default_rng(40 + i))
        sets.append((A, b, xs))
    precs, cost = (O.FP32, O.FP64), (1.0, 2.0)
    oo = O.Options(seed=11, min_k=0, precs=precs, cost={O.FP32: 1.0, O.FP64: 2.0}, op_mask=(0b10, 0b11, 0b11, 0b11),
                   joint=1)
    E, tmax = 8, 300
    qt = O.QTable.zeros(oo)
    assert qt.Q.shape == (oo.n_states, 16) and qt.visits.shape == (oo.n_states,)
    it_o = np.array([O.train_round(oo, [s[0] for s in sets], [s[1] for s in sets], 1e-6, tmax, e, E, qt)
                     for e in range(1, E + 1)])
    ctx = M.Context(0, M.Options(min_k=0, seed=11, precs=precs, cost=cost, op_mask=oo.op_mask, joint=1))
    mats = [ctx.matrix(_dev(A)) for A, _, _ in sets]
    bs = [torch.as_tensor(b).cuda() for _, b, _ in sets]
    qs, vs = ctx.qtable_shapes()
    pol = ctx.policy_qtable(np.zeros(qs), np.zeros(vs, dtype=np.int32))
    it_g = ctx.train_qtable(mats, bs, 1e-6, tmax, E, pol, want_iters=True)
    Qg, vg = pol.qtable()
    assert np.array_equal(it_g, it_o), (it_g, it_o)
    assert np.array_equal(vg, qt.visits)
    # entries of joint actions with the product in fp32 are outside the mask: never updated
    outside = [a for a in range(16) if (a >> 3) & 1 == 0]
    assert not Qg[:, outside].any() and not qt.Q[:, outside].any()
    assert np.allclose(Qg, qt.Q, rtol=1e-6, atol=1e-9), float(np.max(np.abs(Qg - qt.Q)))
    for (A, b, _), mat in zip(sets, mats):
        x = torch.zeros(A[0], dtype=torch.float64, device="cuda")
        r, h = ctx.solve(mat, torch.as_tensor(b).cuda(), x, 1e-6, tmax, pol, history_cap=tmax)
        ref = O.solve(oo, A, b, 1e-6, tmax, qtable=qt)
        assert r["outcome"] == ref.outcome == O.CONVERGED
        n = min(len(h), len(ref.hist), r["iters"])
        differ = int(np.sum(np.any(h["fmt"][:n] != ref.hist["fmt"][:n], axis=1)))
        assert differ <= r["near_edge_count"], (differ, r["near_edge_count"])
        if differ == 0:
            assert r["iters"] == ref.iters


def test_adam_step_matches_oracle(M):
    """mpcg_mlp_adam (the fp32 kernel of mpcg_mlp_train) against the oracle's fp64 Adam on the
    same gradients, one and several steps."""
    H, nprec = 64, 5
    ctx = M.Context(0, M.Options(mlp_hidden=H))
    npar = M.mlp_nparams(H, nprec)
    rng = np.random.default_rng(12)
    w = rng.standard_normal(npar).astype(np.float32) * 0.1
    m = np.zeros(npar, dtype=np.float32)
    v = np.zeros(npar, dtype=np.float32)
    wo, mo, vo = w.astype(np.float64), np.zeros(npar), np.zeros(npar)
    lr = 1e-3
    for t in range(1, 6):
        g = (rng.standard_normal(npar) * 10.0 ** rng.uniform(-5, 0, npar)).astype(np.float32)
        g[rng.random(npar) < 0.05] = 0.0
        w_before = w.copy()
        ctx.mlp_adam(w, m, v, g, t, lr)
        O.adam(wo, mo, vo, g.astype(np.float64), t, lr=lr)
        # the kernel works in fp32 with beta1 = 0.9 and beta2 = 0.999 rounded to fp32: 1 - beta2
        # is then 1.3e-5 (relative) away from the oracle's fp64 value, so the moments agree to
        # 1e-4 relative; the steps (a ratio of the moments) to a small fraction of lr
        assert np.allclose(m, mo, rtol=1e-4, atol=1e-12)
        assert np.allclose(v, vo, rtol=1e-4, atol=1e-20)
        step_g = w.astype(np.float64) - w_before
        step_o = wo - w_before.astype(np.float64)
        assert np.all(np.abs(step_g - step_o) <= 1e-4 * lr + 2e-7 * np.abs(wo)), t
        wo = w.astype(np.float64)  # continue from the same parameters on both sides


def test_all_fp16_assignment_stagnates_like_the_oracle(M):
    """The 32 x 32 Poisson problem with every operation in fp16 to tau = 1e-10 and a cap of
    1000 iterations: the residual stagnates near 2e-6 (fp16's unit roundoff times the
    conditioning); GPU and oracle agree on the history until it reaches the stagnation
    level, on the outcome and on the stagnation level."""
    A, b, xs = I.cfg_poisson32()
    ctx = M.Context(0, M.Options())
    mat = ctx.matrix(_dev(A))
    bd = torch.as_tensor(b).cuda()
    x = torch.zeros_like(bd)
    pol = ctx.policy_fixed((0, 0, 0, 0))
    res, hist = ctx.solve(mat, bd, x, 1e-10, 1000, pol, history_cap=1000)
    ref = O.solve(O.Options(), A, b, 1e-10, 1000, fixed=(0, 0, 0, 0))
    assert res["outcome"] == ref.outcome == O.MAX_ITER and res["iters"] == ref.iters == 1000
    rg, ro = hist["rho"][:1000], ref.hist["rho"][:1000]
    err = np.abs(rg - ro) / ro
    first = int(np.argmax(err > TOL_LOW)) if np.any(err > TOL_LOW) else 1000
    assert first >= 40, first  # the histories agree through the descent
    lg, lo = rg[100:].min(), ro[100:].min()
    assert lo / 3 <= lg <= 3 * lo, (lg, lo)
    assert 5e-7 < lo < 1e-5
    eg = np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs)
    eo = np.linalg.norm(ref.x - xs) / np.linalg.norm(xs)
    assert eg <= 10 * eo
    print(f"all-fp16: stagnation rho GPU {lg:.3g} oracle {lo:.3g}, histories agree for {first} iterations, "
          f"error to x* GPU {eg:.3g} oracle {eo:.3g}")
