"""Pins for the oracle's MDP and Q-learning (Section 4.1, Algorithm 1, Algorithm 2).

Independent references: bin indices worked out by hand at and around the edges of
Section 4.1's formulas, rewards worked out by hand from the Section 5 weights and cost
table, the closed form Q = (1 - (1 - lr)^m) R for a one-step episode repeated m times, the
Bellman fixed point of a deterministic chain (value iteration) for the update rule, and
the equivalence of the batched reading with Algorithm 1 when there is one lane."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2504_14268_gb300 import inputs as I


def test_iteration_bins():
    """b = 10 bins over T_max = 1000: width ceil(1000 / 10) = 100, saturating at b - 1."""
    o = O.Options()
    rho = 0.5  # residual bin 0
    for k, i in [(0, 0), (99, 0), (100, 1), (555, 5), (999, 9), (1000, 9), (20000, 9)]:
        assert O.state(o, k, rho) == i * 10 + 0
    o2 = O.Options(b_bins=7, t_bin=100)  # width ceil(100 / 7) = 15
    assert [O.state(o2, k, rho) // 10 for k in (14, 15, 29, 30, 89, 90, 500)] == [0, 1, 1, 2, 5, 6, 6]


@pytest.mark.parametrize("rho,j", [(1.0, 0), (10.0, 0), (10 ** -1.5, 0), (10 ** -1.7, 1), (1e-3, 1),
                                   (1e-4, 2), (1e-8, 5), (10 ** -8.1, 5), (1e-15, 9), (1e-16, 9),
                                   (1e-30, 9), (0.0, 9)])
def test_residual_bins(rho, j):
    """r = 10 bins, eps_min = 1e-16: delta = 1.6 decades; j = min(floor(-log10 max(rho, eps_min) / 1.6), 9)."""
    assert O.state(O.Options(), 0, rho) == j


def test_reward_by_hand():
    """Section 4.1 reward with w = (1, 0.1, 10) and cost setting C1 (Section 5)."""
    o = O.Options()  # precs = (fp16, bf16, tf32, fp32, fp64), C1 costs (0.8, 0.6, 0.8, 1.0, 2.0)
    # rho' = 1e-3, all fp16: 3 - 0.1 * 3.2 = 2.68
    assert O.reward(o, 1e-3, [0, 0, 0, 0], 1e-6) == pytest.approx(2.68, abs=1e-12)
    # rho' = 1e-7 < tau = 1e-6, actions (bf16, tf32, fp32, fp64): 7 - 0.1 * 4.4 + 10 = 16.56
    assert O.reward(o, 1e-7, [1, 2, 3, 4], 1e-6) == pytest.approx(16.56, abs=1e-12)
    # rho' = 0 clamps at -log10(1e-16) = 16; C2 costs, all fp64: 16 - 0.1 * 12 + 10 = 24.8
    o2 = O.Options(cost=dict(O.COST_C2))
    assert O.reward(o2, 0.0, [4, 4, 4, 4], 1e-6) == pytest.approx(24.8, abs=1e-12)
    # rho' > 1 gives a negative accuracy term: -1 - 0.32 = -1.32
    assert O.reward(o, 10.0, [0, 0, 0, 0], 1e-6) == pytest.approx(-1.32, abs=1e-12)


def test_epsilon_schedule():
    """epsilon = eps0 (1 - e / E) with the 0.1 floor of Section 5."""
    o = O.Options()
    assert O.epsilon(o, 1, 200) == pytest.approx(0.995)
    assert O.epsilon(o, 100, 200) == pytest.approx(0.5)
    assert O.epsilon(o, 180, 200) == pytest.approx(0.1)
    assert O.epsilon(o, 200, 200) == pytest.approx(0.1)


def _scaled_identity(n=8, c=2.0):
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    return (n, rp, ci, np.full(n, c))


def test_one_step_episode_closed_form():
    """A = 2 I with an fp16-exact right-hand side converges in one CG step with rho' = 0 for
    every action. Greedy selection on a zero table picks index 0 (fp16) for each op, so after
    m episodes Q_j(s_0, fp16) = (1 - (1 - lr)^m) R with R = 16 - 0.1 * 3.2 + 10 = 25.68."""
    A = _scaled_identity()
    b = np.arange(1.0, 9.0)
    o = O.Options(min_k=0, eps0=0.0, eps_floor=0.0)
    qt = O.QTable.zeros(o)
    m = 25
    iters = O.train_sequential(o, A, b, 1e-6, 50, m, qt)
    assert np.all(iters == 1)
    R = 25.68
    expect = (1 - 0.9 ** m) * R
    s0 = O.state(o, 0, 1.0)
    for j in range(4):
        assert qt.Q[j, s0, 0] == pytest.approx(expect, rel=1e-12)
        assert qt.visits[j, s0] == m
    mask = np.ones_like(qt.Q, dtype=bool)
    mask[:, s0, 0] = False
    assert not qt.Q[mask].any()


def test_update_rule_converges_to_bellman_fixed_point():
    """Deterministic chain s0 -> s1 -> s2 -> end with rewards (1, 2, 5), one action per op:
    the fixed point is Q(s2) = 5, Q(s1) = 2 + 0.9 * 5, Q(s0) = 1 + 0.9 * Q(s1)."""
    o = O.Options()
    qt = O.QTable.zeros(o)
    chain = np.zeros(3, dtype=O.TRANS_DTYPE)
    for t, (s, sn, r, term) in enumerate([(0, 1, 1.0, 0), (1, 2, 2.0, 0), (2, 2, 5.0, 1)]):
        chain[t]["s"], chain[t]["s_next"], chain[t]["reward"], chain[t]["terminal"] = s, sn, r, term
        chain[t]["act"] = [3, 3, 3, 3]
    for _ in range(400):
        O.q_update(o, qt, chain)
    q2 = 5.0
    q1 = 2.0 + 0.9 * q2
    q0 = 1.0 + 0.9 * q1
    for j in range(4):
        assert qt.Q[j, [0, 1, 2], 3] == pytest.approx([q0, q1, q2], rel=1e-9)
    assert qt.visits[0, 0] == 400


def test_greedy_tie_rule_and_unvisited_fallback():
    """First-index argmax in the order (fp16, bf16, tf32, fp32, fp64); a never-updated row uses
    the fallback format (fp64 by default) or, with the fallback off, plain argmax (fp16)."""
    A, b, _ = I.cfg_poisson32()
    o = O.Options(min_k=0)
    qt = O.QTable.zeros(o)
    out = O.solve(o, A, b, 1e-6, 3, qtable=qt)
    assert np.all(out.hist["fmt"] == O.FP64)
    o_off = O.Options(min_k=0, unvisited_fallback=-1)
    out = O.solve(o_off, A, b, 1e-6, 3, qtable=qt)
    assert np.all(out.hist["fmt"] == O.FP16)
    s0 = O.state(o, 0, 1.0)
    qt.Q[:, s0, :] = [1.0, 3.0, 3.0, 0.0, 0.0]
    qt.visits[:, s0] = 1
    out = O.solve(o, A, b, 1e-6, 1, qtable=qt)
    assert np.all(out.hist["fmt"][0] == O.BF16)


def test_batched_round_with_one_lane_is_algorithm_1():
    """One lane per round, E rounds == Algorithm 1 with E episodes, bit for bit."""
    A, b, _ = I.cfg_poisson32()
    o = O.Options(seed=11, min_k=0)
    E, tmax = 12, 120
    q_seq = O.QTable.zeros(o)
    it_seq = O.train_sequential(o, A, b, 1e-6, tmax, E, q_seq)
    q_bat = O.QTable.zeros(o)
    it_bat = []
    for e in range(1, E + 1):
        it_bat.append(O.train_round(o, [A], [b], 1e-6, tmax, e, E, q_bat)[0])
    assert np.array_equal(q_seq.Q, q_bat.Q)
    assert np.array_equal(q_seq.visits, q_bat.visits)
    assert list(it_seq) == it_bat


def test_batched_round_replays_in_lane_order():
    """The shared table after a round equals replaying lane 0's then lane 1's transitions
    (each recorded with its private copy) onto the round-start table."""
    mats = I.cfg_train_set(count=2, m_lo=6, m_hi=8)
    o = O.Options(seed=3, min_k=0)
    qt = O.QTable.zeros(o)
    O.train_round(o, [m[0] for m in mats], [m[1] for m in mats], 1e-6, 150, 1, 10, qt)
    ref = O.QTable.zeros(o)
    eps = O.epsilon(o, 1, 10)
    for lane, (A, b, _) in enumerate(mats):
        priv = O.QTable.zeros(o)
        out = O.solve(o, A, b, 1e-6, 150, qtable=priv, train=True, episode=1, lane=lane, eps=eps,
                      want_trans=True)
        O.q_update(o, ref, out.trans)
    assert np.array_equal(qt.Q, ref.Q)
    assert np.array_equal(qt.visits, ref.visits)


def test_exploration_rate_matches_epsilon():
    """Over an episode with epsilon = 0.5 about half of the operation choices explore."""
    A, b, _ = I.cfg_poisson32()
    o = O.Options(seed=5, min_k=0)
    qt = O.QTable.zeros(o)
    out = O.solve(o, A, b, 1e-12, 400, qtable=qt, train=True, episode=1, lane=0, eps=0.5)
    frac = np.mean(out.hist["flags"] & 8 > 0)  # some op explored in that iteration
    assert abs(frac - (1 - 0.5 ** 4)) < 0.08


def test_training_learns_cheap_safe_schedule_on_easy_problem():
    """On the 32 x 32 Poisson problem with tau = 1e-6 (cost C2), training drives the greedy
    policy to a schedule that still converges and costs less than all-fp64 (qualitative)."""
    A, b, xs = I.cfg_poisson32()
    o = O.Options(seed=1, min_k=10, cost=dict(O.COST_C2))
    qt = O.QTable.zeros(o)
    O.train_sequential(o, A, b, 1e-6, 1000, 60, qt)
    out = O.solve(o, A, b, 1e-6, 1000, qtable=qt)
    assert out.outcome == O.CONVERGED
    cost = sum(o.cost[int(f)] for f in out.hist["fmt"].ravel()) / len(out.hist)
    assert cost < 4 * o.cost[O.FP64]


def test_operation_masks_restrict_greedy_and_exploration():
    """op_mask: op 0 may use only fp32/fp64 (indices 3, 4). The one-step episode of the closed
    form test then updates Q_0(s_0, fp32) (first allowed index), the other operations keep
    fp16; exploration draws stay uniform over the allowed entries."""
    A = _scaled_identity()
    b = np.arange(1.0, 9.0)
    o = O.Options(min_k=0, eps0=0.0, eps_floor=0.0, op_mask=(0b11000, 0, 0, 0))
    qt = O.QTable.zeros(o)
    m = 10
    O.train_sequential(o, A, b, 1e-6, 50, m, qt)
    s0 = O.state(o, 0, 1.0)
    R = 16 - 0.1 * (1.0 + 0.8 * 3) + 10  # fp32 for op 0, fp16 for the others
    assert qt.Q[0, s0, 3] == pytest.approx((1 - 0.9 ** m) * R, rel=1e-12)
    assert qt.Q[0, s0, 0] == 0.0
    for j in (1, 2, 3):
        assert qt.Q[j, s0, 0] == pytest.approx((1 - 0.9 ** m) * R, rel=1e-12)
    # exploration with epsilon = 1 picks only allowed entries, uniformly
    A2, b2, _ = I.cfg_poisson32()
    o2 = O.Options(min_k=0, seed=4, op_mask=(0b10110, 0, 0, 0))
    out = O.solve(o2, A2, b2, 1e-30, 600, qtable=O.QTable.zeros(o2), train=True, episode=1, eps=1.0)
    picks = out.hist["act"][:, 0]
    assert set(np.unique(picks)) <= {1, 2, 4}
    cnt = np.array([np.sum(picks == a) for a in (1, 2, 4)])
    exp = len(picks) / 3
    assert np.sum((cnt - exp) ** 2 / exp) < 13.8  # chi-square, 2 dof, p ~ 0.001


def test_bootstrap_max_runs_over_the_allowed_set():
    """Section 4.1's update bootstraps on max over P; with a customised per-operation set
    P_j (op_mask) the max runs over P_j. One update by hand: op j may choose only fp64
    (index 4), Q_j(s', .) = (0, 0, 0, 0, -5) with the zeros never allowed, Q_j(s, fp64) = -2,
    R = -1: target = -1 + 0.9 (-5) = -5.5 and Q_j(s, fp64) = -2 + 0.1 (-5.5 + 2) = -2.35
    (an unrestricted max would bootstrap on 0 and give -1.9)."""
    o = O.Options(op_mask=(0b10000,) * 4)
    qt = O.QTable.zeros(o)
    qt.Q[:, 7, 4] = -5.0
    qt.Q[:, 3, 4] = -2.0
    t = np.zeros(1, dtype=O.TRANS_DTYPE)
    t[0]["s"], t[0]["s_next"], t[0]["reward"], t[0]["terminal"] = 3, 7, -1.0, 0
    t[0]["act"] = [4, 4, 4, 4]
    O.q_update(o, qt, t)
    for j in range(4):
        assert qt.Q[j, 3, 4] == pytest.approx(-2.35, abs=1e-15)
        assert qt.Q[j, 7, 4] == -5.0 and not qt.Q[j, :, :4].any()
    # a mix of allowed entries: op 0 may use fp32 and fp64 (indices 3, 4) with
    # Q_0(s', .) = (9, 9, 9, -4, -6): target = -1 + 0.9 (-4) = -4.6, Q = -2 + 0.1 (-2.6)
    o2 = O.Options(op_mask=(0b11000, 0, 0, 0))
    q2 = O.QTable.zeros(o2)
    q2.Q[0, 7] = [9.0, 9.0, 9.0, -4.0, -6.0]
    q2.Q[0, 3, 4] = -2.0
    t[0]["act"] = [4, 4, 4, 4]
    O.q_update(o2, q2, t)
    assert q2.Q[0, 3, 4] == pytest.approx(-2.26, abs=1e-15)
    # operations without a mask keep the full set: op 1 bootstraps on max(0, ..., 0) = 0
    assert q2.Q[1, 3, 4] == pytest.approx(-0.1, abs=1e-15)


def test_masked_chain_reaches_the_restricted_bellman_fixed_point():
    """Chain s0 -> s1 -> end with negative rewards (-1, -3), every operation restricted to
    fp64: value iteration on the restricted MDP gives Q(s1, fp64) = -3 and Q(s0, fp64) =
    -1 + 0.9 (-3) = -3.7. The never-allowed entries (still 0) must not lift Q(s0) to -1."""
    o = O.Options(op_mask=(0b10000,) * 4)
    qt = O.QTable.zeros(o)
    chain = np.zeros(2, dtype=O.TRANS_DTYPE)
    for t, (s, sn, r, term) in enumerate([(0, 1, -1.0, 0), (1, 1, -3.0, 1)]):
        chain[t]["s"], chain[t]["s_next"], chain[t]["reward"], chain[t]["terminal"] = s, sn, r, term
        chain[t]["act"] = [4, 4, 4, 4]
    for _ in range(400):
        O.q_update(o, qt, chain)
    for j in range(4):
        assert qt.Q[j, [0, 1], 4] == pytest.approx([-3.7, -3.0], rel=1e-9)


def test_greedy_action_is_the_solvers_decision():
    """orc_greedy_action (used to check GPU decisions on a replayed trajectory) gives the
    action the oracle's own greedy solve takes at every iteration of that solve."""
    A, b, _ = I.cfg_poisson32()
    o = O.Options(seed=2, min_k=0, cost=dict(O.COST_C2))
    qt = O.QTable.zeros(o)
    O.train_sequential(o, A, b, 1e-6, 300, 15, qt)
    out = O.solve(o, A, b, 1e-6, 300, qtable=qt)
    rho = 1.0
    for k, rec in enumerate(out.hist):
        s, fm = O.greedy_action(o, qt, k, rho)
        assert s == rec["state"] and fm == tuple(int(f) for f in rec["fmt"]), k
        rho = rec["rho"]


def test_joint_table_equals_the_free_operations_table():
    """With operations 2-4 restricted to fp64 the joint table's entries (a, fp64, fp64, fp64)
    are operation 1's table, update for update: the joint set is operation 1's set, its
    exploration draw and pick are operation 1's, and every target is the same max."""
    A, b, _ = I.cfg_poisson32()
    precs, cost = (O.FP32, O.FP64), {O.FP32: 1.0, O.FP64: 2.0}
    masks = (0b11, 0b10, 0b10, 0b10)
    sep = O.Options(seed=5, min_k=0, precs=precs, cost=cost, op_mask=masks)
    jnt = O.Options(seed=5, min_k=0, precs=precs, cost=cost, op_mask=masks, joint=1)
    qs, qj = O.QTable.zeros(sep), O.QTable.zeros(jnt)
    it_s = O.train_sequential(sep, A, b, 1e-6, 200, 12, qs)
    it_j = O.train_sequential(jnt, A, b, 1e-6, 200, 12, qj)
    assert list(it_s) == list(it_j)
    assert qj.Q.shape == (100, 16) and qj.visits.shape == (100,)
    # joint index of (a, fp64, fp64, fp64) = a * 8 + 1 * 4 + 1 * 2 + 1
    assert np.array_equal(qj.Q[:, [7, 15]], qs.Q[0])
    assert np.array_equal(qj.visits, qs.visits[0])
    out_s = O.solve(sep, A, b, 1e-6, 200, qtable=qs)
    out_j = O.solve(jnt, A, b, 1e-6, 200, qtable=qj)
    assert np.array_equal(out_s.hist["fmt"], out_j.hist["fmt"])


def test_joint_table_one_step_closed_form_and_bellman_chain():
    """A = 2 I converges in one step: the greedy joint action on a zero table is the first
    joint index (all fp16), and after m episodes Q(s_0, 0) = (1 - (1 - lr)^m) R, R = 25.68.
    A chain s0 -> s1 -> end with rewards (1, 5) on joint action (fp32, fp32, fp32, fp32):
    Q(s1) = 5, Q(s0) = 1 + 0.9 * 5 (the max over the joint row of s1)."""
    A = _scaled_identity()
    b = np.arange(1.0, 9.0)
    o = O.Options(min_k=0, eps0=0.0, eps_floor=0.0, joint=1)
    qt = O.QTable.zeros(o)
    m = 15
    O.train_sequential(o, A, b, 1e-6, 50, m, qt)
    s0 = O.state(o, 0, 1.0)
    assert qt.Q[s0, 0] == pytest.approx((1 - 0.9 ** m) * 25.68, rel=1e-12)
    assert qt.visits[s0] == m and np.count_nonzero(qt.Q) == 1
    o2 = O.Options(joint=1)
    q2 = O.QTable.zeros(o2)
    chain = np.zeros(2, dtype=O.TRANS_DTYPE)
    for t, (s, sn, r, term) in enumerate([(0, 1, 1.0, 0), (1, 1, 5.0, 1)]):
        chain[t]["s"], chain[t]["s_next"], chain[t]["reward"], chain[t]["terminal"] = s, sn, r, term
        chain[t]["act"] = [3, 3, 3, 3]
    for _ in range(400):
        O.q_update(o2, q2, chain)
    a = ((3 * 5 + 3) * 5 + 3) * 5 + 3
    assert q2.Q[[0, 1], a] == pytest.approx([1 + 0.9 * 5.0, 5.0], rel=1e-9)
    assert np.count_nonzero(q2.Q) == 2
