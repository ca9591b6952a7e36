"""A reduced form of the paper's experiment protocol (Section 5) on the GPU against the oracle:
training systems of the Section 5.2 family (Poisson on random subdomains, n = 6400), the
fp32 IC(0) preconditioner (the reading of Section 5's fp32 incomplete factorization),
tau = 1e-6 with k >= 10, iteration cap 1000, batched Algorithm 1 rounds, then Algorithm 2 on
test systems of the family.

With P = {fp32, fp64} both sides take the same actions (the IC(0) factor and substitutions
are the same fp32 operations in the same order), so iteration counts and visits are equal and
the tables and the greedy histories agree to the accuracy of the residual histories. With the
paper's full set P = {fp16, bf16, tf32, fp32, fp64} trajectories separate at rounding ties, so
the full-set run is compared through the quantities Tables 2 and 4 report."""
import numpy as np
import pytest

import oracle as O
from paper_2504_14268_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TAU, TMAX = 1e-6, 1000


@pytest.fixture(scope="module")
def M():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2504_14268_gb300 import mpcg

    return mpcg


def _dev(A):
    n, rp, ci, val = A
    return (n, torch.as_tensor(rp).cuda(), torch.as_tensor(ci).cuda(), torch.as_tensor(val).cuda())


def test_reduced_protocol_fp32_fp64_matches_oracle(M):
    train = [I.poisson_subdomain(s) for s in (0, 1)]
    test = [I.poisson_subdomain(s) for s in range(100000, 100005)]
    E = 20
    oo = O.Options(precs=(3, 4), cost={3: 1.0, 4: 2.0}, precond=2, min_k=10, t_bin=TMAX, seed=4)
    qt = O.QTable.zeros(oo)
    it_o = np.array([O.train_round(oo, [a for a, _ in train], [b for _, b in train], TAU, TMAX, e, E, qt)
                     for e in range(1, E + 1)])
    ctx = M.Context(0, M.Options(precs=(3, 4), cost=(1.0, 2.0), precond=2, min_k=10, t_bin=TMAX, seed=4))
    mats = [ctx.matrix(_dev(A)) for A, _ in train]
    bs = [torch.as_tensor(b).cuda() for _, b in train]
    pol = ctx.policy_qtable(np.zeros((4, 100, 2)), np.zeros((4, 100), dtype=np.int32))
    it_g = ctx.train_qtable(mats, bs, TAU, TMAX, E, pol, want_iters=True)
    Qg, vg = pol.qtable()
    assert np.array_equal(it_g, it_o), (it_g[:3], it_o[:3])
    assert np.array_equal(vg, qt.visits)
    assert np.allclose(Qg, qt.Q, rtol=1e-6, atol=1e-9), float(np.max(np.abs(Qg - qt.Q)))
    # greedy on the test systems, batched, against the oracle's greedy solves
    tm = [ctx.matrix(_dev(A)) for A, _ in test]
    tb = [torch.as_tensor(b).cuda() for _, b in test]
    xs = [torch.zeros_like(b) for b in tb]
    res = ctx.solve_batched(tm, tb, xs, [TAU] * 5, [TMAX] * 5, pol)
    for (A, b), r, x in zip(test, res, xs):
        ref = O.solve(oo, A, b, TAU, TMAX, qtable=qt)
        assert r["outcome"] == ref.outcome == O.CONVERGED
        assert abs(r["iters"] - ref.iters) <= 1
        assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-5 * np.linalg.norm(ref.x)


def test_reduced_protocol_full_set_statistics(M):
    """The paper's precision set and cost setting C1, 2 training systems x 30 rounds: the GPU's
    and the oracle's runs give the same kind of policy (format shares within 0.15 of each
    other -- the oracle alone moves them by up to 0.12 between two exploration seeds of this
    short training --, mean iterations of the greedy test solves within 15%), both converging.
    The greedy solves restart in fp64 after a breakdown (on small subdomains the five-point
    values 1/h^2 exceed fp16's range, so an fp16 product overflows)."""
    train = [I.poisson_subdomain(s) for s in (2, 3)]
    test = [I.poisson_subdomain(s) for s in range(100010, 100014)]
    E = 30
    cost = {0: 0.8, 1: 0.6, 2: 0.8, 3: 1.0, 4: 2.0}
    oo = O.Options(cost=cost, precond=2, min_k=10, t_bin=TMAX, seed=6, on_breakdown=1)
    qt = O.QTable.zeros(oo)
    for e in range(1, E + 1):
        O.train_round(oo, [a for a, _ in train], [b for _, b in train], TAU, TMAX, e, E, qt)
    ctx = M.Context(0, M.Options(cost=(0.8, 0.6, 0.8, 1.0, 2.0), precond=2, min_k=10, t_bin=TMAX, seed=6,
                                 on_breakdown=1))
    mats = [ctx.matrix(_dev(A)) for A, _ in train]
    bs = [torch.as_tensor(b).cuda() for _, b in train]
    pol = ctx.policy_qtable(np.zeros((4, 100, 5)), np.zeros((4, 100), dtype=np.int32))
    ctx.train_qtable(mats, bs, TAU, TMAX, E, pol)
    tm = [ctx.matrix(_dev(A)) for A, _ in test]
    tb = [torch.as_tensor(b).cuda() for _, b in test]
    xs = [torch.zeros_like(b) for b in tb]
    res = ctx.solve_batched(tm, tb, xs, [TAU] * len(test), [TMAX] * len(test), pol)
    share_g = np.zeros(5)
    share_o = np.zeros(5)
    it_g, it_o = [], []
    for (A, b), r in zip(test, res):
        ref = O.solve(oo, A, b, TAU, TMAX, qtable=qt)
        assert r["outcome"] == O.CONVERGED and ref.outcome == O.CONVERGED
        share_g += np.asarray(r["action_hist"])[:, :5].sum(axis=0)
        share_o += np.array([np.sum(ref.hist["fmt"] == f) for f in range(5)])
        it_g.append(r["iters"])
        it_o.append(ref.iters)
    share_g /= share_g.sum()
    share_o /= share_o.sum()
    print("format shares GPU", np.round(share_g, 3), "oracle", np.round(share_o, 3), "iterations", it_g, it_o)
    assert np.max(np.abs(share_g - share_o)) <= 0.15
    assert abs(np.mean(it_g) - np.mean(it_o)) <= 0.15 * np.mean(it_o)
