"""GPU parity of the learned policy (MLP Q-function, an extension of the paper): the
gradient of the fitted-Q loss computed by the library's kernels against the oracle's fp64
gradient (itself pinned by finite differences), the transitions the solver records against
the oracle's episode with the same exploration draws, the MLP inference fused in the
persistent kernel against the oracle's MLP policy, and the training loop reducing its loss."""
import numpy as np
import pytest

import oracle as O
from paper_2504_14268_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H, NPREC = 64, 5


@pytest.fixture(scope="module")
def M():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2504_14268_gb300 import mpcg

    return mpcg


def _dev(A):
    n, rp, ci, val = A
    return (n, torch.as_tensor(rp).cuda(), torch.as_tensor(ci).cuda(), torch.as_tensor(val).cuda())


def _params(rng, scale=0.2):
    n = O.mlp_nparams(H, 4 * NPREC)
    return (rng.standard_normal(n) * scale).astype(np.float32)


def test_mlp_gradient_matches_oracle(M):
    rng = np.random.default_rng(0)
    ctx = M.Context(0, M.Options(mlp_hidden=H))
    w = _params(rng)
    B = 300
    feats = rng.standard_normal((B, 16)).astype(np.float32)
    acts = rng.integers(0, NPREC, (B, 4)).astype(np.int32)
    y = rng.standard_normal((B, 4)).astype(np.float32)
    loss_g, g = ctx.mlp_loss_grad(w, feats, acts, y)
    loss_o, go = O.mlp_loss_grad(w.astype(np.float64), H, NPREC, feats.astype(np.float64), acts, y.astype(np.float64))
    assert loss_g == pytest.approx(loss_o, rel=1e-5)
    scale = np.abs(go).max()
    assert np.max(np.abs(g - go)) <= 1e-4 * scale


@pytest.mark.parametrize("masks", [(0, 0, 0, 0), (0b11000, 0b10000, 0b00110, 0b10101)])
def test_fitted_q_targets_match_oracle(M, masks):
    """The targets of the fitted-Q regression (Bellman backup through the target network,
    max over each operation's allowed entries) against the oracle's fp64 targets."""
    rng = np.random.default_rng(7)
    ctx = M.Context(0, M.Options(mlp_hidden=H, op_mask=masks))
    wt = _params(rng, 0.3)
    B = 257
    fn = rng.standard_normal((B, 16)).astype(np.float32)
    rew = rng.standard_normal(B).astype(np.float32)
    done = (rng.random(B) < 0.2).astype(np.int32)
    y = ctx.mlp_targets(wt, fn, rew, done)
    yo = O.mlp_targets(wt.astype(np.float64), H, NPREC, fn.astype(np.float64), rew.astype(np.float64), done, 0.9,
                       masks)
    assert np.allclose(y, yo, rtol=1e-5, atol=1e-5 * np.abs(yo).max())


def test_collected_transitions_match_oracle_episode(M):
    """One epsilon-greedy episode with a zero Q-table (epsilon = 0.6): the recorded actions,
    rewards and features follow the oracle's episode with the same Philox draws."""
    A, b, xs = I.cfg_poisson32()
    ctx = M.Context(0, M.Options(min_k=0, seed=9))
    mat = ctx.matrix(_dev(A))
    pol = ctx.policy_qtable(np.zeros((4, 100, 5)), np.zeros((4, 100), dtype=np.int32))
    bd = torch.as_tensor(b).cuda()
    tr = ctx.collect([mat], [bd], 1e-6, 150, pol, eps=0.6, episode=3)
    oo = O.Options(min_k=0, seed=9)
    qt = O.QTable.zeros(oo)
    out = O.solve(oo, A, b, 1e-6, 150, qtable=qt, train=True, episode=3, lane=0, eps=0.6, want_feats=True,
                  want_trans=True, feat_static=O.static_features(A))
    n = min(len(tr), len(out.trans))
    assert n > 5
    # actions agree while the residual histories agree (the first few dozen iterations at least)
    same = np.all(tr["act"][:n] == out.trans["act"][:n], axis=1)
    first_diff = int(np.argmin(same)) if not same.all() else n
    assert first_diff >= min(n, 20)
    k = first_diff
    # with fp16 operations the residual histories drift apart at the 5e-3 level and then
    # separate (one side may break down or replace its residual first); rewards and features
    # are compared while both agree to that level (-log10 of a 5e-3 relative change is 2.2e-3)
    rg, ro = tr["reward"][:k], out.trans["reward"][:k]
    ok = np.abs(rg - ro) <= 5e-3 * np.maximum(1.0, np.abs(ro))
    ok &= np.all(np.isclose(tr["f"][:k], out.feats[:k], rtol=1e-3, atol=1e-3), axis=1)
    m = k if ok.all() else int(np.argmin(ok))
    assert m >= min(k, 15)
    assert np.array_equal(tr["done"][:m], out.trans["terminal"][:m])


def test_fused_mlp_inference_matches_oracle_policy(M):
    """Greedy solve with an MLP policy: the kernel evaluates the network on the fly; the
    oracle evaluates the same network in fp64. Actions agree except where two Q-values are
    within fp32 rounding of each other."""
    A, b, xs = I.cfg_poisson32()
    rng = np.random.default_rng(4)
    w = _params(rng, 0.3)
    ctx = M.Context(0, M.Options(min_k=0, mlp_hidden=H))
    mat = ctx.matrix(_dev(A))
    pol = ctx.policy_mlp(w)
    bd = torch.as_tensor(b).cuda()
    x = torch.zeros_like(bd)
    res, hist = ctx.solve(mat, bd, x, 1e-6, 200, pol, history_cap=200)
    oo = O.Options(min_k=0)
    ref = O.solve(oo, A, b, 1e-6, 200, mlp=w.astype(np.float64), feat_static=O.static_features(A), want_feats=True)
    n = min(len(ref.hist), res["iters"])
    agree = 0
    for k in range(n):
        if np.array_equal(hist["fmt"][k], ref.hist["fmt"][k]):
            agree += 1
            continue
        f = ref.feats[k]
        q, _, _ = O.mlp_forward(w.astype(np.float64), H, 4 * NPREC, f)
        q = q.reshape(4, NPREC)
        top2 = np.sort(q, axis=1)[:, -2:]
        assert np.min(top2[:, 1] - top2[:, 0]) < 1e-3, k  # a near tie explains the difference
        break
    assert agree >= min(n, 5)


def test_mlp_training_reduces_loss(M):
    A, b, xs = I.cfg_poisson32()
    ctx = M.Context(0, M.Options(min_k=0, seed=1, mlp_hidden=H))
    mat = ctx.matrix(_dev(A))
    bd = torch.as_tensor(b).cuda()
    beh = ctx.policy_qtable(np.zeros((4, 100, 5)), np.zeros((4, 100), dtype=np.int32))
    data = np.concatenate([ctx.collect([mat], [bd], 1e-6, 300, beh, eps=0.5, episode=e) for e in range(1, 9)])
    assert len(data) > 100
    rng = np.random.default_rng(2)
    pol = ctx.policy_mlp(_params(rng, 0.1))
    losses = ctx.mlp_train(pol, data, steps=300, batch=256, lr=1e-3, target_sync=100, seed=3)
    assert np.all(np.isfinite(losses))
    assert losses[-20:].mean() < 0.5 * losses[:20].mean()
    w2 = pol.mlp_params()
    assert np.all(np.isfinite(w2))


MASK_3264 = (0b11000,) * 4  # fp32 and fp64 for every operation
COST_C1 = dict(zip((0, 1, 2, 3, 4), (0.8, 0.6, 0.8, 1.0, 2.0)))


def _mean_cost(res):
    ah = np.asarray(res["action_hist"])[:, :5]
    return sum(COST_C1[f] * ah[:, f].sum() for f in range(5)) / max(1, ah.sum())


def test_trained_mlp_generalizes_beyond_the_training_horizon(M):
    """What the learned Q-function adds to the tabular method: both are trained on the same
    small systems (episodes of at most ~160 iterations, so the table's iteration bins beyond
    the second are never visited and fall back to fp64 at inference); on a larger system of
    the family (about 300 iterations) the network, which sees k / T_max and the residual
    history as continuous features, keeps choosing the cheaper format where the table has no
    entry. Both reach the tolerance with an error within 10x of fp64 CG's; the network's mean
    precision cost per operation (cost setting C1) is the lower one. Iterations and times
    are printed for the record (wall time is not asserted)."""
    o = M.Options(true_res_at_conv=1, on_breakdown=1, op_mask=MASK_3264, mlp_hidden=H, seed=5)
    ctx = M.Context(0, o)
    train = [I.cfg_poisson32()[:2]]
    for i, (m, an) in enumerate([(24, 1e-3), (32, 1e-3), (40, 1e-2), (48, 3e-3)]):
        At = I.fem27_aniso(m, an)
        train.append((At, I.rhs_from_xstar(At, np.random.default_rng(100 + i))[1]))
    mats = [ctx.matrix(_dev(A)) for A, _ in train]
    bs = [torch.as_tensor(b).cuda() for _, b in train]
    tab = ctx.policy_qtable(np.zeros((4, 100, NPREC)), np.zeros((4, 100), dtype=np.int32))
    its = ctx.train_qtable(mats, bs, 1e-8, 1000, 100, tab, want_iters=True)
    assert its.max() < 200
    _, visits = tab.qtable()
    assert not visits[:, 20:].any()  # iteration bins >= 2 never visited
    data = np.concatenate([ctx.collect(mats, bs, 1e-8, 1000, tab, eps=0.3, episode=1000 + e) for e in range(1, 13)])
    rng = np.random.default_rng(0)
    mlp = ctx.policy_mlp(_params(rng, 0.1))
    losses = ctx.mlp_train(mlp, data, steps=4000, batch=1024, lr=1e-3, target_sync=500, seed=3)
    assert losses[-100:].mean() < 0.5 * losses[:100].mean()
    A = I.fem27_aniso(128, 3e-3)
    xs, b = I.rhs_from_xstar(A, np.random.default_rng(7))
    mat = ctx.matrix(_dev(A))
    mat.autotune(2)
    bd = torch.as_tensor(b).cuda()
    out = {}
    for name, pol in (("fp64", ctx.policy_fixed((4, 4, 4, 4))), ("tabular", tab), ("mlp", mlp)):
        x = torch.zeros_like(bd)
        ctx.solve(mat, bd, x, 1e-8, 5000, pol)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        res, _ = ctx.solve(mat, bd, x, 1e-8, 5000, pol)
        ev[1].record()
        torch.cuda.synchronize()
        err = float(np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs))
        out[name] = (res, err, ev[0].elapsed_time(ev[1]))
        print(f"{name:8s} outcome {res['outcome']} iters {res['iters']} err {err:.2e} "
              f"mean cost {_mean_cost(res):.2f} time {out[name][2]:.1f} ms")
    e64 = out["fp64"][1]
    for name in ("tabular", "mlp"):
        assert out[name][0]["outcome"] == 0
        assert out[name][1] <= 10 * e64
    assert out["fp64"][0]["iters"] > 200  # beyond the training episodes
    assert _mean_cost(out["mlp"][0]) < _mean_cost(out["tabular"][0]) - 0.05
