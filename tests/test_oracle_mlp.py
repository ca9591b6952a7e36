"""Pins for the oracle's MLP Q-function (an extension: the paper uses tables and names deep
RL as future work in Section 7).

Independent references: central finite differences of the loss, numpy's least-squares
solver for the special case in which the network is linear in its last layer, and the
closed form of Adam's step under a constant gradient."""
import numpy as np
import pytest

import oracle as O

H, NPREC = 16, 5
NOUT = 4 * NPREC


def _params(rng, H=H):
    n = O.mlp_nparams(H, NOUT)
    return rng.standard_normal(n) * 0.3


def _batch(rng, B=12):
    feats = rng.standard_normal((B, O.NFEAT))
    acts = rng.integers(0, NPREC, (B, 4)).astype(np.int32)
    y = rng.standard_normal((B, 4))
    return feats, acts, y


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    w = _params(rng)
    feats, acts, y = _batch(rng)
    loss, g = O.mlp_loss_grad(w, H, NPREC, feats, acts, y)
    h = 1e-6
    idx = rng.choice(w.size, 150, replace=False)
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (O.mlp_loss_grad(wp, H, NPREC, feats, acts, y)[0] - O.mlp_loss_grad(wm, H, NPREC, feats, acts, y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8


def test_forward_shapes_and_relu():
    rng = np.random.default_rng(1)
    w = _params(rng)
    out, h1, h2 = O.mlp_forward(w, H, NOUT, rng.standard_normal(O.NFEAT))
    assert out.shape == (NOUT,) and np.all(h1 >= 0) and np.all(h2 >= 0)


def test_last_layer_least_squares_special_case():
    """With W1 = [I; 0], b1 = 0, W2 = I, b2 = 0 and positive features every ReLU passes its
    input, so Q is linear in (W3, b3). At numpy's least-squares solution for the taken
    outputs the loss equals the least-squares residual and its last-layer gradient vanishes."""
    rng = np.random.default_rng(2)
    Hh = 16
    n = O.mlp_nparams(Hh, NOUT)
    w = np.zeros(n)
    w[: Hh * 16] = np.eye(Hh, 16).ravel()     # W1
    o = Hh * 16 + Hh                          # skip b1
    w[o:o + Hh * Hh] = np.eye(Hh).ravel()     # W2
    o += Hh * Hh + Hh                         # skip b2; W3, b3 follow
    B = 64
    feats = rng.uniform(0.5, 1.5, (B, 16))
    acts = np.zeros((B, 4), dtype=np.int32)   # every op takes action 0
    y = rng.standard_normal((B, 4))
    Hm = np.column_stack([feats, np.ones(B)])
    theta, res, *_ = np.linalg.lstsq(Hm, y, rcond=None)
    W3 = w[o: o + NOUT * Hh].reshape(NOUT, Hh)
    b3 = w[o + NOUT * Hh:]
    for j in range(4):
        W3[j * NPREC] = theta[:16, j]
        b3[j * NPREC] = theta[16, j]
    loss, g = O.mlp_loss_grad(w, Hh, NPREC, feats, acts, y)
    assert loss == pytest.approx(0.5 * res.sum() / (B * 4), rel=1e-10)
    assert np.abs(g[o:]).max() < 1e-12
    # moving one taken-output weight off the optimum gives a non-zero gradient of the right sign
    W3[0, 0] += 0.1
    _, g2 = O.mlp_loss_grad(w, Hh, NPREC, feats, acts, y)
    assert g2[o] > 0


def test_adam_closed_form_under_constant_gradient():
    """With a constant gradient g, m_hat = g and v_hat = g^2 at every step, so each step moves
    w by -lr g / (|g| + eps)."""
    w = np.array([1.0, -2.0, 0.5])
    m = np.zeros(3)
    v = np.zeros(3)
    g = np.array([0.3, -4.0, 1e-3])
    lr, eps = 1e-2, 1e-8
    for t in range(1, 51):
        O.adam(w, m, v, g, t, lr=lr, eps=eps)
    expect = np.array([1.0, -2.0, 0.5]) - 50 * lr * g / (np.abs(g) + eps)
    assert np.allclose(w, expect, rtol=0, atol=1e-12)


def test_static_features_poisson():
    """n = 1024, mean nnz/row = 4.875, equal diagonals, Gershgorin ratio 2, no entry outside
    the fp16 normal range."""
    from paper_2504_14268_gb300 import inputs as I

    A, b, _ = I.cfg_poisson32()
    f = O.static_features(A)
    assert f == pytest.approx([np.log10(1024) / 8, 4.875 / 64, 0.0, np.log10(2.0) / 16, 0.0])


def test_fitted_q_targets_closed_form_and_masks():
    """With W1 = W2 = W3 = 0 the network's output is its last bias b3 whatever the features,
    so y_bj = r_b + gamma (1 - done_b) max over the allowed p of b3[j nprec + p]; a terminal
    sample keeps its reward alone."""
    H, nprec = 8, 5
    nout = 4 * nprec
    w = np.zeros(O.mlp_nparams(H, nout))
    rng = np.random.default_rng(3)
    b3 = rng.normal(size=nout)
    w[-nout:] = b3
    B = 6
    fn = rng.normal(size=(B, 16))
    rew = rng.normal(size=B)
    done = np.array([0, 1, 0, 0, 1, 0], dtype=np.int32)
    masks = (0, 0b11000, 0b00110, 0b10000)
    y = O.mlp_targets(w, H, nprec, fn, rew, done, 0.9, masks)
    for b in range(B):
        for j in range(4):
            allowed = [p for p in range(nprec) if masks[j] == 0 or (masks[j] >> p) & 1]
            m = max(b3[j * nprec + p] for p in allowed)
            assert y[b, j] == pytest.approx(rew[b] + (0.0 if done[b] else 0.9 * m), abs=1e-15)


def test_fitted_q_targets_match_forward_pass():
    """General weights: each target equals the reward plus gamma times the largest allowed
    output of the forward pass on f_next (forward pass pinned separately)."""
    H, nprec = 6, 3
    nout = 4 * nprec
    rng = np.random.default_rng(4)
    w = rng.normal(size=O.mlp_nparams(H, nout)) * 0.5
    fn = rng.normal(size=(3, 16))
    rew = np.array([1.0, -2.0, 0.5])
    done = np.array([0, 0, 1], dtype=np.int32)
    y = O.mlp_targets(w, H, nprec, fn, rew, done, 0.5, (0b011, 0, 0b100, 0b101))
    out0, _, _ = O.mlp_forward(w, H, nout, fn[0])
    assert y[0, 0] == pytest.approx(1.0 + 0.5 * max(out0[0], out0[1]))
    assert y[0, 1] == pytest.approx(1.0 + 0.5 * max(out0[3:6]))
    assert y[0, 2] == pytest.approx(1.0 + 0.5 * out0[8])
    assert y[0, 3] == pytest.approx(1.0 + 0.5 * max(out0[9], out0[11]))
    assert np.all(y[2] == 0.5)
