"""Pins of the oracle's single-reduction iteration (orc_run_sr: Chronopoulos and Gear's form
of CG with the residual norm of the next state from the same reduction), a widening beyond
the paper's iteration. Independent references: the oracle's CG of Section 3 (itself pinned
by dense solves and Krylov projections) in fp64, where the two are the same method up to
rounding; finite termination with d distinct eigenvalues; and a step-by-step recomputation
of the first iterations with exact sums and numpy's own float16 / float32 roundings."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2504_14268_gb300 import inputs as I
from test_oracle_iteration_by_hand import TYPES, _chop, _exact_dot, _round_to


def _dense_csr(A):
    n = A.shape[0]
    rp = np.arange(0, n * n + 1, n, dtype=np.int32)
    ci = np.tile(np.arange(n, dtype=np.int32), n)
    return (n, rp, ci, A.ravel().copy())


def _stable_prefix(A, b, tol, rel=1e-14):
    """Iterations over which the oracle's CG agrees (1e-6) with itself run on b perturbed by
    `rel`: beyond them a change of rounding alone moves the history."""
    o = O.Options(min_k=0)
    ref = O.solve(o, A, b, tol, 500, fixed=(4, 4, 4, 4))
    b2 = b * (1 + rel * np.random.default_rng(1).standard_normal(b.size))
    twin = O.solve(o, A, b2, tol, 500, fixed=(4, 4, 4, 4))
    n = min(ref.iters, twin.iters)
    e = np.abs(twin.hist["rho"][:n] - ref.hist["rho"][:n]) / ref.hist["rho"][:n]
    return ref, int(np.argmax(e > 1e-6)) if np.any(e > 1e-6) else n


@pytest.mark.parametrize("which", ["random", "poisson", "fem"])
def test_fp64_single_reduction_is_cg(which):
    """In fp64 the two forms are one method up to rounding: equal histories over the prefix on
    which rounding alone does not move the oracle's own CG, equal scalars alpha there, the
    same iteration count within a few, and solutions as accurate."""
    rng = np.random.default_rng(3)
    if which == "random":
        A = I.random_spd_small(60, rng)
    elif which == "poisson":
        A = I.poisson2d(14)
    else:
        A = I.fem27_aniso(6, 1e-2)
    b = rng.uniform(-1, 1, A[0])
    ref, prefix = _stable_prefix(A, b, 1e-11)
    out = O.solve(O.Options(min_k=0, variant=1), A, b, 1e-11, 500, fixed=(4, 4, 4, 4))
    assert out.outcome == ref.outcome == O.CONVERGED
    assert abs(out.iters - ref.iters) <= max(2, ref.iters // 10)
    assert prefix >= min(10, ref.iters)
    err = np.abs(out.hist["rho"][:prefix] - ref.hist["rho"][:prefix]) / ref.hist["rho"][:prefix]
    assert np.all(err < 1e-6), float(err.max())
    assert np.allclose(out.hist["alpha"][:prefix], ref.hist["alpha"][:prefix], rtol=1e-6)
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla

    n, rp, ci, val = A
    S = sp.csr_matrix((val, ci, rp), shape=(n, n))
    xs = sla.spsolve(S.tocsc(), b)
    assert np.linalg.norm(out.x - xs) <= 10 * np.linalg.norm(ref.x - xs) + 1e-13 * np.linalg.norm(xs)
    # the recurrence norm of the last state agrees with the norm of the vector r
    assert out.hist["rho"][out.iters - 1] == pytest.approx(out.rho_rec, rel=1e-5)


def test_finite_termination_with_d_distinct_eigenvalues():
    rng = np.random.default_rng(9)
    n, d = 30, 5
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.repeat([1.0, 2.0, 3.5, 7.0, 11.0], n // d)
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    b = rng.uniform(-1, 1, n)
    out = O.solve(O.Options(min_k=0, variant=1), _dense_csr(A), b, 1e-10, 50, fixed=(4, 4, 4, 4))
    assert out.outcome == O.CONVERGED and out.iters <= d
    assert np.linalg.norm(A @ out.x - b) <= 1e-9 * np.linalg.norm(b)


def _by_hand_sr(A, b, fmts, iters):
    """Chronopoulos and Gear's recurrences, every rounding done by numpy, every sum exact."""
    n = len(b)
    t1, t2, t3, t4 = (TYPES[f] for f in fmts)
    Av = A if t1 is None else np.vectorize(lambda v: float(t1(v)))(A)
    x = np.zeros(n)
    r = b.astype(np.float64).copy()
    p, s = np.zeros(n), np.zeros(n)
    bnorm = sum(float(v) * float(v) for v in b) ** 0.5
    gamma_prev = alpha_prev = None
    out = []
    for k in range(iters):
        u = _chop(r, t2)
        ul = _chop(u, t1)
        w = np.array([_round_to(_exact_dot(Av[i], ul), t1) if t1 else float(_exact_dot(Av[i], ul)) for i in range(n)])
        ru, uu = _chop(r, t4), _chop(u, t4)
        gamma = _round_to(_exact_dot(ru, uu), t4) if t4 else float(_exact_dot(ru, uu))
        wu, uw = _chop(w, t3), _chop(u, t3)
        delta = _round_to(_exact_dot(wu, uw), t3) if t3 else float(_exact_dot(wu, uw))
        if k == 0:
            beta, nu = 0.0, delta
        else:
            beta = gamma / gamma_prev
            nu = delta - beta * gamma / alpha_prev
        alpha = gamma / nu
        # the next residual norm from the pre-update vectors (exact sums, then fp64)
        rr = float(_exact_dot(r, r))
        rw, rs = float(_exact_dot(r, w)), float(_exact_dot(r, s))
        ww, ws, ss = float(_exact_dot(w, w)), float(_exact_dot(w, s)), float(_exact_dot(s, s))
        rr1 = rr - 2.0 * alpha * (rw + beta * rs) + alpha * alpha * (ww + 2.0 * beta * ws + beta * beta * ss)
        p = np.array([u[i] + beta * p[i] for i in range(n)])
        s = np.array([w[i] + beta * s[i] for i in range(n)])
        x = np.array([x[i] + alpha * p[i] for i in range(n)])
        r = np.array([r[i] - alpha * s[i] for i in range(n)])
        out.append((max(rr1, 0.0) ** 0.5 / bnorm, nu, alpha, gamma, beta, x.copy()))
        gamma_prev, alpha_prev = gamma, alpha
    return out


@pytest.mark.parametrize("fmts", [(0, 3, 0, 3), (3, 0, 3, 0), (0, 0, 0, 3), (3, 3, 0, 4), (4, 4, 4, 4)])
def test_first_iterations_match_a_hand_recomputation(fmts):
    rng = np.random.default_rng(7)
    n = 7
    G = rng.standard_normal((n, n))
    A = G @ G.T + n * np.eye(n)
    b = rng.uniform(-1, 1, n)
    out = O.solve(O.Options(min_k=0, variant=1), _dense_csr(A), b, 1e-30, 3, fixed=fmts)
    ref = _by_hand_sr(A, b, fmts, 3)
    for k in range(3):
        rho, nu, alpha, gamma, beta, xk = ref[k]
        h = out.hist[k]
        # gamma (op 4) and delta (op 3) in the low formats: the rounded exact sum, bit for bit
        if fmts[3] != 4:
            assert h["sigma"] == gamma, (k, fmts)
        else:
            assert h["sigma"] == pytest.approx(gamma, rel=1e-14)
        assert h["nu"] == pytest.approx(nu, rel=1e-13) and h["alpha"] == pytest.approx(alpha, rel=1e-13)
        assert h["beta"] == pytest.approx(beta, rel=1e-13, abs=0)
        assert h["rho"] == pytest.approx(rho, rel=1e-9)
    assert np.allclose(out.x, ref[2][5], rtol=1e-12, atol=0)


def test_training_and_greedy_with_the_single_reduction_iteration():
    """Algorithm 1 and Algorithm 2 drive the variant like the CG of Section 3: training on the
    Poisson problem with P = {fp32, fp64} gives a greedy policy that converges."""
    A, b, _ = I.cfg_poisson32()
    o = O.Options(seed=2, min_k=0, variant=1, precs=(O.FP32, O.FP64), cost={O.FP32: 1.0, O.FP64: 2.0})
    qt = O.QTable.zeros(o)
    its = O.train_sequential(o, A, b, 1e-8, 400, 20, qt)
    assert np.all(its < 400)
    out = O.solve(o, A, b, 1e-8, 400, qtable=qt)
    assert out.outcome == O.CONVERGED
    assert qt.visits.sum() == 4 * int(its.sum())
    with pytest.raises(ValueError, match="single-reduction"):
        O.solve(O.Options(variant=1, precond=2), A, b, 1e-8, 10, fixed=(4, 4, 4, 4))
