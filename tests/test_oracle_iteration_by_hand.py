"""Pin of the composition of one mixed-precision CG iteration (Eq. 1-4 with the operation
precisions of Section 4.2): the oracle's first two iterations on a small SPD system against
a step-by-step recomputation that shares nothing with it. Sums are exact (Python Fractions)
and each operation output is rounded once to its format by nearest-even selection between
numpy's own float16 / float32 neighbours (the oracle's low-precision results must equal
these bit for bit); the fp64 steps (alpha, x and r updates, beta, the
direction update) are plain Python floats."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O


def _round_to(v: Fraction, t):
    """The element of numpy type t nearest to the exact value v (ties to even)."""
    c = t(float(v))  # within one unit of the answer (double rounding can be off by one)
    best = None
    for cand in (np.nextafter(c, t(-np.inf)), c, np.nextafter(c, t(np.inf))):
        if not np.isfinite(cand):
            continue
        d = abs(Fraction(float(cand)) - v)
        key = (d, int(np.frombuffer(cand.tobytes(), dtype=np.uint16 if t is np.float16 else np.uint32)[0]) & 1)
        if best is None or key < best[0]:
            best = (key, cand)
    return float(best[1])


def _exact_dot(a, b):
    return sum((Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b)), Fraction(0))


def _chop(x, t):
    return np.array([float(t(v)) for v in x]) if t is not None else np.array(x, dtype=np.float64)


TYPES = {0: np.float16, 3: np.float32, 4: None}


def _by_hand(A, b, fmts, iters):
    n = len(b)
    t1, t2, t3, t4 = (TYPES[f] for f in fmts)
    Av = A if t1 is None else np.vectorize(lambda v: float(t1(v)))(A)
    x = np.zeros(n)
    r = b.astype(np.float64).copy()
    p = r.copy()  # z_0 = r_0 (M = I), p_0 = z_0
    sigma = sum(float(v) * float(v) for v in r)  # fp64, in index order
    bnorm = sum(float(v) * float(v) for v in b) ** 0.5
    out = []
    for k in range(iters):
        pl = _chop(p, t1)
        q = np.array([_round_to(_exact_dot(Av[i], pl), t1) if t1 else float(_exact_dot(Av[i], pl)) for i in range(n)])
        pn, qn = _chop(p, t3), _chop(q, t3)
        nu = _round_to(_exact_dot(pn, qn), t3) if t3 else float(_exact_dot(pn, qn))
        alpha = sigma / nu
        x = np.array([x[i] + alpha * p[i] for i in range(n)])
        r = np.array([r[i] - alpha * q[i] for i in range(n)])
        rho = sum(float(v) * float(v) for v in r) ** 0.5 / bnorm
        z = _chop(r, t2)
        rs, zs = _chop(r, t4), _chop(z, t4)
        sig_new = _round_to(_exact_dot(rs, zs), t4) if t4 else float(_exact_dot(rs, zs))
        beta = sig_new / sigma
        p = np.array([z[i] + beta * p[i] for i in range(n)])
        sigma = sig_new
        out.append((rho, nu, alpha, sig_new, beta, x.copy()))
    return out


@pytest.mark.parametrize("fmts", [(0, 3, 0, 3), (3, 0, 3, 0), (0, 0, 0, 3), (0, 3, 3, 0), (3, 0, 0, 3), (0, 0, 3, 3), (3, 3, 0, 4), (4, 4, 4, 4)])
def test_first_iterations_match_a_hand_recomputation(fmts):
    rng = np.random.default_rng(7)
    n = 7
    G = rng.standard_normal((n, n))
    A = G @ G.T + n * np.eye(n)
    b = rng.uniform(-1, 1, n)
    rp = np.arange(0, n * n + 1, n, dtype=np.int32)
    ci = np.tile(np.arange(n, dtype=np.int32), n)
    csr = (n, rp, ci, A.ravel())
    out = O.solve(O.Options(min_k=0), csr, b, 1e-30, 2, fixed=fmts)
    ref = _by_hand(A, b, fmts, 2)
    for k in range(2):
        rho, nu, alpha, sig, beta, xk = ref[k]
        h = out.hist[k]
        # low formats: the rounded exact sum, bit for bit; fp64: the oracle sums in index
        # order, within a few units of the exact sum
        for got, want, f in ((h["nu"], nu, fmts[2]), (h["sigma"], sig, fmts[3])):
            if f == 4:
                assert got == pytest.approx(want, rel=1e-14), (k, fmts)
            else:
                assert got == want, (k, fmts)
        assert h["alpha"] == pytest.approx(alpha, rel=1e-15) and h["beta"] == pytest.approx(beta, rel=1e-15)
        assert h["rho"] == pytest.approx(rho, rel=1e-13)
    assert np.allclose(out.x, ref[1][5], rtol=1e-13, atol=0)
