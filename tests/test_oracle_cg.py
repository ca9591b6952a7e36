"""Pins for the oracle's CG (Section 3 Eq. (1)-(4), Section 4.2, Algorithm 2).

Independent references: dense Cholesky / LAPACK solves, the Krylov-projection
characterisation of CG iterates (brute force), finite termination for matrices with d
distinct eigenvalues, A-orthogonality of the directions, monotone A-norm error, scipy's
CG (a library routine) for the all-fp64 special case, numpy float16/float32 rounding
(library routines) for the low-precision building blocks, and the closed-form spectrum of
the 2D Poisson matrix."""
import math

import numpy as np
import pytest
import scipy.linalg as la
import scipy.sparse as sp

import oracle as O
from paper_2504_14268_gb300 import inputs as I

ALL64 = (O.FP64, O.FP64, O.FP64, O.FP64)


def _dense(A):
    n, rp, ci, val = A
    return sp.csr_matrix((val, ci, rp), shape=(n, n)).toarray()


def _csr_from_dense(D):
    S = sp.csr_matrix(D)
    S.sort_indices()
    return (D.shape[0], S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))


def _opts(**kw):
    kw.setdefault("min_k", 0)
    return O.Options(**kw)


def _iterates(A, b, kmax):
    """x_k for k = 0..kmax by running the oracle with max_iter = k (x_0 = 0)."""
    xs = [np.zeros(A[0])]
    for k in range(1, kmax + 1):
        out = O.solve(_opts(), A, b, 0.0, k, fixed=ALL64)
        xs.append(out.x)
    return xs


@pytest.mark.parametrize("n,seed", [(8, 0), (30, 1), (64, 2)])
def test_fp64_cg_matches_cholesky(n, seed):
    rng = np.random.default_rng(seed)
    A = I.random_spd_small(n, rng)
    D = _dense(A)
    xs = rng.uniform(-1, 1, n)
    b = D @ xs
    ref = la.cho_solve(la.cho_factor(D), b)
    out = O.solve(_opts(), A, b, 1e-13, 10 * n, fixed=ALL64)
    assert out.outcome == O.CONVERGED
    assert np.linalg.norm(out.x - ref) / np.linalg.norm(ref) < 1e-9
    assert out.rho_true < 1e-11


def test_iterates_are_krylov_projections():
    """x_k = argmin over K_k(A, b) of ||x - x*||_A, computed by a dense solve on a basis."""
    rng = np.random.default_rng(3)
    n = 24
    A = I.random_spd_small(n, rng, density=0.4, shift=1.0)
    D = _dense(A)
    b = rng.standard_normal(n)
    xs = _iterates(A, b, 8)
    K = [b / np.linalg.norm(b)]
    for k in range(1, 9):
        V, _ = np.linalg.qr(np.column_stack(K))
        y = np.linalg.solve(V.T @ D @ V, V.T @ b)
        ref = V @ y
        assert np.linalg.norm(xs[k] - ref) <= 1e-9 * np.linalg.norm(ref)
        nxt = D @ K[-1]
        K.append(nxt / np.linalg.norm(nxt))


def test_finite_termination_distinct_eigenvalues():
    """CG on a matrix with d distinct eigenvalues terminates in at most d iterations."""
    rng = np.random.default_rng(4)
    n, d = 40, 5
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.repeat(np.array([1.0, 2.5, 4.0, 7.0, 11.0]), n // d)
    D = (Q * lam) @ Q.T
    D = 0.5 * (D + D.T)
    A = _csr_from_dense(D)
    b = rng.standard_normal(n)
    out = O.solve(_opts(), A, b, 1e-10, 100, fixed=ALL64)
    assert out.outcome == O.CONVERGED and out.iters <= d


def test_a_orthogonality_and_monotone_a_norm():
    rng = np.random.default_rng(5)
    n = 50
    A = I.random_spd_small(n, rng, density=0.2, shift=2.0)
    D = _dense(A)
    xstar = rng.uniform(-1, 1, n)
    b = D @ xstar
    xs = _iterates(A, b, 12)
    dirs = [xs[k + 1] - xs[k] for k in range(12)]  # alpha_k p_k
    for i in range(12):
        for j in range(i):
            c = dirs[i] @ D @ dirs[j] / math.sqrt((dirs[i] @ D @ dirs[i]) * (dirs[j] @ D @ dirs[j]))
            assert abs(c) < 1e-8
    errs = [math.sqrt((x - xstar) @ D @ (x - xstar)) for x in xs]
    assert all(errs[k + 1] <= errs[k] * (1 + 1e-12) for k in range(12))
    # residuals of successive iterates are mutually orthogonal
    rs = [b - D @ x for x in xs[:8]]
    for i in range(8):
        for j in range(i):
            assert abs(rs[i] @ rs[j]) <= 1e-8 * np.linalg.norm(rs[i]) * np.linalg.norm(rs[j])


def test_all_fp64_equals_scipy_cg():
    """With every operation in fp64 the method is plain CG: scipy.sparse.linalg.cg after k
    iterations (rtol 0, so it does not stop early) gives the same iterate."""
    from scipy.sparse.linalg import cg

    A, b, _ = I.cfg_poisson32()
    S = sp.csr_matrix((A[3], A[2], A[1]), shape=(A[0], A[0]))
    for k in (1, 5, 20, 60):
        ref, _ = cg(S, b, x0=np.zeros(A[0]), rtol=0.0, atol=0.0, maxiter=k)
        out = O.solve(_opts(), A, b, 0.0, k, fixed=ALL64)
        assert np.linalg.norm(out.x - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("fmt,np_t", [(O.FP16, np.float16), (O.FP32, np.float32)])
def test_spmv_and_dot_building_blocks_match_library_rounding(fmt, np_t):
    """q = fl(A fl(p)) and fl(x^T y) against numpy's own float16/float32 rounding with an fp64
    sparse product: equal up to a one-ulp difference where the fp64 sums differ in order."""
    rng = np.random.default_rng(6)
    A, b, _ = I.cfg_poisson32()
    n = A[0]
    p = rng.standard_normal(n)
    S = sp.csr_matrix((A[3].astype(np_t).astype(np.float64), A[2], A[1]), shape=(n, n))
    acc = S @ p.astype(np_t).astype(np.float64)
    ref = acc.astype(np_t).astype(np.float64)
    got = O.spmv(A, fmt, p)
    ulp = np.spacing(np.abs(ref).astype(np_t)).astype(np.float64)
    assert np.all(np.abs(got - ref) <= ulp)
    assert np.mean(got == ref) > 0.99
    x, y = rng.standard_normal(n), rng.standard_normal(n)
    s = math.fsum((x.astype(np_t).astype(np.float64) * y.astype(np_t).astype(np.float64)).tolist())
    ref_d = float(np_t(s))
    got_d = O.dot(x, y, fmt)
    assert abs(got_d - ref_d) <= float(np.spacing(np_t(abs(ref_d))))


def test_row_scaled_spmv_is_scale_invariant():
    """Scaling A by a power of two scales a row-scaled product exactly; for a matrix inside
    the format's normal range the row-scaled product equals the unscaled one."""
    rng = np.random.default_rng(7)
    A, b, _ = I.cfg_poisson32()
    p = rng.uniform(-1, 1, A[0])
    big = (A[0], A[1], A[2], A[3] * 2.0 ** 40)
    for fr, f in ((O.FP16R, O.FP16), (O.BF16R, O.BF16)):
        q1 = O.spmv(A, fr, p)
        q2 = O.spmv(big, fr, p)
        assert np.array_equal(q2, q1 * 2.0 ** 40)
        assert np.array_equal(q1, O.spmv(A, f, p))
    # plain fp16 overflows on the scaled matrix, row-scaled fp16 does not
    assert not np.any(np.isfinite(O.spmv(big, O.FP16, p)))
    assert np.all(np.isfinite(O.spmv(big, O.FP16R, p)))


def test_poisson32_iteration_count_within_closed_form_bound():
    """lambda_ij = 4 - 2 cos(i pi / 33) - 2 cos(j pi / 33); CG's Chebyshev bound on the residual
    ||r_k|| / ||r_0|| <= 2 sqrt(kappa) ((sqrt(kappa) - 1) / (sqrt(kappa) + 1))^k caps the count."""
    A, b, xs = I.cfg_poisson32()
    th = np.arange(1, 33) * math.pi / 33
    lam = (2 - 2 * np.cos(th))[:, None] + (2 - 2 * np.cos(th))[None, :]
    kappa = lam.max() / lam.min()
    assert abs(kappa - 440.69) < 0.01
    ev = np.linalg.eigvalsh(_dense(A))
    assert abs(ev.max() / ev.min() - kappa) < 1e-6 * kappa
    sk = math.sqrt(kappa)
    kbound = math.ceil(math.log(1e-10 / (2 * sk)) / math.log((sk - 1) / (sk + 1)))
    out = O.solve(_opts(), A, b, 1e-10, 1000, fixed=ALL64)
    assert out.outcome == O.CONVERGED and out.iters <= kbound
    assert np.linalg.norm(out.x - xs) / np.linalg.norm(xs) < 1e-7


def test_fixed_low_precision_stagnates_at_roundoff_level():
    """All-fp32 / all-fp16 operations: the true residual stalls near c u kappa, below one but
    far above the fp64 level (invariant: lower precision never beats the fp64 solve)."""
    A, b, xs = I.cfg_poisson32()
    res = {}
    for f in (O.FP64, O.FP32, O.FP16):
        out = O.solve(_opts(), A, b, 1e-10, 1000, fixed=(f, f, f, f))
        res[f] = out.rho_true
    assert res[O.FP64] < 1e-9
    assert 1e-9 < res[O.FP32] < 1e-3
    assert res[O.FP32] < res[O.FP16] < 1.0


def test_zero_rhs_and_empty():
    A, b, _ = I.cfg_poisson32()
    out = O.solve(_opts(), A, np.zeros(A[0]), 1e-8, 100, fixed=ALL64)
    assert out.outcome == O.CONVERGED and out.iters == 0 and not out.x.any()
    E = (0, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    out = O.solve(_opts(), E, np.zeros(0), 1e-8, 100, fixed=ALL64)
    assert out.outcome == O.CONVERGED and out.iters == 0


def test_breakdown_on_indefinite_matrix():
    """p_0^T A p_0 < 0: the curvature test stops at k = 0 and keeps x_0."""
    D = np.diag([1.0, -3.0, 2.0])
    A = _csr_from_dense(D)
    out = O.solve(_opts(), A, np.array([0.0, 1.0, 0.0]), 1e-8, 50, fixed=ALL64)
    assert out.outcome == O.BREAKDOWN and out.iters == 0 and not out.x.any()


def test_breakdown_on_fp16_overflow():
    """Entries above 65504 overflow fp16: q becomes infinite and nu is not finite."""
    A, b, _ = I.cfg_poisson32()
    big = (A[0], A[1], A[2], A[3] * 1e5)
    out = O.solve(_opts(), big, b, 1e-8, 50, fixed=(O.FP16, O.FP64, O.FP64, O.FP64))
    assert out.outcome == O.BREAKDOWN and out.iters == 0
    out = O.solve(_opts(), big, b, 1e-8, 50, fixed=(O.FP16R, O.FP64, O.FP64, O.FP64))
    assert out.outcome != O.BREAKDOWN


def test_min_k_rule_gives_eleven_iterations():
    """Section 5 stops when rho_k < tol and k >= 10, so a system that converges in a few
    iterations still reports 11, as Table 4's fp64 rows do (11.0 everywhere)."""
    rng = np.random.default_rng(8)
    A = I.random_spd_small(12, rng, density=0.5, shift=4.0)
    b = rng.standard_normal(12)
    quick = O.solve(_opts(), A, b, 1e-6, 1000, fixed=ALL64)
    assert quick.outcome == O.CONVERGED and quick.iters <= 10
    out = O.solve(O.Options(min_k=10), A, b, 1e-6, 1000, fixed=ALL64)
    assert out.outcome == O.CONVERGED and out.iters == 11


def test_exact_solution_before_min_k_is_convergence():
    """A = 2 I is solved exactly in one step; with the k >= 10 rule the next direction is zero
    (nu = 0) and the solve ends as converged, not as a breakdown."""
    D = np.diag(np.full(6, 2.0))
    A = _csr_from_dense(D)
    b = np.arange(1.0, 7.0)
    out = O.solve(O.Options(min_k=10), A, b, 1e-6, 1000, fixed=ALL64)
    assert out.outcome == O.CONVERGED and out.iters == 1
    assert np.array_equal(out.x, b / 2)


def test_true_residual_replacement_restores_accuracy():
    """With fp16 products the recursive residual drifts below the true one; confirming a
    claimed convergence with b - A x (fp64) replaces r and the solve continues."""
    A, b, xs = I.cfg_poisson32()
    sched = [(O.FP16, O.FP16, O.FP32, O.FP32)] * 60 + [ALL64] * 1000
    plain = O.solve(_opts(), A, b, 1e-8, 1000, sched=sched)
    checked = O.solve(_opts(true_res_at_conv=1), A, b, 1e-8, 1000, sched=sched)
    assert checked.outcome == O.CONVERGED and checked.rho_true < 1e-8
    assert plain.rho_true >= checked.rho_true or plain.rho_true < 1e-8


# ---- Jacobi preconditioning (op 2 with M = diag(A)) ------------------------------------

def _scaled(A):
    """D^-1/2 A D^-1/2 for a CSR matrix with positive diagonal D."""
    n, rp, ci, val = A
    D = np.zeros(n)
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            if ci[e] == i:
                D[i] = val[e]
    s = 1.0 / np.sqrt(D)
    rows = np.repeat(np.arange(n), np.diff(rp))
    return (n, rp.copy(), ci.copy(), val * s[rows] * s[ci]), s


def test_jacobi_pcg_is_cg_on_the_symmetrically_scaled_system():
    """Jacobi-preconditioned CG on A x = b and plain CG on (D^-1/2 A D^-1/2) y = D^-1/2 b
    produce the same iterates x_k = D^-1/2 y_k (exact arithmetic); in fp64 they agree to
    rounding after every number of steps."""
    rng = np.random.default_rng(5)
    A = I.diffusion_varcoef((7, 6, 5), 2.0, rng)
    _, b = I.rhs_from_xstar(A, rng)
    As, s = _scaled(A)
    for k in (1, 3, 8, 20):
        xo = O.solve(_opts(precond=1), A, b, 1e-30, k, fixed=(4, 4, 4, 4)).x
        ys = O.solve(_opts(), As, b * s, 1e-30, k, fixed=(4, 4, 4, 4)).x
        assert np.allclose(xo, ys * s, rtol=1e-9, atol=1e-12 * np.abs(xo).max())


def test_jacobi_on_a_diagonal_matrix_converges_in_one_step():
    """M = A: z_0 = A^-1 b is the solution and the first step reaches it."""
    n = 12
    d = np.linspace(0.5, 40.0, n)
    A = (n, np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d)
    b = np.arange(1.0, n + 1.0)
    out = O.solve(_opts(precond=1), A, b, 1e-12, 5, fixed=(4, 4, 4, 4))
    assert out.outcome == O.CONVERGED and out.iters == 1
    assert np.allclose(out.x, b / d, rtol=1e-15)
    plain = O.solve(_opts(), A, b, 1e-12, 50, fixed=(4, 4, 4, 4))
    assert plain.iters > 1


def test_jacobi_with_power_of_two_diagonal_is_plain_cg_bit_for_bit():
    """The 2D Poisson matrix has 4 on the diagonal: M = 4 I scales z, p and sigma by exact
    powers of two, so every iterate and residual equals plain CG's exactly."""
    A, b, _ = I.cfg_poisson32()
    o1 = O.solve(_opts(precond=1), A, b, 1e-10, 200, fixed=(4, 4, 4, 4))
    o0 = O.solve(_opts(), A, b, 1e-10, 200, fixed=(4, 4, 4, 4))
    assert o1.iters == o0.iters
    assert np.array_equal(o1.x, o0.x)
    assert np.array_equal(o1.hist["rho"], o0.hist["rho"])


def test_jacobi_reduces_iterations_on_variable_coefficients():
    """Coefficients varying over orders of magnitude: diagonal scaling removes most of the
    ill-conditioning that comes from the coefficient contrast."""
    rng = np.random.default_rng(8)
    A = I.diffusion_varcoef((10, 10, 10), 2.5, rng)
    _, b = I.rhs_from_xstar(A, rng)
    o0 = O.solve(_opts(), A, b, 1e-8, 5000, fixed=(4, 4, 4, 4))
    o1 = O.solve(_opts(precond=1), A, b, 1e-8, 5000, fixed=(4, 4, 4, 4))
    assert o0.outcome == o1.outcome == O.CONVERGED
    assert o1.iters < 0.7 * o0.iters


def test_jacobi_low_precision_z_is_the_rounded_fp64_product():
    """With p2 = fp16 the first direction after the start is z_1 = fl_16(r_1 d) (one rounding
    of the fp64 product): a one-step solve recovers it from p_1 = z_1 + beta_0 p_0."""
    rng = np.random.default_rng(9)
    A = I.diffusion_varcoef((5, 5, 4), 1.0, rng)
    _, b = I.rhs_from_xstar(A, rng)
    n, rp, ci, val = A
    out = O.solve(_opts(precond=1), A, b, 1e-30, 1, fixed=(4, 0, 4, 4))
    h = out.hist[0]
    D = np.array([val[rp[i]:rp[i + 1]][ci[rp[i]:rp[i + 1]] == i][0] for i in range(n)])
    dinv = 1.0 / D
    r0 = b.copy()
    p0 = r0 * dinv
    r1 = r0 - h["alpha"] * np.asarray(O.spmv(A, 4, p0))
    z1 = O.chop(r1 * dinv, O.FP16)
    assert h["sigma"] == pytest.approx(float(np.dot(r1, z1)), rel=1e-12)


def test_jacobi_refuses_a_row_without_positive_diagonal():
    A = _csr_from_dense(np.array([[2.0, 1.0], [1.0, 0.0]]))
    with pytest.raises(ValueError, match="positive diagonal"):
        O.solve(_opts(precond=1), A, np.ones(2), 1e-8, 10, fixed=(4, 4, 4, 4))
