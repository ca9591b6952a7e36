"""Pins of the oracle's fp32 incomplete Cholesky preconditioner (IC(0), the SPD reading of
Section 5's fixed-precision fp32 incomplete factorization) against facts fixed by the
mathematics: the exact Cholesky factor where IC(0) drops no fill, the defining property
(L L^T)_ij = a_ij on the pattern of A, triangular solves against a dense solver, Kershaw's
SPD matrix on which IC(0) breaks down, and the effect on CG iteration counts."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import oracle as O
from paper_2504_14268_gb300 import inputs as I


def _csr(S):
    S = sp.csr_matrix(S)
    S.sort_indices()
    return (S.shape[0], S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))


def _lower_dense(A, L):
    n, rp, ci, _ = A
    D = np.zeros((n, n))
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            if ci[e] <= i:
                D[i, ci[e]] = L[e]
    return D


def _tridiag(n, rng):
    off = rng.uniform(-1, 1, n - 1)
    d = np.abs(np.concatenate([[0], off])) + np.abs(np.concatenate([off, [0]])) + rng.uniform(0.5, 2, n)
    return _csr(sp.diags([off, d, off], [-1, 0, 1]))


def test_no_fill_pattern_gives_the_cholesky_factor():
    """A tridiagonal matrix has no fill: IC(0) is its Cholesky factor (to fp32 rounding)."""
    A = _tridiag(200, np.random.default_rng(0))
    L = O.ic0(A)
    Ld = _lower_dense(A, L)
    dense = sp.csr_matrix((A[3], A[2], A[1])).toarray()
    C = np.linalg.cholesky(dense)
    assert np.allclose(Ld, C, rtol=0, atol=2e-6 * np.abs(C).max())


def test_product_matches_A_on_its_pattern_and_drops_fill():
    """(L L^T)_ij = a_ij wherever A stores an entry (the definition of IC(0)); the fill
    that a complete factor would need appears only off the pattern."""
    A = I.poisson2d(20)
    n, rp, ci, val = A
    L = O.ic0(A)
    Ld = _lower_dense(A, L)
    P = Ld @ Ld.T
    dense = sp.csr_matrix((val, ci, rp)).toarray()
    on = dense != 0
    assert np.max(np.abs(P[on] - dense[on])) <= 1e-5 * np.abs(dense).max()
    assert np.max(np.abs(P[~on])) > 1e-2  # the dropped fill is visible off the pattern
    # lower part only on the pattern of A, positive diagonal
    assert np.all(Ld[np.tril(~on)] == 0)
    assert np.all(np.diag(Ld) > 0)


def test_upper_positions_hold_the_transposed_factor():
    A = I.poisson2d(12)
    n, rp, ci, _ = A
    L = O.ic0(A)
    pos = {(i, int(ci[e])): e for i in range(n) for e in range(rp[i], rp[i + 1])}
    for (i, j), e in pos.items():
        if j > i:
            assert L[e] == L[pos[(j, i)]]


def test_apply_solves_both_triangles():
    """w = L^-T L^-1 fl32(r): against dense triangular solves of the same factor in fp64."""
    A = I.diffusion_varcoef((7, 6, 5), 1.0, np.random.default_rng(3))
    L = O.ic0(A)
    Ld = _lower_dense(A, L).astype(np.float64)
    r = np.random.default_rng(4).uniform(-1, 1, A[0])
    w = O.ic0_apply(A, L, r)
    assert w.dtype == np.float64 and np.all(w.astype(np.float32).astype(np.float64) == w)
    y = sla.solve_triangular(Ld, r.astype(np.float32).astype(np.float64), lower=True)
    ref = sla.solve_triangular(Ld.T, y, lower=False)
    assert np.allclose(w, ref, rtol=0, atol=1e-5 * np.abs(ref).max())


def test_kershaw_matrix_breaks_down():
    """Kershaw's 4x4 SPD matrix: IC(0) meets a negative pivot."""
    K = np.array([[3.0, -2, 0, 2], [-2, 3, -2, 0], [0, -2, 3, -2], [2, 0, -2, 3]])
    assert np.linalg.eigvalsh(K).min() > 0
    A = _csr(K)
    with pytest.raises(ValueError, match="breaks down"):
        O.ic0(A)
    b = np.ones(4)
    with pytest.raises(ValueError, match="breaks down"):
        O.solve(O.Options(min_k=0, precond=2), A, b, 1e-8, 10, fixed=(4, 4, 4, 4))


def test_unusable_patterns_are_refused():
    n, rp, ci, val = I.poisson2d(4)
    ci2 = ci.copy()
    ci2[[0, 1]] = ci2[[1, 0]]  # row 0 columns out of order
    val2 = val.copy()
    val2[[0, 1]] = val2[[1, 0]]
    with pytest.raises(ValueError, match="strictly increasing"):
        O.ic0((n, rp, ci2, val2))
    # an unsymmetric pattern: drop one off-diagonal entry of row 0
    S = sp.csr_matrix((val, ci, rp)).tolil()
    S[0, 1] = 0.0
    S = sp.csr_matrix(S)
    S.eliminate_zeros()
    with pytest.raises(ValueError, match="symmetric"):
        O.ic0(_csr(S))


def test_exact_factor_gives_one_step_convergence():
    """With no fill dropped, M = A up to fp32: preconditioned CG reaches the fp32 level of
    M^-1 in one or two iterations."""
    A = _tridiag(300, np.random.default_rng(5))
    xs, b = I.rhs_from_xstar(A, np.random.default_rng(6))
    out = O.solve(O.Options(min_k=0, precond=2), A, b, 1e-5, 50, fixed=(4, 4, 4, 4))
    assert out.outcome == O.CONVERGED and out.iters <= 2


def test_ic0_cuts_cg_iterations_on_poisson():
    A, b, xs = I.cfg_poisson32()
    plain = O.solve(O.Options(min_k=0), A, b, 1e-8, 1000, fixed=(4, 4, 4, 4))
    ic = O.solve(O.Options(min_k=0, precond=2), A, b, 1e-8, 1000, fixed=(4, 4, 4, 4))
    assert plain.outcome == ic.outcome == O.CONVERGED
    assert ic.iters <= 0.6 * plain.iters
    assert np.linalg.norm(ic.x - xs) / np.linalg.norm(xs) < 1e-6
    # low-precision operations on top of the fp32 preconditioner still converge
    mixed = O.solve(O.Options(min_k=0, precond=2), A, b, 1e-6, 1000, fixed=(3, 1, 3, 3))
    assert mixed.outcome == O.CONVERGED


def test_fp32_preconditioner_output_is_exact_in_fp32():
    """M^-1 r is computed in fp32, so rounding it to fp32 (p2 = fp32) changes nothing: the
    solve is bit-identical to p2 = fp64, while p2 = fp16 is not."""
    A, b, xs = I.cfg_poisson32()
    o = O.Options(min_k=0, precond=2)
    a = O.solve(o, A, b, 1e-8, 300, fixed=(4, 4, 4, 4))
    c = O.solve(o, A, b, 1e-8, 300, fixed=(4, 3, 4, 4))
    assert a.iters == c.iters and np.array_equal(a.x, c.x) and np.array_equal(a.hist["rho"], c.hist["rho"])
    d = O.solve(o, A, b, 1e-8, 300, fixed=(4, 0, 4, 4))
    assert not np.array_equal(a.hist["rho"][: d.iters], d.hist["rho"][: a.iters][: d.iters])
