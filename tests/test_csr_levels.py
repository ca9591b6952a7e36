"""Host scheduling analysis of the IC(0) substitutions (mpcg_csr_levels, no GPU): levels
against closed forms (2D five-point grid: x + y; 27-point grid: x + 2y + 4z bounds; a
tridiagonal matrix: one row per level; a diagonal matrix: one level) and against a
longest-path computation over the dependency graph."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2504_14268_gb300 import inputs as I


@pytest.fixture(scope="module")
def M():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2504_14268_gb300 import mpcg

    return mpcg


def _longest_paths(A):
    n, rp, ci, _ = A
    lo = [0] * n
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            if ci[e] < i:
                lo[i] = max(lo[i], lo[ci[e]] + 1)
    up = [0] * n
    for i in range(n - 1, -1, -1):
        for e in range(rp[i], rp[i + 1]):
            if ci[e] > i:
                up[i] = max(up[i], up[ci[e]] + 1)
    return np.array(lo), np.array(up)


def test_poisson_levels_are_x_plus_y(M):
    m = 13
    lo, up, depth = M.csr_levels(I.poisson2d(m))
    x, y = np.meshgrid(np.arange(m), np.arange(m))
    assert np.array_equal(lo, (x + y).ravel())
    assert np.array_equal(up, (2 * (m - 1) - x - y).ravel())
    assert depth == (2 * m - 1, 2 * m - 1)


def test_special_patterns(M):
    n = 50
    T = sp.diags([np.ones(n - 1), 2 * np.ones(n), np.ones(n - 1)], [-1, 0, 1]).tocsr()
    lo, up, depth = M.csr_levels((n, T.indptr, T.indices, T.data))
    assert np.array_equal(lo, np.arange(n)) and depth == (n, n)
    D = sp.identity(n, format="csr")
    lo, up, depth = M.csr_levels((n, D.indptr, D.indices, D.data))
    assert not lo.any() and not up.any() and depth == (1, 1)
    assert M.csr_levels((0, np.zeros(1, dtype=np.int32), np.zeros(0, dtype=np.int32), None))[2] == (0, 0)


def test_fem27_and_random_patterns_match_longest_paths(M):
    N = 6
    A = I.fem27_aniso(N)
    lo, up, depth = M.csr_levels(A)
    rlo, rup = _longest_paths(A)
    assert np.array_equal(lo, rlo) and np.array_equal(up, rup)
    # at least x + 2y + 4z along the grid's dependency chains (the substitutions' depth)
    assert depth[0] >= 7 * (N - 1) + 1
    B = I.random_spd_small(60, np.random.default_rng(3))
    lo, up, _ = M.csr_levels(B)
    rlo, rup = _longest_paths(B)
    assert np.array_equal(lo, rlo) and np.array_equal(up, rup)


def test_invalid_csr_is_refused(M):
    rp = np.array([0, 2, 1], dtype=np.int32)
    ci = np.array([0, 1], dtype=np.int32)
    with pytest.raises(M.MpcgError):
        M.csr_levels((2, rp, ci, None))
    with pytest.raises(M.MpcgError):
        M.csr_levels((2, np.array([0, 1, 2], dtype=np.int32), np.array([0, 5], dtype=np.int32), None))
