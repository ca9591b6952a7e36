"""Host scheduling analysis of the IC(0) substitutions (mpcg_csr_levels, no GPU): levels
against closed forms (2D five-point grid: x + y; 27-point grid: x + 2y + 4z bounds; a
tridiagonal matrix: one row per level; a diagonal matrix: one level) and by the two
properties that define the levels on other patterns."""
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


def _check_level_properties(A, lo, up):
    """The two properties that define the levels (by induction over the rows they determine
    every level uniquely): a row's level is above the level of every row it depends on, and a
    row with dependencies sits exactly one above the highest of them (a row without any at 0).
    Lower substitution: dependencies are the stored columns j < i; upper: j > i."""
    n, rp, ci, _ = A
    for lev, dep in ((lo, lambda i, j: j < i), (up, lambda i, j: j > i)):
        for i in range(n):
            deps = [int(j) for j in ci[rp[i]:rp[i + 1]] if dep(i, j)]
            if not deps:
                assert lev[i] == 0, i
                continue
            assert all(lev[j] < lev[i] for j in deps), i
            assert max(lev[j] for j in deps) == lev[i] - 1, i


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


def test_fem27_and_random_patterns_satisfy_the_level_properties(M):
    N = 6
    A = I.fem27_aniso(N)
    lo, up, depth = M.csr_levels(A)
    _check_level_properties(A, lo, up)
    assert depth == (int(lo.max()) + 1, int(up.max()) + 1)
    # at least x + 2y + 4z along the grid's dependency chains (the substitutions' depth)
    assert depth[0] >= 7 * (N - 1) + 1
    B = I.random_spd_small(60, np.random.default_rng(3))
    lo, up, depth = M.csr_levels(B)
    _check_level_properties(B, lo, up)
    assert depth == (int(lo.max()) + 1, int(up.max()) + 1)


def test_invalid_csr_is_refused(M):
    rp = np.array([0, 2, 1], dtype=np.int32)
    ci = np.array([0, 1], dtype=np.int32)
    with pytest.raises(M.MpcgError):
        M.csr_levels((2, rp, ci, None))
    with pytest.raises(M.MpcgError):
        M.csr_levels((2, np.array([0, 1, 2], dtype=np.int32), np.array([0, 5], dtype=np.int32), None))
