"""The generators of the paper's two experiment families (Section 5.1: B B^T + beta I;
Section 5.2: Poisson on random subdomains) against what their descriptions fix: sizes, pair
counts, the range of beta and the Rayleigh-quotient floor it gives, symmetry, and for the
Poisson family the exactness of the five-point scheme on linear functions (which checks the
assembly of the boundary data into b)."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla

from paper_2504_14268_gb300 import inputs as I


def _S(A):
    n, rp, ci, val = A
    return sp.csr_matrix((val, ci, rp), shape=(n, n))


def test_bbt_family():
    for seed in range(5):
        A, b = I.synth_bbt(seed)
        S = _S(A)
        assert S.shape == (5000, 5000) and b.shape == (5000,)
        assert abs(S - S.T).max() == 0.0
        d = S.diagonal()
        # beta I is the floor: a_ii >= beta >= 1e-4 and x^T A x >= beta |x|^2
        assert d.min() >= 1e-4 and d.min() <= 1e-2 + 1e-12
        x = np.random.default_rng(seed).standard_normal(5000)
        assert x @ (S @ x) >= 1e-4 * (x @ x)
        assert np.all(np.abs(b) <= 1.0)
        # B has 5000 entries, so B B^T has at most about that many off-diagonal pairs
        assert S.nnz - 5000 <= 2 * 5000
    ood = [I.synth_bbt(seed, ood=True)[0] for seed in range(5)]
    assert len({_S(A).nnz for A in ood}) > 1


def test_poisson_subdomain_is_exact_on_linear_functions():
    """f = 0 with boundary data from u = c0 + c1 x + c2 y: the five-point scheme reproduces u
    at the interior points exactly (up to the direct solver's rounding)."""
    ax, bx, ay, by, m = 0.3, 1.1, 0.5, 1.9, 20
    c0, c1, c2 = 0.7, -1.3, 2.1
    u = lambda x, y: c0 + c1 * x + c2 * y
    A, b = I.poisson_subdomain_system(
        ax, bx, ay, by, m, lambda x, y: np.zeros_like(x),
        lambda t: u(ax, ay + t * (by - ay)), lambda t: u(bx, ay + t * (by - ay)),
        lambda t: u(ax + t * (bx - ax), ay), lambda t: u(ax + t * (bx - ax), by))
    x = sla.spsolve(_S(A).tocsc(), b)
    hx, hy = (bx - ax) / (m + 1), (by - ay) / (m + 1)
    X, Y = np.meshgrid(ax + hx * np.arange(1, m + 1), ay + hy * np.arange(1, m + 1))
    assert np.allclose(x, u(X, Y).ravel(), rtol=0, atol=1e-10)


def test_poisson_subdomain_family():
    for seed in range(5):
        A, b = I.poisson_subdomain(seed)
        S = _S(A)
        assert S.shape == (6400, 6400) and b.shape == (6400,)
        assert abs(S - S.T).max() == 0.0
        assert np.all(np.diff(A[1]) <= 5)
        # the subdomain lies in [0, 2]^2 with edges of at least 0.1: 2 / h^2 >= 2 (81 / 2)^2
        assert S.diagonal().min() >= 2 * 2 * (81 / 2.0) ** 2 - 1e-6


def test_experiment_statistics_helpers():
    from paper_2504_14268_gb300 import experiments as E

    st = E._stats([1, 2, 3, 4])
    assert st["mean"] == 2.5 and st["max"] == 4 and st["p25"] == 1.75 and st["p75"] == 3.25
    h1 = np.zeros((4, 8), dtype=np.int64)
    h1[:, 4] = 3  # three fp64 iterations
    h2 = np.zeros((4, 8), dtype=np.int64)
    h2[0, 0] = 2  # op 1 in fp16 twice, the other ops in fp32
    h2[1:, 3] = 2
    sh = E.format_shares([h1, h2])
    assert abs(sum(sh.values()) - 1.0) < 1e-12
    assert sh["fp64"] == 12 / 20 and sh["fp16"] == 2 / 20 and sh["fp32"] == 6 / 20
