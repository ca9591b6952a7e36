"""Seeded synthetic workloads (sparse SPD systems in CSR) shaped like the paper's.

This module holds input construction only -- no part of the solver's arithmetic. It is
the one module that both the CUDA path and the CPU oracle take their inputs from.

A CSR matrix is the tuple ``(n, row_ptr int32[n+1], col int32[nnz], val float64[nnz])``,
columns sorted within each row, every row holding its (positive) diagonal entry.

Workloads (Section 5 of the paper uses a synthetic B B^T + beta I family and 2D Poisson
problems; these keep its character at the sizes a GPU needs):

* ``poisson2d``          -- 5-point Dirichlet Laplacian (4 on the diagonal, -1 off).
* ``diffusion_varcoef``  -- 2D 5-point / 3D 7-point cell-centred diffusion with log-normal
                            cell coefficients and harmonic-mean faces.
* ``fem27_aniso``        -- Q1 finite-element 27-point stencil of -div(K grad u),
                            K = diag(1, 1, eps), as K (x) M (x) M + M (x) K (x) M + eps M (x) M (x) K.
* ``banded_spd``         -- banded L L^T (N(0,1) lower factor) shifted by lambda_t I.
* ``ba_laplacian``       -- shifted graph Laplacian of a Barabasi-Albert-style power-law graph.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "poisson2d", "diffusion_varcoef", "fem27_aniso", "fem27_spectrum", "banded_spd", "ba_laplacian",
    "rhs_from_xstar", "rng_for", "cfg_poisson32", "cfg_train_set", "cfg_batched", "random_spd_small",
    "synth_bbt", "poisson_subdomain", "poisson_subdomain_system",
]


def rng_for(*key: int) -> np.random.Generator:
    """Independent generator for a workload key, e.g. rng_for(config, instance)."""
    return np.random.default_rng(np.random.SeedSequence(list(key)))


def _from_scipy(S):
    S = S.tocsr()
    S.sum_duplicates()
    S.sort_indices()
    return (S.shape[0], S.indptr.astype(np.int32), S.indices.astype(np.int32), S.data.astype(np.float64))


def poisson2d(m: int):
    """2D 5-point Laplacian on an m x m interior grid, unscaled: n = m^2, Z = 5 m^2 - 4 m."""
    import scipy.sparse as sp

    T = sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1])
    I = sp.identity(m)
    return _from_scipy(sp.kron(T, I) + sp.kron(I, T))


def diffusion_varcoef(shape, sigma: float, rng: np.random.Generator):
    """Cell-centred finite-volume diffusion on a 2D or 3D grid (5- or 7-point).

    Cell coefficient kappa_c = exp(sigma N(0,1)); the coefficient of an interior face is the
    harmonic mean of its two cells; a Dirichlet boundary face adds 2 kappa_c to the diagonal.
    Rows are ordered lexicographically (last axis fastest)."""
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    n = int(np.prod(shape))
    kap = np.exp(sigma * rng.standard_normal(shape))
    idx = np.arange(n, dtype=np.int64).reshape(shape)
    diag = np.zeros(shape)
    rows, cols, vals = [], [], []
    for ax in range(d):
        lo = [slice(None)] * d
        hi = [slice(None)] * d
        lo[ax] = slice(0, shape[ax] - 1)
        hi[ax] = slice(1, shape[ax])
        a, b = kap[tuple(lo)], kap[tuple(hi)]
        face = 2.0 * a * b / (a + b)
        diag[tuple(lo)] += face
        diag[tuple(hi)] += face
        ia, ib = idx[tuple(lo)].ravel(), idx[tuple(hi)].ravel()
        rows += [ia, ib]
        cols += [ib, ia]
        vals += [-face.ravel(), -face.ravel()]
        first = [slice(None)] * d
        last = [slice(None)] * d
        first[ax] = slice(0, 1)
        last[ax] = slice(shape[ax] - 1, shape[ax])
        diag[tuple(first)] += 2.0 * kap[tuple(first)]
        diag[tuple(last)] += 2.0 * kap[tuple(last)]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    import scipy.sparse as sp

    S = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return _from_scipy(S)


def fem27_aniso(N: int, eps: float = 1e-3, chunk_planes: int = 8):
    """Q1-FEM 27-point matrix K(x)M(x)M + M(x)K(x)M + eps M(x)M(x)K on an N^3 interior grid.

    1D factors: K = tridiag(-1, 2, -1), M = tridiag(1, 4, 1) / 6. Entry values depend only on
    the offset (dx, dy, dz); neighbours outside the grid are dropped (Dirichlet). Built plane
    by plane so that peak memory stays near the size of the result."""
    Kc = {-1: -1.0, 0: 2.0, 1: -1.0}
    Mc = {-1: 1.0 / 6.0, 0: 4.0 / 6.0, 1: 1.0 / 6.0}
    offs = [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)]
    coef = np.array([Kc[dx] * Mc[dy] * Mc[dz] + Mc[dx] * Kc[dy] * Mc[dz] + eps * Mc[dx] * Mc[dy] * Kc[dz]
                     for dx, dy, dz in offs])
    n = N ** 3
    # row lengths: product of per-axis neighbour counts (2 at a face of the grid, 3 inside)
    cnt1 = np.full(N, 3, dtype=np.int64)
    cnt1[0] -= 1
    cnt1[-1] -= 1
    rowlen = (cnt1[:, None, None] * cnt1[None, :, None] * cnt1[None, None, :]).ravel()
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(rowlen, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    assert nnz < 2 ** 31
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    jj, kk = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    jj, kk = jj.ravel(), kk.ravel()
    for i0 in range(0, N, chunk_planes):
        i1 = min(N, i0 + chunk_planes)
        ii = np.repeat(np.arange(i0, i1), N * N)
        j = np.tile(jj, i1 - i0)
        k = np.tile(kk, i1 - i0)
        rows = ii * N * N + j * N + k
        C = np.empty((rows.size, 27), dtype=np.int64)
        V = np.empty((rows.size, 27))
        valid = np.empty((rows.size, 27), dtype=bool)
        for t, (dx, dy, dz) in enumerate(offs):
            a, b, c = ii + dx, j + dy, k + dz
            valid[:, t] = (a >= 0) & (a < N) & (b >= 0) & (b < N) & (c >= 0) & (c < N)
            C[:, t] = a * N * N + b * N + c
            V[:, t] = coef[t]
        s, e = int(row_ptr[rows[0]]), int(row_ptr[rows[-1] + 1])
        col[s:e] = C[valid]
        val[s:e] = V[valid]
    return (n, row_ptr.astype(np.int32), col, val)


def fem27_spectrum(N: int, eps: float = 1e-3):
    """Closed-form extreme eigenvalues of fem27_aniso(N, eps): K and M share the sine
    eigenvectors, so lambda = kx my mz + mx ky mz + eps mx my kz over all index triples."""
    th = np.arange(1, N + 1) * math.pi / (N + 1)
    k = 2.0 - 2.0 * np.cos(th)
    m = (4.0 + 2.0 * np.cos(th)) / 6.0
    # each term is monotone in its own index, so evaluate the full grid lazily via extremes
    lam = (k[:, None, None] * m[None, :, None] * m[None, None, :] + m[:, None, None] * k[None, :, None]
           * m[None, None, :] + eps * m[:, None, None] * m[None, :, None] * k[None, None, :]) if N <= 64 else None
    if lam is not None:
        return float(lam.min()), float(lam.max())
    # for large N the extremes sit at the corners of the index cube
    cands = []
    for a in (0, N - 1):
        for b in (0, N - 1):
            for c in (0, N - 1):
                cands.append(k[a] * m[b] * m[c] + m[a] * k[b] * m[c] + eps * m[a] * m[b] * k[c])
    return float(min(cands)), float(max(cands))


def banded_spd(n: int, kd: int, lam_min_target: float, rng: np.random.Generator):
    """Banded SPD matrix A = L L^T + lam_t I with L lower triangular, half-bandwidth kd and
    N(0,1) entries: L L^T is positive semidefinite with a smallest eigenvalue that is tiny for
    a random triangular factor, so lambda_min(A) ~ lam_t (bounded below by lam_t). A has
    half-bandwidth kd; its diagonals are formed one by one:
    (L L^T)[i, i-d] = sum_{m=d..kd} L[i, i-m] L[i-d, i-m]."""
    import scipy.sparse as sp

    kd = max(1, min(kd, n - 1))
    ab = np.zeros((kd + 1, n))  # ab[m, i] = L[i, i - m]
    for m in range(kd + 1):
        ab[m, m:] = rng.standard_normal(n - m)
    diags, offs = [], []
    for d in range(kd + 1):
        acc = np.zeros(n - d)
        for m in range(d, kd + 1):
            # rows i = d..n-1: L[i, i-m] L[i-d, i-m]; L[i-d, i-m] = ab[m-d, i-d]
            acc += ab[m, d:] * ab[m - d, : n - d]
        diags.append(acc + (lam_min_target if d == 0 else 0.0))
        offs.append(-d)
    L = sp.diags(diags, offs, shape=(n, n))
    U = sp.diags(diags[1:], [-o for o in offs[1:]], shape=(n, n))
    return _from_scipy(L + U)


def ba_laplacian(n: int, m: int, shift: float, rng: np.random.Generator, block: int = 4096):
    """Shifted Laplacian L + shift I of a preferential-attachment graph with m edges per new node.

    Targets of a new node are sampled uniformly from the endpoint list of the edges that
    existed at the start of its block of `block` nodes (degree-proportional sampling with a
    short lag), which keeps the power-law degree tail while vectorising the construction."""
    import scipy.sparse as sp

    m0 = m + 1
    src = [np.repeat(np.arange(m0), m0 - 1)]
    dst = [np.array([j for i in range(m0) for j in range(m0) if j != i])]
    ends = np.concatenate([src[0], dst[0]])
    t = m0
    while t < n:
        t1 = min(n, t + block)
        new = np.arange(t, t1)
        picks = ends[rng.integers(0, ends.size, size=(new.size, m))]
        s_ = np.repeat(new, m)
        d_ = picks.ravel()
        src.append(s_)
        dst.append(d_)
        ends = np.concatenate([ends, s_, d_])
        t = t1
    s_all = np.concatenate(src)
    d_all = np.concatenate(dst)
    keep = s_all != d_all
    s_all, d_all = s_all[keep], d_all[keep]
    Wm = sp.coo_matrix((np.ones(s_all.size), (s_all, d_all)), shape=(n, n)).tocsr()
    Wm = ((Wm + Wm.T) > 0).astype(np.float64)
    deg = np.asarray(Wm.sum(axis=1)).ravel()
    Lap = sp.diags(deg + shift) - Wm
    return _from_scipy(Lap)


def hub_laplacian(n: int, hubs: int, deg_lo: int, deg_hi: int, shift: float, rng: np.random.Generator,
                  hub_rows=None):
    """Shifted Laplacian L + shift I of a ring of n nodes plus `hubs` hub nodes, each joined to
    a log-uniform number in [deg_lo, deg_hi] of distinct random nodes: the few very long rows
    of a power-law graph next to many short ones. `hub_rows` places the hubs (default: spread
    evenly over the rows)."""
    import scipy.sparse as sp

    if hub_rows is None:
        hub_rows = np.linspace(0, n - 1, hubs).astype(np.int64)
    hub_rows = np.asarray(hub_rows, dtype=np.int64)
    src = [np.arange(n), ]
    dst = [(np.arange(n) + 1) % n]
    degs = np.exp(rng.uniform(np.log(deg_lo), np.log(deg_hi), hub_rows.size)).astype(np.int64)
    for h, d in zip(hub_rows, degs):
        nb = rng.choice(n, size=int(min(d, n - 1)), replace=False)
        nb = nb[nb != h]
        src.append(np.full(nb.size, h))
        dst.append(nb)
    s_all = np.concatenate(src)
    d_all = np.concatenate(dst)
    Wm = sp.coo_matrix((np.ones(s_all.size), (s_all, d_all)), shape=(n, n)).tocsr()
    Wm = ((Wm + Wm.T) > 0).astype(np.float64)
    deg = np.asarray(Wm.sum(axis=1)).ravel()
    Lap = sp.diags(deg + shift) - Wm
    return _from_scipy(Lap)


def synth_bbt(seed: int, n: int = 5000, pairs: int = 5000, ood: bool = False):
    """Section 5.1's synthetic family: A = B B^T + beta I with B n x n holding `pairs` entries at
    index pairs drawn uniformly with replacement (repeated pairs add up), values N(0, 1), and
    beta ~ U[1e-4, 1e-2]; with ood the pair count is scaled by U[0.8, 1.2] (the paper's
    out-of-distribution test set). READINGS: the paper's "about 1% nonzeros" contradicts its
    5000 pairs in a 5000 x 5000 B (0.02%): the pair count is used; b ~ U[-1, 1] (the paper
    draws b from a uniform distribution without giving its range). Returns (A, b)."""
    import scipy.sparse as sp

    rng = rng_for(51, seed)
    npairs = int(round(pairs * rng.uniform(0.8, 1.2))) if ood else pairs
    i = rng.integers(0, n, npairs)
    j = rng.integers(0, n, npairs)
    v = rng.standard_normal(npairs)
    B = sp.coo_matrix((v, (i, j)), shape=(n, n)).tocsr()
    beta = rng.uniform(1e-4, 1e-2)
    A = (B @ B.T + beta * sp.identity(n, format="csr")).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    b = rng.uniform(-1.0, 1.0, n)
    return _from_scipy(A), b


def _edge_function(rng):
    """A boundary function g(t), t in [0, 1] along an edge: constant, linear or sinusoidal with
    uniform parameters (equal odds)."""
    kind = int(rng.integers(0, 3))
    if kind == 0:
        c = rng.uniform(-1, 1)
        return lambda t: np.full_like(t, c)
    if kind == 1:
        c0, c1 = rng.uniform(-1, 1, 2)
        return lambda t: c0 + c1 * t
    a, k = rng.uniform(-1, 1), rng.uniform(0.5, 3.0)
    return lambda t: a * np.sin(k * np.pi * t)


def _source_function(rng):
    """A source f(x, y): zero, sinusoidal or a low-degree polynomial (equal odds)."""
    kind = int(rng.integers(0, 3))
    if kind == 0:
        return lambda x, y: np.zeros_like(x)
    if kind == 1:
        a, kx, ky = rng.uniform(-10, 10), rng.uniform(0.5, 3.0), rng.uniform(0.5, 3.0)
        return lambda x, y: a * np.sin(kx * np.pi * x) * np.sin(ky * np.pi * y)
    c = rng.uniform(-5, 5, 6)
    return lambda x, y: c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * x * y + c[5] * y * y


def poisson_subdomain_system(ax, bx, ay, by, m, f, g_left, g_right, g_bottom, g_top):
    """Five-point -lap u = f on [ax, bx] x [ay, by] with m x m interior points (h = (b - a) /
    (m + 1) per direction) and Dirichlet data on the four edges (each g a function of the
    edge coordinate t in [0, 1], left/right along y, bottom/top along x) moved into b.
    Unknowns in x-fastest order. Returns (A, b)."""
    import scipy.sparse as sp

    hx, hy = (bx - ax) / (m + 1), (by - ay) / (m + 1)
    T = sp.diags([-np.ones(m - 1), 2 * np.ones(m), -np.ones(m - 1)], [-1, 0, 1])
    Im = sp.identity(m)
    A = (sp.kron(Im, T / hx ** 2) + sp.kron(T / hy ** 2, Im)).tocsr()
    A.sort_indices()
    xs = ax + hx * np.arange(1, m + 1)
    ys = ay + hy * np.arange(1, m + 1)
    X, Y = np.meshgrid(xs, ys)  # X[j, i] = x_i: rows are y, so ravel() is x-fastest
    b = np.asarray(f(X, Y), dtype=np.float64).copy()
    ty = (ys - ay) / (by - ay)
    tx = (xs - ax) / (bx - ax)
    b[:, 0] += g_left(ty) / hx ** 2
    b[:, -1] += g_right(ty) / hx ** 2
    b[0, :] += g_bottom(tx) / hy ** 2
    b[-1, :] += g_top(tx) / hy ** 2
    return _from_scipy(A), b.ravel()


def poisson_subdomain(seed: int, m: int = 80):
    """Section 5.2's family: a random subdomain [ax, bx] x [ay, by] of [0, 2]^2 (ax ~ U[0, 1.9],
    bx = ax + U[0.1, 2 - ax], the same for y), 80 x 80 interior points, Dirichlet data on each
    edge constant, linear or sinusoidal, source zero, sinusoidal or polynomial (equal odds).
    READING: the paper names the function classes, not their parameter ranges; the ranges
    here are the generator's own. Returns (A, b)."""
    rng = rng_for(52, seed)
    ax = rng.uniform(0.0, 1.9)
    bx = ax + rng.uniform(0.1, 2.0 - ax)
    ay = rng.uniform(0.0, 1.9)
    by = ay + rng.uniform(0.1, 2.0 - ay)
    f = _source_function(rng)
    gs = [_edge_function(rng) for _ in range(4)]
    return poisson_subdomain_system(ax, bx, ay, by, m, f, *gs)


def random_spd_small(n: int, rng: np.random.Generator, density: float = 0.3, shift: float = 0.5):
    """Small sparse SPD matrix B B^T + shift I with a random sparse B (the construction of the
    paper's synthetic set, Section 5.1, at test sizes)."""
    import scipy.sparse as sp

    B = sp.random(n, n, density=density, random_state=rng, data_rvs=rng.standard_normal)
    return _from_scipy(B @ B.T + shift * sp.identity(n))


def rhs_from_xstar(A, rng: np.random.Generator):
    """x* ~ U[-1, 1] and b = A x* (fp64)."""
    import scipy.sparse as sp

    n, rp, ci, val = A
    xs = rng.uniform(-1.0, 1.0, n)
    S = sp.csr_matrix((val, ci, rp), shape=(n, n))
    return xs, S @ xs


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

def cfg_poisson32(seed: int = 0):
    """2D 5-point Poisson Laplacian on a 32 x 32 grid, b = A x*, x* ~ U[-1,1] (seed 0)."""
    A = poisson2d(32)
    xs, b = rhs_from_xstar(A, np.random.default_rng(seed))
    return A, b, xs


def cfg_train_set(count: int = 64, m_lo: int = 16, m_hi: int = 40, sig_lo: float = 0.5, sig_hi: float = 3.0,
                  seed: int = 2):
    """Variable-coefficient 3D 7-point diffusion matrices: edge m ~ U{m_lo..m_hi}, log-normal
    coefficients with sigma ~ U[sig_lo, sig_hi]; b = A x*, x* ~ U[-1, 1]."""
    out = []
    for i in range(count):
        rng = rng_for(seed, i)
        mm = int(rng.integers(m_lo, m_hi + 1))
        sig = float(rng.uniform(sig_lo, sig_hi))
        A = diffusion_varcoef((mm, mm, mm), sig, rng)
        xs, b = rhs_from_xstar(A, rng)
        out.append((A, b, xs))
    return out


def cfg_batched(count: int = 512, n_lo: float = 1e3, n_hi: float = 2e5, seed: int = 4):
    """Uneven batch: n log-uniform on [n_lo, n_hi]; types in thirds: 2D 5-point and 3D 7-point
    variable-coefficient diffusion (sigma ~ U[0.5, 3]), and banded SPD matrices L L^T + lam I
    with half-bandwidth kd ~ U{5..64} and lam log-uniform on [1e-6, 1e-2] (lambda_min ~ lam)."""
    out = []
    for i in range(count):
        rng = rng_for(seed, i)
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        kind = i % 3
        if kind == 0:
            e = max(2, int(round(math.sqrt(n))))
            A = diffusion_varcoef((e, e), float(rng.uniform(0.5, 3.0)), rng)
        elif kind == 1:
            e = max(2, int(round(n ** (1.0 / 3.0))))
            A = diffusion_varcoef((e, e, e), float(rng.uniform(0.5, 3.0)), rng)
        else:
            kd = int(rng.integers(5, 65))
            lam = math.exp(rng.uniform(math.log(1e-6), math.log(1e-2)))
            A = banded_spd(n, min(kd, n - 1), lam, rng)
        xs, b = rhs_from_xstar(A, rng)
        out.append((A, b, xs))
    return out
