"""GPU parity on matrices with rows longer than 1024 nonzeros (power-law hubs), which the
vector and vector-load product schedules sum with a whole CTA (a strided pass, a warp
butterfly and a cross-warp merge of the compensated partials): op 1 of Section 4.2 in every
value format and schedule against the oracle, the case where a CTA meets more long rows
than its queue holds, and CG solves (single and batched) on a hub graph."""
import numpy as np
import pytest

import oracle as O
from paper_2504_14268_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCHEDULES = [(0, 1), (0, 2), (0, 4), (0, 32), (2, 1), (1, 1), (1, 4), (3, 1), (4, 1)]


@pytest.fixture(scope="module")
def M():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2504_14268_gb300 import mpcg

    return mpcg


def _dev(A):
    n, rp, ci, val = A
    return (n, torch.as_tensor(rp).cuda(), torch.as_tensor(ci).cuda(), torch.as_tensor(val).cuda())


def _check_products(M, A, fmts, schedules, seed):
    n, rp, ci, val = A
    rng = np.random.default_rng(seed)
    ctx = M.Context(0, M.Options(min_k=0))
    mat = ctx.matrix(_dev(A))
    x = rng.uniform(-1, 1, n)
    xd = torch.as_tensor(x).cuda()
    yd = torch.empty_like(xd)
    absA = (n, rp, ci, np.abs(val))
    lens = np.diff(rp)
    tried = 0
    for fmt in fmts:
        ref = O.spmv(A, fmt, x)
        mag = O.spmv(absA, 4, np.abs(O.chop(x, fmt if fmt < 5 or fmt == 7 else (0 if fmt == 6 else 1))))
        for sched, lanes in schedules:
            try:
                mat.set_schedule(fmt, sched, lanes)
            except M.MpcgError:
                assert sched == 1  # a hub row's tile does not fit a stream stage
                continue
            tried += 1
            ctx.spmv(mat, fmt, xd, yd)
            y = yd.cpu().numpy()
            if fmt == 4:
                assert np.all(np.abs(y - ref) <= 1e-14 * mag + 1e-300), (fmt, sched, lanes)
            elif fmt == 3:
                # fp32 accumulation: one unit of the output plus the recursive-summation bound
                # for the row's length
                bound = np.abs(ref) * 2.0 ** -23 + (lens + 64) * 2.0 ** -24 * mag * 2
                assert np.all(np.abs(y - ref) <= bound), (fmt, sched, lanes, np.max(np.abs(y - ref) - bound))
            else:
                # 16-bit, tf32 and q52 formats: the correctly rounded row sum
                bad = np.flatnonzero(y != ref)
                assert bad.size == 0, (fmt, sched, lanes, bad[:5], lens[bad[:5]])
    mat.close()
    return tried


def test_hub_rows_every_format_and_schedule(M):
    A = I.hub_laplacian(60000, 24, 1100, 20000, 1.0, np.random.default_rng(2))
    assert np.diff(A[1]).max() > 10000
    assert _check_products(M, A, range(8), SCHEDULES, seed=3) >= 8 * 7


def test_merge_path_splits_rows_at_every_kind_of_boundary(M):
    """The merge-path schedule on rows of mixed lengths (the diagonal alone, a few entries,
    rows of a few dozen to a few thousand entries, in runs, so that shares of the merged list
    begin and end inside rows and exactly at row ends), every format, against the oracle: bit
    for bit where the row sum is correctly rounded."""
    rng = np.random.default_rng(7)
    n = 6000
    lens = rng.choice([0, 1, 2, 5, 27, 33, 257, 3000], size=n, p=[.3, .15, .1, .15, .15, .1, .04, .01])
    rows, vals = [], []
    for i, k in enumerate(lens):
        others = rng.choice(n - 1, size=int(k), replace=False)
        cols = np.sort(np.concatenate([[i], others + (others >= i)]))  # the diagonal and k others
        v = rng.uniform(-2, 2, cols.size)
        v[cols == i] = 4.0 + k  # the library takes matrices with a positive diagonal
        rows.append(cols)
        vals.append(v)
    rp = np.concatenate([[0], np.cumsum([r.size for r in rows])]).astype(np.int32)
    ci = np.concatenate(rows).astype(np.int32)
    val = np.concatenate(vals)
    A = (n, rp, ci, val)
    assert _check_products(M, A, range(8), [(3, 1), (4, 1)], seed=8) == 16


def test_long_row_queue_overflow(M):
    """A periodic band of 1031 nonzeros per row on 40000 rows: every CTA's range holds more
    long rows than its queue (32), so rows are summed both by the CTA and in place."""
    n, kd = 40000, 515
    rng = np.random.default_rng(4)
    offs = np.arange(-kd, kd + 1)
    cols = (np.arange(n)[:, None] + offs[None, :]) % n
    order = np.argsort(cols, axis=1)
    cols = np.take_along_axis(cols, order, axis=1)
    vals = rng.uniform(-1, 1, cols.shape)
    vals[cols == np.arange(n)[:, None]] = 2.0 * kd + 2.0
    rp = np.arange(0, n * (2 * kd + 1) + 1, 2 * kd + 1, dtype=np.int32)
    A = (n, rp, cols.ravel().astype(np.int32), vals.ravel())
    assert _check_products(M, A, (0, 2, 3, 4), [(0, 1), (0, 32), (2, 1), (3, 1)], seed=5) == 16


def _stable_prefix(ref, twin, lim):
    """Iterations over which the oracle's history agrees with that of its own twin run on a
    perturbed right-hand side (within lim / 10): CG on a graph with hubs amplifies rounding
    differences by orders of magnitude within a few dozen iterations (the large isolated
    eigenvalues of the hubs), so histories are only comparable over that prefix."""
    k = min(ref.iters, twin.iters)
    e = np.abs(ref.hist["rho"][:k] - twin.hist["rho"][:k]) / np.abs(ref.hist["rho"][:k])
    return int(np.argmax(e > lim / 10)) if np.any(e > lim / 10) else k


@pytest.mark.parametrize("fmts,tol", [((4, 4, 4, 4), 1e-10), ((3, 3, 3, 4), 1e-6), ((1, 3, 3, 4), 1e-4), ((6, 3, 3, 4), 1e-4)])
@pytest.mark.parametrize("sched", [(2, 1), (0, 32), (3, 1)])
def test_solve_on_hub_graph_matches_oracle(M, fmts, tol, sched):
    A = I.hub_laplacian(20000, 12, 1100, 8000, 1.0, np.random.default_rng(6))
    xs, b = I.rhs_from_xstar(A, np.random.default_rng(7))
    ctx = M.Context(0, M.Options(min_k=0))
    mat = ctx.matrix(_dev(A))
    for f in range(8):
        mat.set_schedule(f, *sched)
    bd = torch.as_tensor(b).cuda()
    x = torch.zeros_like(bd)
    maxit = 2000
    res, hist = ctx.solve(mat, bd, x, tol, maxit, ctx.policy_fixed(fmts), history_cap=maxit)
    ref = O.solve(O.Options(min_k=0), A, b, tol, maxit, fixed=fmts)
    # the twin's perturbation is of the size of the rounding differences between the two
    # sides: fp64 sums in another order, or one unit of an fp32 product
    eps = 1e-6 if fmts[0] == 3 else 1e-13
    b2 = b * (1 + eps * np.random.default_rng(8).standard_normal(b.size))
    twin = O.solve(O.Options(min_k=0), A, b2, tol, maxit, fixed=fmts)
    assert res["outcome"] == ref.outcome == O.CONVERGED
    assert abs(res["iters"] - ref.iters) <= max(2, ref.iters // 10)
    lim = 1e-6 if fmts == (4, 4, 4, 4) else 5e-3
    k = _stable_prefix(ref, twin, lim)
    assert k >= 8
    err = np.abs(hist["rho"][:k] - ref.hist["rho"][:k]) / np.abs(ref.hist["rho"][:k])
    assert np.all(err <= lim), (k, float(err.max()))
    eg = np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs)
    eo = np.linalg.norm(ref.x - xs) / np.linalg.norm(xs)
    assert eg <= 10 * eo + 1e-15


def test_batched_solve_on_hub_graphs(M):
    """The lockstep batch kernel on three hub graphs: each system as the oracle's."""
    sets = []
    for s in range(3):
        A = I.hub_laplacian(8000 + 3000 * s, 6, 1100, 5000, 1.0, np.random.default_rng(20 + s))
        xs, b = I.rhs_from_xstar(A, np.random.default_rng(30 + s))
        sets.append((A, b, xs))
    ctx = M.Context(0, M.Options(min_k=0, batch_mode=2))
    mats = [ctx.matrix(_dev(A)) for A, _, _ in sets]
    bs = [torch.as_tensor(b).cuda() for _, b, _ in sets]
    xg = [torch.zeros_like(b) for b in bs]
    fm = (4, 4, 4, 4)
    res = ctx.solve_batched(mats, bs, xg, [1e-10] * 3, [2000] * 3, ctx.policy_fixed(fm))
    for (A, b, xs), r, x in zip(sets, res, xg):
        ref = O.solve(O.Options(min_k=0), A, b, 1e-10, 2000, fixed=fm)
        assert r["outcome"] == ref.outcome == O.CONVERGED
        assert abs(r["iters"] - ref.iters) <= 2
        eg = np.linalg.norm(x.cpu().numpy() - xs)
        eo = np.linalg.norm(ref.x - xs)
        assert eg <= 10 * eo + 1e-12
