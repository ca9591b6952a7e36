"""GPU parity of the fp32 incomplete Cholesky preconditioner (precond = 2, IC(0): the SPD
reading of Section 5's fixed-precision fp32 incomplete factorization) against the oracle:
the factor bit for bit, the refusals, and preconditioned solves through the persistent
kernel, the per-system teams and the lockstep batch kernel (histories within the parity
tolerances, iteration counts, error to x*)."""
import numpy as np
import pytest

import oracle as O
from paper_2504_14268_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALL64 = (4, 4, 4, 4)
TOL64, TOL_LOW = 1e-6, 5e-3


@pytest.fixture(scope="module")
def M():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2504_14268_gb300 import mpcg

    return mpcg


def _dev(A):
    n, rp, ci, val = A
    return (n, torch.as_tensor(rp).cuda(), torch.as_tensor(ci).cuda(), torch.as_tensor(val).cuda())


def _cases():
    rng = np.random.default_rng(1)
    return {
        "poisson40": I.poisson2d(40),
        "diffusion": I.diffusion_varcoef((11, 13, 9), 1.5, rng),
        "fem12": I.fem27_aniso(12),
        "banded": I.banded_spd(1500, 40, 1e-3, rng),
        "hubs": I.hub_laplacian(20000, 12, 1100, 8000, 1.0, np.random.default_rng(6)),
    }


@pytest.mark.parametrize("name", ["poisson40", "diffusion", "fem12", "banded", "hubs"])
def test_factor_is_bit_exact(M, name):
    A = _cases()[name]
    ctx = M.Context(0, M.Options(min_k=0))
    mat = ctx.matrix(_dev(A))
    out = torch.full((len(A[2]),), float("nan"), dtype=torch.float32, device="cuda")
    mat.ic0(out)
    got = out.cpu().numpy()
    ref = O.ic0(A)
    bad = np.flatnonzero(got.view(np.uint32) != ref.view(np.uint32))
    assert bad.size == 0, (name, bad[:5], got[bad[:5]], ref[bad[:5]])
    mat.ic0(None)  # kept with the matrix: a second call is a no-op


def test_refusals(M):
    ctx = M.Context(0, M.Options(min_k=0, precond=2))
    # Kershaw's SPD matrix: IC(0) meets a negative pivot
    K = np.array([[3.0, -2, 0, 2], [-2, 3, -2, 0], [0, -2, 3, -2], [2, 0, -2, 3]])
    rp = np.array([0, 3, 6, 9, 12], dtype=np.int32)
    ci = np.array([0, 1, 3, 0, 1, 2, 1, 2, 3, 0, 2, 3], dtype=np.int32)
    val = np.array([K[i, j] for i in range(4) for j in ci[rp[i]:rp[i + 1]]])
    mat = ctx.matrix(_dev((4, rp, ci, val)))
    with pytest.raises(M.MpcgError, match="breaks down"):
        mat.ic0()
    b = torch.ones(4, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(M.MpcgError, match="breaks down"):
        ctx.solve(mat, b, x, 1e-8, 10, ctx.policy_fixed(ALL64))
    # an unsymmetric pattern: (1, 0) stored without (0, 1)
    n, rp2, ci2, val2 = I.poisson2d(3)
    keep = np.ones(len(ci2), dtype=bool)
    keep[1] = False  # row 0's entry in column 1
    rp3 = np.concatenate([[0], np.cumsum([np.count_nonzero(keep[rp2[i]:rp2[i + 1]]) for i in range(n)])]).astype(np.int32)
    mat2 = ctx.matrix(_dev((n, rp3, ci2[keep], val2[keep])))
    with pytest.raises(M.MpcgError, match="symmetric"):
        mat2.ic0()
    # the no-allocation solve does not run IC(0)
    A = I.poisson2d(8)
    mat3 = ctx.matrix(_dev(A))
    b3 = torch.ones(A[0], dtype=torch.float64, device="cuda")
    with pytest.raises(M.MpcgError, match="no-allocation"):
        ctx.solve_noalloc(mat3, b3, torch.zeros_like(b3), 1e-8, 10, ctx.policy_fixed(ALL64))


def _hist_err(hg, ho, n):
    rg, ro = hg["rho"][:n], ho["rho"][:n]
    return np.abs(rg - ro) / np.maximum(np.abs(ro), 1e-300)


@pytest.mark.parametrize("name", ["poisson40", "diffusion", "fem12"])
@pytest.mark.parametrize("fmts,tol", [(ALL64, 1e-10), ((3, 3, 3, 4), 1e-6), ((3, 1, 3, 3), 1e-5), ((0, 3, 3, 4), 1e-3)])
def test_preconditioned_solve_matches_oracle(M, name, fmts, tol):
    A = _cases()[name]
    xs, b = I.rhs_from_xstar(A, np.random.default_rng(7))
    ctx = M.Context(0, M.Options(min_k=0, precond=2))
    mat = ctx.matrix(_dev(A))
    bd = torch.as_tensor(b).cuda()
    x = torch.zeros_like(bd)
    res, hist = ctx.solve(mat, bd, x, tol, 1000, ctx.policy_fixed(fmts), history_cap=1000)
    ref = O.solve(O.Options(min_k=0, precond=2), A, b, tol, 1000, fixed=fmts)
    assert res["outcome"] == ref.outcome == O.CONVERGED
    assert abs(res["iters"] - ref.iters) <= max(1, ref.iters // 20)
    n = min(res["iters"], ref.iters)
    err = _hist_err(hist, ref.hist, n)
    assert np.all(err <= (TOL64 if fmts == ALL64 else TOL_LOW)), (float(err.max()), int(np.argmax(err)))
    eg = np.linalg.norm(x.cpu().numpy() - xs) / np.linalg.norm(xs)
    eo = np.linalg.norm(ref.x - xs) / np.linalg.norm(xs)
    assert eg <= 10 * eo + 1e-15
    plain = O.solve(O.Options(min_k=0), A, b, tol, 3000, fixed=fmts)
    assert res["iters"] < plain.iters


def test_residual_replacement_and_restart_with_ic0(M):
    """The true-residual check at claimed convergence and the restart direction p = M^-1 r
    run the substitutions inside the check and restart phases."""
    A, b, xs = I.cfg_poisson32()
    sched = [(0, 0, 3, 3)] * 8 + [(3, 3, 3, 3)] * 8 + [ALL64] * 200
    ctx = M.Context(0, M.Options(min_k=0, precond=2, true_res_at_conv=1))
    mat = ctx.matrix(_dev(A))
    bd = torch.as_tensor(b).cuda()
    x = torch.zeros_like(bd)
    res, hist = ctx.solve(mat, bd, x, 1e-9, 200, ctx.policy_schedule(sched), history_cap=200)
    ref = O.solve(O.Options(min_k=0, precond=2, true_res_at_conv=1), A, b, 1e-9, 200, sched=sched)
    assert res["outcome"] == ref.outcome == O.CONVERGED
    assert res["rel_res_true"] < 1e-9
    assert abs(res["iters"] - ref.iters) <= 2
    n = min(res["iters"], ref.iters, 8)
    assert np.all(_hist_err(hist, ref.hist, n) <= TOL_LOW)


@pytest.mark.parametrize("batch_mode", [1, 2])
@pytest.mark.parametrize("fmts", [ALL64, (3, 3, 3, 4)])
def test_batched_ic0_matches_oracle(M, batch_mode, fmts):
    """Six diffusion systems and a hub graph in one launch: per-system teams (1) and the
    lockstep kernel (2)."""
    sets = I.cfg_train_set(count=6, m_lo=8, m_hi=14)
    A = I.hub_laplacian(8000, 6, 1100, 5000, 1.0, np.random.default_rng(20))
    xs, b = I.rhs_from_xstar(A, np.random.default_rng(30))
    sets.append((A, b, xs))
    ctx = M.Context(0, M.Options(min_k=0, precond=2, batch_mode=batch_mode))
    mats = [ctx.matrix(_dev(A)) for A, _, _ in sets]
    bs = [torch.as_tensor(b).cuda() for _, b, _ in sets]
    xg = [torch.zeros_like(b) for b in bs]
    tol = 1e-10 if fmts == ALL64 else 1e-6
    res = ctx.solve_batched(mats, bs, xg, [tol] * len(sets), [1000] * len(sets), ctx.policy_fixed(fmts))
    for (A, b, xs), r, x in zip(sets, res, xg):
        ref = O.solve(O.Options(min_k=0, precond=2), A, b, tol, 1000, fixed=fmts)
        assert r["outcome"] == ref.outcome == O.CONVERGED
        assert abs(r["iters"] - ref.iters) <= max(2, ref.iters // 20)
        eg = np.linalg.norm(x.cpu().numpy() - xs)
        eo = np.linalg.norm(ref.x - xs)
        assert eg <= 10 * eo + 1e-12
