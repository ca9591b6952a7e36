"""GPU parity of the Jacobi-preconditioned variant (op 2 with M = diag(A): z = fl_p2(r_i d_i),
d_i = 1 / a_ii in fp64) against the oracle: residual histories within 1e-6 for all-fp64
iterations and 5e-3 otherwise, final error within 10x the oracle's, batched (lockstep)
solves per system, bit-identity with plain CG when the diagonal is a power of two, and the
refusal (at matrix creation) of a row lacking a positive diagonal entry."""
import numpy as np
import pytest

import oracle as O
from paper_2504_14268_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALL64 = (4, 4, 4, 4)


@pytest.fixture(scope="module")
def M():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2504_14268_gb300 import mpcg

    return mpcg


def _dev(A):
    n, rp, ci, val = A
    return (n, torch.as_tensor(rp).cuda(), torch.as_tensor(ci).cuda(), torch.as_tensor(val).cuda())


def _system(seed=3, shape=(12, 11, 10), sigma=2.0):
    rng = np.random.default_rng(seed)
    A = I.diffusion_varcoef(shape, sigma, rng)
    xs, b = I.rhs_from_xstar(A, rng)
    return A, b, xs


@pytest.mark.parametrize("fmts,tol", [(ALL64, 1e-10), ((3, 3, 3, 3), 1e-6), ((0, 0, 3, 3), 1e-3),
                                      ((1, 4, 4, 4), 1e-3), ((3, 0, 4, 3), 1e-4)])
def test_jacobi_fixed_policy_history_matches_oracle(M, fmts, tol):
    A, b, xs = _system()
    ctx = M.Context(0, M.Options(min_k=0, precond=1))
    mat = ctx.matrix(_dev(A))
    bd = torch.as_tensor(b).cuda()
    x = torch.zeros_like(bd)
    res, hist = ctx.solve(mat, bd, x, tol, 2000, ctx.policy_fixed(fmts), history_cap=2000)
    ref = O.solve(O.Options(min_k=0, precond=1), A, b, tol, 2000, fixed=fmts)
    assert res["outcome"] == ref.outcome == O.CONVERGED
    n = min(res["iters"], ref.iters, 40 if fmts != ALL64 else 10 ** 6)
    err = np.abs(hist["rho"][:n] - ref.hist["rho"][:n]) / np.abs(ref.hist["rho"][:n])
    assert np.all(err <= (1e-6 if fmts == ALL64 else 5e-3)), (fmts, float(err.max()), int(np.argmax(err)))
    assert abs(res["iters"] - ref.iters) <= max(2, ref.iters // 20)
    eg = np.linalg.norm(x.cpu().numpy() - xs)
    eo = np.linalg.norm(ref.x - xs)
    assert eg <= 10 * eo + 1e-14


def test_jacobi_cuts_iterations_and_matches_plain_cg_where_it_must(M):
    A, b, xs = _system(seed=4, shape=(12, 12, 12), sigma=2.0)
    bd = torch.as_tensor(b).cuda()
    its = {}
    for pc in (0, 1):
        ctx = M.Context(0, M.Options(precond=pc))
        mat = ctx.matrix(_dev(A))
        x = torch.zeros_like(bd)
        res, _ = ctx.solve(mat, bd, x, 1e-8, 20000, ctx.policy_fixed(ALL64))
        assert res["outcome"] == 0
        its[pc] = res["iters"]
    assert its[1] < 0.7 * its[0]
    # power-of-two diagonal (2D Poisson, 4 on the diagonal): identical iterates bit for bit
    P, pb, _ = I.cfg_poisson32()
    pbd = torch.as_tensor(pb).cuda()
    xs2 = []
    for pc in (0, 1):
        ctx = M.Context(0, M.Options(precond=pc))
        mat = ctx.matrix(_dev(P))
        x = torch.zeros_like(pbd)
        ctx.solve(mat, pbd, x, 1e-10, 500, ctx.policy_fixed(ALL64))
        xs2.append(x.cpu().numpy())
    assert np.array_equal(xs2[0], xs2[1])


def test_jacobi_batched_lockstep_matches_oracle_per_system(M):
    sets = I.cfg_train_set(count=6, m_lo=6, m_hi=12)
    ctx = M.Context(0, M.Options(min_k=0, precond=1))
    mats = [ctx.matrix(_dev(A)) for A, _, _ in sets]
    bs = [torch.as_tensor(b).cuda() for _, b, _ in sets]
    xs = [torch.zeros_like(b) for b in bs]
    res = ctx.solve_batched(mats, bs, xs, [1e-8] * 6, [3000] * 6, ctx.policy_fixed((3, 4, 4, 4)))
    for (A, b, xstar), r, x in zip(sets, res, xs):
        ref = O.solve(O.Options(min_k=0, precond=1), A, b, 1e-8, 3000, fixed=(3, 4, 4, 4))
        assert r["outcome"] == ref.outcome
        assert abs(r["iters"] - ref.iters) <= max(2, ref.iters // 20)
        eg = np.linalg.norm(x.cpu().numpy() - xstar)
        eo = np.linalg.norm(ref.x - xstar)
        assert eg <= 10 * eo + 1e-12


def test_jacobi_is_defined_for_every_accepted_matrix(M):
    """Matrix creation already refuses a row without a positive diagonal entry (the CSR
    validation), so every matrix a Jacobi solve can receive has M = diag(A) invertible."""
    n = 4
    rp = np.array([0, 2, 4, 6, 8], dtype=np.int32)
    ci = np.array([0, 1, 0, 1, 2, 3, 2, 3], dtype=np.int32)
    val = np.array([2.0, 1.0, 1.0, 2.0, -1.0, 0.5, 0.5, 3.0])  # row 2 has a negative diagonal
    ctx = M.Context(0, M.Options(precond=1))
    with pytest.raises(M.MpcgError, match="diagonal"):
        ctx.matrix(_dev((n, rp, ci, val)))
