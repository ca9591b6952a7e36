"""mpcg_solve_noalloc: the solve for callers that cannot allocate device memory while
they solve (a fixed device-memory budget, a pool that must not grow). Its scratch is a
static device array of the library, so the call itself allocates nothing. Checked through
the C ABI against the regular mpcg_solve on two calls in a row (the array keeps the
previous call's contents, so the second call shows that what must start cleared is
cleared). This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2504_14268_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2504_14268_gb300 import mpcg

    return mpcg


def _dev(A):
    n, rp, ci, val = A
    return (n, torch.as_tensor(rp).cuda(), torch.as_tensor(ci).cuda(), torch.as_tensor(val).cuda())


@pytest.mark.parametrize("fmts", [(4, 4, 4, 4), (0, 0, 3, 3)])
def test_noalloc_solve_matches_regular_solve_twice(M, fmts):
    A, b, xs = I.cfg_poisson32()
    ctx = M.Context(0, M.Options(min_k=0))
    mat = ctx.matrix(_dev(A))
    pol = ctx.policy_fixed(fmts)
    bd = torch.as_tensor(b).cuda()
    x_ref = torch.zeros_like(bd)
    ref, _ = ctx.solve(mat, bd, x_ref, 1e-8, 500, pol)
    for call in range(2):
        x = torch.full_like(bd, 3.0)  # any content: x_0 = 0 is set by the kernel
        res = ctx.solve_noalloc(mat, bd, x, 1e-8, 500, pol)
        assert res["outcome"] == ref["outcome"]
        assert res["iters"] == ref["iters"]
        assert res["rel_res_true"] == pytest.approx(ref["rel_res_true"], rel=1e-6, abs=1e-15)
        err = (x - x_ref).abs().max().item() / x_ref.abs().max().item()
        tol = 1e-12 if fmts == (4, 4, 4, 4) else 5e-3
        assert err <= tol, (call, err)


def test_noalloc_rejects_systems_beyond_its_scratch(M):
    n = (1 << 20) + 1
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    val = np.full(n, 2.0)
    ctx = M.Context(0, M.Options(min_k=0))
    mat = ctx.matrix(_dev((n, rp, ci, val)))
    pol = ctx.policy_fixed((4, 4, 4, 4))
    b = torch.ones(n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(M.MpcgError, match="at most"):
        ctx.solve_noalloc(mat, b, x, 1e-8, 10, pol)
    A, bs, _ = I.cfg_poisson32()
    small = ctx.matrix(_dev(A))
    with pytest.raises(M.MpcgError, match="device pointers"):
        ctx.solve_noalloc(small, torch.as_tensor(bs), torch.zeros(A[0], dtype=torch.float64), 1e-8, 10, pol)


def _compare_twice(M, ctx, A, b, fmts, tol, maxit, rtol_x, sched=None):
    """Regular solve first, then two no-allocation calls; the second must leave the device's
    free memory unchanged (the call allocates nothing) and both must match the regular solve."""
    mat = ctx.matrix(_dev(A))
    if sched is not None:
        for f in set(fmts[:1]) | {4}:  # the product's format and the fp64 residual recomputation
            mat.set_schedule(f, *sched)
    pol = ctx.policy_fixed(fmts)
    bd = torch.as_tensor(b).cuda()
    x_ref = torch.zeros_like(bd)
    ref, _ = ctx.solve(mat, bd, x_ref, tol, maxit, pol)
    xs = [torch.full_like(bd, -1.0) for _ in range(2)]
    torch.cuda.synchronize()
    free = []
    for call in range(2):
        free.append(torch.cuda.mem_get_info()[0])
        res = ctx.solve_noalloc(mat, bd, xs[call], tol, maxit, pol)
        torch.cuda.synchronize()
        assert res["outcome"] == ref["outcome"] and res["iters"] == ref["iters"], (call, res, ref)
        assert res["rel_res_true"] == pytest.approx(ref["rel_res_true"], rel=1e-6, abs=1e-15)
        err = (xs[call] - x_ref).abs().max().item() / x_ref.abs().max().item()
        assert err <= rtol_x, (call, err)
    assert torch.cuda.mem_get_info()[0] == free[1]
    return ref


def test_noalloc_multi_cta_team_and_stream_schedule(M):
    """A 27-point system large enough for a team of many CTAs (barriers and partial sums of
    several CTAs in the shared array), with the regular and the staged stream product."""
    A = I.fem27_aniso(40, 1e-2)
    _, b = I.rhs_from_xstar(A, np.random.default_rng(2))
    ctx = M.Context(0, M.Options(min_k=0))
    ref = _compare_twice(M, ctx, A, b, (4, 4, 4, 4), 1e-8, 2000, 1e-12)
    assert ref["iters"] > 20
    _compare_twice(M, ctx, A, b, (3, 4, 3, 4), 1e-6, 2000, 5e-3, sched=(1, 4))


def test_noalloc_near_the_row_limit(M):
    """n = 101^3 = 1,030,301 rows, within 2^20: the work vectors fill most of the array."""
    A = I.fem27_aniso(101, 1e-2)
    assert A[0] <= 1 << 20 and A[0] > 1 << 19
    _, b = I.rhs_from_xstar(A, np.random.default_rng(3))
    ctx = M.Context(0, M.Options(min_k=0))
    _compare_twice(M, ctx, A, b, (3, 4, 4, 4), 1e-6, 300, 5e-3)


def test_noalloc_jacobi(M):
    """The Jacobi preconditioner (precond = 1) reads its diagonal from the matrix object."""
    rng = np.random.default_rng(4)
    A = I.diffusion_varcoef((14, 12, 10), 1.5, rng)
    _, b = I.rhs_from_xstar(A, rng)
    ctx = M.Context(0, M.Options(min_k=0, precond=1))
    _compare_twice(M, ctx, A, b, (4, 4, 4, 4), 1e-8, 3000, 1e-12)
