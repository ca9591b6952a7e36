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
