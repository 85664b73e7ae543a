"""Failure detection on the device, without a fault: the persistent operator kernel's bounded waits for its own
asynchronous copies (bulk copies and cp.async completing on mbarriers) are made to give up (wait limit 0 through mk_ctx_set_option), the library reports it (the
context's fault word, MK_ERR_TIMEOUT from a solve), the kernel still waits for every copy it issued before it
ends, and the same context then applies the operator and solves correctly again."""
import numpy as np
import pytest

from tests._cases import case, maxrel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def test_wait_that_gives_up_is_reported_and_the_context_recovers(torch):
    from paper_2103_02824_gb300 import build, mk
    build.build()
    c = case("mol4_p2_small")
    lv = c["level"]
    ctx = mk.Context(0)
    cc, ct, fc, ft, par = c["meshes"]
    m = mk.Mesh(ctx, fc, ft, cc, ct, par, c["wl"]["order"])
    mol = mk.Molecule(c["wl"]["Z"], c["wl"]["R"])
    n, N, ld, sigma = m.info["n_nodes"], c["N"], 8, c["sigma"]
    X = np.random.default_rng(2).standard_normal((n, ld))
    X[lv.fine.boundary] = 0.0
    ref = np.zeros((n, ld))
    ref[lv.fine.free] = lv.operator(sigma) @ X[lv.fine.free]
    x = torch.from_numpy(X).float().cuda()
    rhs = np.zeros((n, ld))
    rhs[:, :N] = c["out"]["rhs"]
    u = np.zeros((n, ld))
    u[:, :N] = c["out"]["u"]
    rhs_d = torch.from_numpy(rhs).cuda()
    try:
        assert mk.ctx_fault(ctx) == 0
        # the FP32 operator on the persistent two-group kernel, the one whose copies complete on mbarriers
        mk.ctx_set_option(ctx, mk.MK_OPT_PATCH_PIPELINE, 2)
        mk.ctx_set_option(ctx, mk.MK_OPT_WAIT_LIMIT, 0)
        mk.mk_operator_apply(ctx, m, mol, sigma, x, torch.full_like(x, 3.0))
        assert mk.ctx_fault(ctx) & mk.MK_FAULT_PATCH_WAIT      # read and cleared
        # a mixed solve whose inner operator gives up returns MK_ERR_TIMEOUT
        xs = torch.from_numpy(u).cuda()
        rep = mk.mk_correction_solve(ctx, m, mol, sigma, rhs_d, xs, N,
                                     opt=mk.opts(precision="mixed", rtol=1e-12, maxit=10, check_every=5),
                                     allow=(mk.MK_ERR_TIMEOUT,))
        assert rep["code"] == mk.MK_ERR_TIMEOUT
        assert mk.ctx_fault(ctx) & mk.MK_FAULT_PATCH_WAIT
    finally:
        mk.ctx_set_option(ctx, mk.MK_OPT_WAIT_LIMIT, -1)
        mk.ctx_set_option(ctx, mk.MK_OPT_PATCH_PIPELINE, 1)
    # the same context after the failure: the operator and a full mixed-precision solve are right again
    y = torch.full_like(x, 3.0)
    mk.mk_operator_apply(ctx, m, mol, sigma, x, y)
    torch.cuda.synchronize()
    assert maxrel(y.double().cpu().numpy(), ref) < 3e-6
    xs = torch.from_numpy(u).cuda()
    rep = mk.mk_correction_solve(ctx, m, mol, sigma, rhs_d, xs, N,
                                 opt=mk.opts(precision="mixed", rtol=1e-12, inner_rtol=1e-4, check_every=5))
    assert rep["max_rel_residual"] <= 1e-12
    assert maxrel(xs.cpu().numpy()[:, :N], c["out"]["psihat"]) < 1e-8
    assert mk.ctx_fault(ctx) == 0
    with pytest.raises(mk.MkError):
        mk.ctx_set_option(ctx, mk.MK_OPT_WAIT_LIMIT, -2)
    m.close()
    ctx.close()
