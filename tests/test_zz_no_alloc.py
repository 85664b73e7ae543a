"""mk_small_eigensolve_static, the variant of the per-orbital small eigensolve for callers that must not allocate
device memory (its workspace is a fixed array inside the library), gives the same eigenpairs as
mk_small_eigensolve_shared, on two calls in a row.  Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest
import scipy.linalg as sla

from tests._cases import case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def test_static_matches_shared_twice(torch):
    from paper_2103_02824_gb300 import build, mk
    build.build()
    o = case("mol4_p2_small")["out"]
    N, NH = o["b"].shape[1], o["AH"].shape[0]
    assert NH <= 512 and N <= 16
    dvals, V = sla.eigh(o["AH"], o["MH"])          # shared decomposition as input (same for both entry points)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    d_d, d_V = dev(dvals), dev(V)
    ins = [dev(o[k]) for k in ("b", "c", "beta", "gamma")]
    ctx = mk.Context(0)
    ref_lam = torch.zeros(N, dtype=torch.float64, device="cuda")
    ref_coef = torch.zeros((NH + 1, N), dtype=torch.float64, device="cuda")
    ref_st = torch.zeros(N, dtype=torch.int32, device="cuda")
    mk.mk_small_eigensolve_shared(ctx, NH, N, d_d, d_V, *ins, ref_lam, ref_coef, ref_st)
    torch.cuda.synchronize()
    for call in range(2):
        lam = torch.full((N,), 123.0, dtype=torch.float64, device="cuda")
        coef = torch.full((NH + 1, N), -5.0, dtype=torch.float64, device="cuda")
        st = torch.full((N,), 99, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        code = mk.mk_small_eigensolve_static(NH, N, d_d, d_V, *ins, lam, coef, st)
        torch.cuda.synchronize()
        assert code == mk.MK_OK, call
        if call == 1:   # after the first call's one-time set-up: the call takes no device memory at all
            assert torch.cuda.mem_get_info()[0] == free0
        assert torch.equal(st, ref_st)
        assert np.abs(lam.cpu().numpy() - ref_lam.cpu().numpy()).max() < 1e-10
        assert np.abs(coef.cpu().numpy() - ref_coef.cpu().numpy()).max() < 1e-8 * np.abs(ref_coef.cpu().numpy()).max()
    # and both match the oracle's dense solve
    assert np.abs(lam.cpu().numpy() - o["lam"]).max() < 1e-10
    ctx.close()


def test_static_rejects_sizes_beyond_its_maximum(torch):
    from paper_2103_02824_gb300 import mk
    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = torch.zeros(8, dtype=torch.int32, device="cuda")
    assert mk.mk_small_eigensolve_static(513, 1, z, z, z, z, z, z, z, z, st) == mk.MK_ERR_INVALID_ARG
    assert "exceeds the fixed maximum" in mk._err()
    assert mk.mk_small_eigensolve_static(10, 17, z, z, z, z, z, z, z, z, st) == mk.MK_ERR_INVALID_ARG
