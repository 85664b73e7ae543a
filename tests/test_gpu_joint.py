"""The joint augmented space V_H + span{psi^_1..psi^_N} on the GPU (mk_joint_ritz, mk_joint_assemble) against the
oracle's Rayleigh-Ritz in the same space (oracle/linalg.joint_ritz): eigenvalues, M-orthonormal coefficient
vectors (up to sign), a correction that lies in V_H (dropped), and the chained step on the GPU."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import linalg as olin
from tests._cases import case, maxrel

pytestmark = pytest.mark.gpu

CASES = ["h_p1", "mol4_p2_small"]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def ctx(torch):
    from paper_2103_02824_gb300 import build, mk
    build.build()
    c = mk.Context(0)
    yield c
    c.close()


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _joint_gpu(torch, ctx, AH, MH, B, C, GA, GM, k):
    from paper_2103_02824_gb300 import mk
    NH, N = B.shape
    d, V = sla.eigh(AH, MH)          # the shared decomposition (the GPU's own is tested elsewhere)
    lam = torch.zeros(k, dtype=torch.float64, device="cuda")
    X = torch.zeros((NH + N, k), dtype=torch.float64, device="cuda")
    kept = mk.mk_joint_ritz(ctx, NH, N, k, dev(torch, d), dev(torch, V), dev(torch, B), dev(torch, C),
                            dev(torch, GA), dev(torch, GM), lam, X)
    torch.cuda.synchronize()
    return lam.cpu().numpy(), X.cpu().numpy(), kept


def _signed(X, Xref):
    s = np.sign(np.sum(X * Xref, axis=0))
    s[s == 0] = 1.0
    return X * s[None, :]


@pytest.mark.parametrize("name", CASES)
def test_joint_ritz_matches_oracle(ctx, torch, name):
    o = case(name)["out"]
    N = o["b"].shape[1]
    for k in sorted({1, N}):
        lo, Xo = olin.joint_ritz(o["AH"], o["MH"], o["b"], o["c"], o["gramA"], o["gramM"], k)
        lg, Xg, kept = _joint_gpu(torch, ctx, o["AH"], o["MH"], o["b"], o["c"], o["gramA"], o["gramM"], k)
        assert kept == N
        assert np.abs(lg - lo).max() < 1e-10 * max(1.0, np.abs(lo).max())
        assert maxrel(_signed(Xg, Xo), Xo) < 1e-8
        Mj = np.block([[o["MH"], o["c"]], [o["c"].T, 0.5 * (o["gramM"] + o["gramM"].T)]])
        assert np.abs(Xg.T @ Mj @ Xg - np.eye(k)).max() < 1e-9


def test_joint_ritz_drops_a_correction_in_the_coarse_space(ctx, torch):
    """Correction 0 replaced by a coarse function P t: its direction is dropped on both sides, the rest agree."""
    o = case("mol4_p2_small")["out"]
    AH, MH = o["AH"], o["MH"]
    N = o["b"].shape[1]
    t = np.random.default_rng(5).standard_normal(AH.shape[0])
    B, Cc, GA, GM = o["b"].copy(), o["c"].copy(), o["gramA"].copy(), o["gramM"].copy()
    B[:, 0], Cc[:, 0] = AH @ t, MH @ t
    GA[0, :] = GA[:, 0] = t @ o["b"]
    GA[0, 0] = t @ AH @ t
    GM[0, :] = GM[:, 0] = t @ o["c"]
    GM[0, 0] = t @ MH @ t
    lo, _ = olin.joint_ritz(AH, MH, B, Cc, GA, GM, N)
    lg, _, kept = _joint_gpu(torch, ctx, AH, MH, B, Cc, GA, GM, N)
    assert kept == N - 1
    assert np.abs(lg - lo).max() < 1e-10 * max(1.0, np.abs(lo).max())


def test_joint_space_after_the_gpu_step(ctx, torch):
    """The step on the GPU (projection and coarse decomposition included), then the joint solve and the joint
    orbitals on the fine mesh, against the oracle's joint Ritz pairs built from the oracle's step."""
    from paper_2103_02824_gb300 import mk
    from paper_2103_02824_gb300.step import CorrectionStep
    c = case("mol4_p2_small")
    o, lv = c["out"], c["level"]
    cc, ct, fc, ft, par = c["meshes"]
    m = mk.Mesh(ctx, fc, ft, cc, ct, par, 2)
    N, NH = c["N"], m.info["n_free_coarse"]
    st = CorrectionStep(ctx, m, c["wl"]["Z"], c["wl"]["R"], N, ld=8)
    st.run(c["psiH"], c["lamH"], c["occ"], c["sigma"], xc=c["xc"], hartree_bc="multipole",
           solve_opts=mk.opts(precision="mixed", rtol=1e-13, check_every=5),
           poisson_opts=mk.opts(precision="mixed", rtol=1e-13, check_every=5, coarse=True))
    lam = torch.zeros(N, dtype=torch.float64, device="cuda")
    X = torch.zeros((NH + N, N), dtype=torch.float64, device="cuda")
    kept = mk.mk_joint_ritz(ctx, NH, N, N, st.d, st.V, st.b, st.c, st.gramA, st.gramM, lam, X)
    psi = torch.zeros_like(st.psi)
    mk.mk_joint_assemble(ctx, m, N, N, X, st.psihat, st.u, psi)
    torch.cuda.synchronize()
    lo, Xo = olin.joint_ritz(o["AH"], o["MH"], o["b"], o["c"], o["gramA"], o["gramM"], N)
    assert kept == N
    assert np.abs(lam.cpu().numpy() - lo).max() < 1e-9
    # every one-orbital space V_H + span{psi^_i} is a subspace of the joint one: its lowest N Ritz values bound the
    # joint ones from above
    for i in range(N):
        A1 = np.block([[o["AH"], o["b"][:, i:i + 1]], [o["b"][:, i:i + 1].T, o["gramA"][i:i + 1, i:i + 1]]])
        M1 = np.block([[o["MH"], o["c"][:, i:i + 1]], [o["c"][:, i:i + 1].T, o["gramM"][i:i + 1, i:i + 1]]])
        assert np.all(lam.cpu().numpy() <= sla.eigh(A1, M1, eigvals_only=True)[:N] + 1e-9)
    fr = lv.fine.free
    ref = np.zeros((lv.fine.n_nodes, N))
    ref[fr] = lv.Pf @ Xo[:NH] + o["psihat"][fr] @ Xo[NH:]
    sgn = np.sign(np.sum(ref[fr] * (lv.Mff @ o["u"][fr]), axis=0))
    ref *= np.where(sgn == 0, 1.0, sgn)[None, :]
    got = psi.cpu().numpy()[:, :N]
    for j in range(N):
        assert maxrel(got[:, j], ref[:, j]) < 1e-6
    m.close()
