"""The outer AFEM loop's Estimate and Mark steps on the GPU (mk_error_indicators, mk_dorfler_mark) against the
oracle (oracle/afem.py): the indicator element by element on the oracle's corrected orbitals of a P1, a P2 and a
graded P2 workload, the closed forms of the oracle's pins (a global quadratic, the kink of |x| across a mesh
plane), and Dorfler's set (the unique part equal; elements tied with the cut marked)."""
import numpy as np
import pytest

from oracle import afem
from oracle.fem import FEMesh
from tests._cases import case, maxrel

pytestmark = pytest.mark.gpu


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


def _pad(a, ld):
    a = a.reshape(a.shape[0], -1)
    out = np.zeros((a.shape[0], ld))
    out[:, :a.shape[1]] = a
    return out


def _gpu_eta2(torch, ctx, mesh, mol, psi, lam, vq):
    from paper_2103_02824_gb300 import mk
    N = len(lam)
    ld = max(4, (N + 3) // 4 * 4)
    eta2 = torch.zeros(mesh.info["n_elems"], dtype=torch.float64, device="cuda")
    mk.mk_error_indicators(ctx, mesh, mol, dev(torch, _pad(psi, ld)), N, lam, dev(torch, vq), eta2)
    torch.cuda.synchronize()
    return eta2


@pytest.mark.parametrize("name", ["h_p1", "mol4_p2_small", "cluster12_p2_small"])
def test_indicators_match_oracle(ctx, torch, name):
    """The step's corrected orbitals and eigenvalues, the Hartree potential of their density (oracle), V_xc of
    that density: the GPU indicator against the oracle's, element by element, and the marked sets."""
    from oracle.poisson import density_at_quad, hartree
    from paper_2103_02824_gb300 import mk
    c = case(name)
    lv, o, wl = c["level"], c["out"], c["wl"]
    psi, lam, occ = o["psi"], o["lam"], c["occ"]
    w, _ = hartree(lv.fine, density_at_quad(lv.fine, psi, occ), bc="multipole", tol=1e-13, K=lv.K)
    ref = afem.indicators(lv.fine, psi, lam, afem.ks_potential(lv, psi, occ, w, wl["xc"]))
    cc, ct, fc, ft, par = c["meshes"]
    mesh = mk.Mesh(ctx, fc, ft, cc, ct, par, wl["order"])
    mol = mk.Molecule(wl["Z"], wl["R"])
    info = mesh.info
    N = len(lam)
    ld = max(4, (N + 3) // 4 * 4)
    vq = torch.zeros((info["n_elems"], info["n_quad"]), dtype=torch.float64, device="cuda")
    mk.mk_frozen_potential(ctx, mesh, dev(torch, _pad(psi, ld)), occ, N, dev(torch, w), wl["xc"], vq)
    eta2 = _gpu_eta2(torch, ctx, mesh, mol, psi, lam, vq.cpu().numpy())
    g = eta2.cpu().numpy()
    err = maxrel(g, ref)
    print(f"\n{name}: indicator max rel err {err:.2e}, total {g.sum():.6e}")
    assert err < 1e-10, err
    # Dorfler, theta = 0.4 (the paper's experiments): the oracle's smallest set; the GPU's adds only cut ties
    marked = torch.zeros(info["n_elems"], dtype=torch.uint8, device="cuda")
    nm, t = mk.mk_dorfler_mark(ctx, eta2, 0.4, marked)
    gm = marked.cpu().numpy().astype(bool)
    om = afem.dorfler(g, 0.4)
    assert nm == gm.sum()
    assert np.all(gm[om]) and np.all(g[gm & ~om] == t)
    assert g[gm].sum() >= 0.4 * g.sum() and t == g[om].min()
    mesh.close()


def test_closed_forms_on_the_gpu(ctx, torch):
    """The oracle's pins through the GPU: a global quadratic (eta^2 = 9 h_T^2 |T|, no jumps) and u = |x| (only the
    faces in the plane x = 0 contribute, h_e |e| each, per orbital squared scale)."""
    from paper_2103_02824_gb300 import mk, synth
    for order in (1, 2):
        cm, tm = synth.cube_mesh(4, 1.0)
        f = FEMesh(cm, tm, order)
        mesh = mk.Mesh(ctx, cm, tm, cm, tm, np.arange(tm.shape[0], dtype=np.int32), order)
        mol = mk.Molecule(np.zeros(0), np.zeros((0, 3)))
        x = f.nodes
        cases = [(np.stack([np.abs(x[:, 0]), 2 * np.abs(x[:, 0])], axis=1), [-0.3, -0.3], -0.3)]
        if order == 2:
            cases.append((x[:, 0] ** 2 + 2 * x[:, 1] ** 2 - x[:, 2] + 3, [0.7], 0.7))
        for u, lam, V in cases:
            Vq = np.full((f.n_elems, 27), V)
            ref = afem.indicators(f, u, lam, Vq)
            g = _gpu_eta2(torch, ctx, mesh, mol, u, lam, Vq).cpu().numpy()
            assert maxrel(g, ref) < 1e-12, maxrel(g, ref)
        mesh.close()


def test_dorfler_on_ties_and_extremes(ctx, torch):
    from paper_2103_02824_gb300 import mk
    rng = np.random.default_rng(7)
    v = rng.random(100_003) ** 4
    v[rng.integers(0, v.size, 500)] = v[17]            # a block of ties
    e = dev(torch, v)
    m = torch.zeros(v.size, dtype=torch.uint8, device="cuda")
    for theta in (1e-6, 0.3, 0.4, 0.9):
        nm, t = mk.mk_dorfler_mark(ctx, e, theta, m)
        gm = m.cpu().numpy().astype(bool)
        om = afem.dorfler(v, theta)
        assert nm == gm.sum() and np.all(gm[om]) and np.all(v[gm & ~om] == t)
    with pytest.raises(mk.MkError):
        mk.mk_dorfler_mark(ctx, torch.zeros(10, dtype=torch.float64, device="cuda"), 0.4, m)
