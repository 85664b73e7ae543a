"""The Refine step on the GPU (mk_refine) against the oracle's newest-vertex bisection (oracle/refine.py): identical
vertices, tetrahedra, tags and parent map (the numbering rules are deterministic on both sides) over several
successive refinements with random marks, one whole Estimate -> Mark -> Refine cycle on the graded 12-nucleus mesh,
and the capacity check."""
import numpy as np
import pytest

from oracle import afem
from oracle import refine as R

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


def _same(g, o):
    Xg, Tg, Kg, Pg, rg = g
    Xo, To, Ko, Po, ro = o
    assert rg == ro
    assert np.array_equal(Tg, To) and np.array_equal(Kg, Ko) and np.array_equal(Pg, Po)
    assert np.array_equal(Xg, Xo)            # midpoints 0.5 (a + b) in FP64 on both sides


def test_successive_refinements_match_oracle(ctx, torch):
    from paper_2103_02824_gb300 import mk, synth
    rng = np.random.default_rng(11)
    nvb = synth.NVBMesh.kuhn(3, 2.0)
    X, T, K = nvb.coords().copy(), nvb.T.copy(), nvb.K.copy()
    for step in range(5):
        marked = rng.random(len(T)) < (0.3 if step < 2 else 0.05)
        g = mk.refine_mesh(ctx, X, T, K, marked)
        o = R.refine(X, T, K, marked)
        _same(g, o)
        X, T, K = o[0], o[1], o[2]
    assert len(T) > 6 * 27 * 4


def test_estimate_mark_refine_cycle_matches_oracle(ctx, torch):
    """One AFEM cycle on the graded 12-nucleus mesh: the oracle's corrected orbitals, their indicator and Dorfler's
    marks on the GPU, the refined mesh on the GPU, against the same three steps on the oracle."""
    from oracle.poisson import density_at_quad, hartree
    from paper_2103_02824_gb300 import mk, synth
    from tests._cases import case
    c = case("cluster12_p2_small")
    lv, o, wl = c["level"], c["out"], c["wl"]
    keep = []
    synth.graded_mesh(wl["n_coarse"], wl["half"], wl["R"], h_min=wl["h_min"], alpha=wl["alpha"], maubach=keep)
    nvb = keep[0]
    assert np.array_equal(nvb.coords(), lv.fine.coords) and nvb.T.shape[0] == lv.fine.n_elems
    psi, lam, occ = o["psi"], o["lam"], c["occ"]
    w, _ = hartree(lv.fine, density_at_quad(lv.fine, psi, occ), bc="multipole", tol=1e-13, K=lv.K)
    eta_o = afem.indicators(lv.fine, psi, lam, afem.ks_potential(lv, psi, occ, w, wl["xc"]))
    mark_o = afem.dorfler(eta_o, 0.4)
    ref = R.refine(nvb.coords(), nvb.T, nvb.K, mark_o)
    # the GPU's own indicator and marks
    cc, ct, fc, ft, par = c["meshes"]
    mesh = mk.Mesh(ctx, fc, ft, cc, ct, par, wl["order"])
    info = mesh.info
    N = len(lam)
    ld = max(4, (N + 3) // 4 * 4)
    pd = torch.zeros((info["n_nodes"], ld), dtype=torch.float64, device="cuda")
    pd[:, :N] = torch.from_numpy(psi).cuda()
    vq = torch.zeros((info["n_elems"], info["n_quad"]), dtype=torch.float64, device="cuda")
    mk.mk_frozen_potential(ctx, mesh, pd, occ, N, torch.from_numpy(w).cuda(), wl["xc"], vq)
    eta = torch.zeros(info["n_elems"], dtype=torch.float64, device="cuda")
    mk.mk_error_indicators(ctx, mesh, mk.Molecule(wl["Z"], wl["R"]), pd, N, lam, vq, eta)
    marked = torch.zeros(info["n_elems"], dtype=torch.uint8, device="cuda")
    nm, _ = mk.mk_dorfler_mark(ctx, eta, 0.4, marked)
    mark_g = marked.cpu().numpy().astype(bool)
    assert np.array_equal(mark_g, mark_o), (nm, mark_o.sum())
    g = mk.refine_mesh(ctx, nvb.coords(), nvb.T, nvb.K, mark_g)
    _same(g, ref)
    print(f"\ncluster12_p2_small: {mark_g.sum()} marked, {len(nvb.T)} -> {len(g[1])} elements in {g[4]} rounds")
    mesh.close()


def test_capacity_and_input_are_checked(ctx, torch):
    from paper_2103_02824_gb300 import mk, synth
    nvb = synth.NVBMesh.kuhn(2, 1.0)
    with pytest.raises(mk.MkError) as e:
        mk.refine_mesh(ctx, nvb.coords(), nvb.T, nvb.K, np.ones(48, dtype=bool), max_elems=60)
    assert e.value.code == mk.MK_ERR_INVALID_ARG
    bad = nvb.K.copy()
    bad[5] = 0                                   # a tag outside {1, 2, 3} is rejected before any bisection
    with pytest.raises(mk.MkError) as e:
        mk.refine_mesh(ctx, nvb.coords(), nvb.T, bad, np.ones(48, dtype=bool))
    assert e.value.code == mk.MK_ERR_INVALID_ARG
