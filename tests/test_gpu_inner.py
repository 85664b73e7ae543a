"""The paper's own form of the correction step on the GPU (mk_correction_solve_vq, mk_inner_*) against the oracle's
(oracle/inner.py): Algorithm 2's inner SCF with Algorithm 3's precomputations from the same corrections and
Hartree potential (eigenvalues, coefficients, inner Hartree coefficients, iteration count, output orbitals and
potential), the whole step 5-7 from the step's input orbitals, and the case P = I where the extra Hartree direction
lies in V_H and a self-consistent orbital is a fixed point."""
import numpy as np
import pytest

from oracle import inner as OI
from oracle.correction import Level
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
    out = np.zeros((a.shape[0], ld))
    out[:, :a.shape[1]] = a
    return out


def _upload(ctx, meshes, order):
    from paper_2103_02824_gb300 import mk
    cc, ct, fc, ft, par = meshes
    return mk.Mesh(ctx, fc, ft, cc, ct, par, order)


# (name, inner tol, max_inner): hydrogen to convergence, the 7-orbital molecule over five iterations (tol 0)
INNER = [("h_p1", 1e-10, 200), ("mol4_p2_small", 0.0, 5)]


def _gpu_inner(torch, ctx, mesh, wl, N, ld, U, phit, wt, occ, tol, max_inner):
    from paper_2103_02824_gb300 import mk
    info = mesh.info
    f64 = dict(dtype=torch.float64, device="cuda")
    u = dev(torch, _pad(U, ld))
    vxc = torch.zeros((info["n_elems"], info["n_quad"]), **f64)
    mk.mk_frozen_potential(ctx, mesh, u, occ, N, torch.zeros(info["n_nodes"], **f64), wl["xc"], vxc)
    ph = dev(torch, _pad(phit, ld))
    inner = mk.Inner(ctx, mesh, mk.Molecule(wl["Z"], wl["R"]), ph, N, dev(torch, wt), vxc)
    NH = info["n_free_coarse"]
    lam, coef = torch.zeros(N, **f64), torch.zeros((NH + 1, N), **f64)
    wH, status = torch.zeros(NH, **f64), torch.zeros(N, dtype=torch.int32, device="cuda")
    rep = inner.run(occ, lam, coef, status, wH, tol=tol, max_inner=max_inner, mix=0.5)
    w = torch.zeros(info["n_nodes"], **f64)
    inner.potential(w)
    psi = torch.zeros((info["n_nodes"], ld), **f64)
    mk.mk_orbital_assemble(ctx, mesh, coef, ph, ph, N, psi)
    torch.cuda.synchronize()
    out = dict(lam=lam.cpu().numpy(), X=coef.cpu().numpy(), wH=wH.cpu().numpy(), w=w.cpu().numpy(),
               psi=psi.cpu().numpy()[:, :N], status=status.cpu().numpy(), w_in_VH=inner.w_in_VH, **rep)
    inner.close()
    return out


@pytest.mark.parametrize("name,tol,max_inner", INNER)
def test_inner_iteration_matches_oracle(ctx, torch, name, tol, max_inner):
    """Same corrections phi~ and Hartree potential w~ on both sides: Algorithm 2 with Algorithm 3's data on the GPU
    against the oracle's precomputed route, element by element."""
    c = case(name)
    lv, o, wl, N, occ = c["level"], c["out"], c["wl"], c["N"], c["occ"]
    phit, wt, vxc, _ = OI.correction_paper_form(lv, o["u"], c["lamH"], occ, c["sigma"], o["w"], c["xc"])
    ref = OI.inner_iteration(lv, phit, wt, vxc, occ, tol=tol, max_inner=max_inner, split=True, mix=0.5)
    mesh = _upload(ctx, c["meshes"], wl["order"])
    ld = max(4, (N + 3) // 4 * 4)
    g = _gpu_inner(torch, ctx, mesh, wl, N, ld, o["u"], phit, wt, occ, tol, max_inner)
    mesh.close()
    assert g["iters"] == ref["iters"], (g["iters"], ref["iters"])
    assert not g["w_in_VH"]
    lam_err = np.abs(g["lam"] - ref["lam"]).max()
    assert lam_err < 1e-9, (g["lam"], ref["lam"])
    errs = dict(X=maxrel(g["X"], ref["X"]), wH=maxrel(g["wH"], ref["wH"]), theta1=abs(g["theta1"] - ref["theta1"]),
                w=maxrel(g["w"], ref["w"]), psi=maxrel(g["psi"], ref["psi"]))
    print(f"{name}: {g['iters']} inner iterations, lambda err {lam_err:.2e}, " +
          ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    assert errs["X"] < 1e-7 and errs["wH"] < 1e-7 and errs["theta1"] < 1e-8, errs
    assert errs["w"] < 1e-8 and errs["psi"] < 1e-7, errs


@pytest.mark.parametrize("name,tol,max_inner", INNER)
def test_paper_step_matches_oracle(ctx, torch, name, tol, max_inner):
    """Steps 5-7 on the GPU from the step's input orbitals and the previous Hartree potential (the frozen potential
    on the left of the correction problems) against the oracle's paper_step."""
    from paper_2103_02824_gb300 import mk
    from paper_2103_02824_gb300.step import PaperStep
    c = case(name)
    lv, o, wl, N, occ = c["level"], c["out"], c["wl"], c["N"], c["occ"]
    ref = OI.paper_step(lv, o["u"], c["lamH"], occ, c["sigma"], o["w"], c["xc"], inner_tol=tol,
                        max_inner=max_inner)
    mesh = _upload(ctx, c["meshes"], wl["order"])
    st = PaperStep(ctx, mesh, wl["Z"], wl["R"], N)
    reps = st.run(o["u"], c["lamH"], occ, c["sigma"], o["w"], xc=wl["xc"], solve_opts=mk.opts(rtol=1e-12),
                  poisson_opts=mk.opts(rtol=1e-12), inner_tol=tol, max_inner=max_inner)
    torch.cuda.synchronize()
    phit = st.phit.cpu().numpy()[:, :N]
    lam, psi, w = st.lam.cpu().numpy(), st.psi.cpu().numpy()[:, :N], st.w.cpu().numpy()
    st.close()
    mesh.close()
    assert reps["inner"]["iters"] == ref["iters"], (reps["inner"], ref["iters"])
    errs = dict(phit=maxrel(phit, ref["phit"]), wt=maxrel(st.wt.cpu().numpy(), ref["wt"]),
                lam=np.abs(lam - ref["lam"]).max(), psi=maxrel(psi, ref["psi"]), w=maxrel(w, ref["w"]))
    print(f"{name}: paper step, " + ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    assert errs["phit"] < 1e-9 and errs["wt"] < 1e-9, errs
    assert errs["lam"] < 1e-8 and errs["psi"] < 1e-6 and errs["w"] < 1e-8, errs


def test_fixed_point_with_coarse_equal_fine(ctx, torch):
    """P = I (the coarse mesh is the fine mesh): w~0 lies in V_H, so the extra Hartree direction is dropped (its
    new coefficient is 0 in every inner iteration), and the self-consistent hydrogen orbital (Hartree + Slater exchange, computed by the oracle) is a
    fixed point of the GPU's whole paper-form step."""
    from oracle.poisson import density_at_quad, hartree
    from paper_2103_02824_gb300 import mk, synth
    from paper_2103_02824_gb300.step import PaperStep
    from tests.test_oracle_pins import _scf_hydrogen
    cm, tm = synth.cube_mesh(4, 8.0)
    Z, R = synth.hydrogen()
    lv = Level(cm, tm, cm, tm, np.arange(tm.shape[0]), 2, Z, R)
    u, lam, _ = _scf_hydrogen(lv, "slater")
    w, _ = hartree(lv.fine, density_at_quad(lv.fine, u[:, None], [1.0]), bc="multipole", tol=1e-14, K=lv.K)
    mesh = mk.Mesh(ctx, cm, tm, cm, tm, np.arange(tm.shape[0], dtype=np.int32), 2)
    st = PaperStep(ctx, mesh, Z, R, 1)
    reps = st.run(u[:, None], [lam], [1.0], 1.0, w, xc="slater", solve_opts=mk.opts(rtol=1e-13),
                  poisson_opts=mk.opts(rtol=1e-13), inner_tol=1e-11)
    torch.cuda.synchronize()
    assert st.inner.w_in_VH
    fr = lv.fine.free
    phit, psi, wg = st.phit.cpu().numpy()[:, 0], st.psi.cpu().numpy()[:, 0], st.w.cpu().numpy()
    lam_g = float(st.lam.cpu().numpy()[0])
    st.close()
    mesh.close()
    # the dropped direction's coefficient only decays under the mixing: theta_1 = 0.5^s after s iterations
    assert abs(reps["inner"]["theta1"] - 0.5 ** reps["inner"]["iters"]) < 1e-15, reps["inner"]
    assert np.abs(phit[fr] - u[fr]).max() < 1e-9 * np.abs(u).max()
    assert abs(lam_g - lam) < 1e-9, (lam_g, lam)
    assert np.abs(psi[fr] - u[fr]).max() < 1e-8 * np.abs(u).max()
    assert np.abs(wg - w).max() < 1e-8 * np.abs(w).max()
