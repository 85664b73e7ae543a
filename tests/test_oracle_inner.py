"""Pins of the oracle's paper-form correction step with its inner iteration (oracle/inner.py), no GPU: Algorithm 3's
precomputed route equals the definition (fine-mesh assembly every inner iteration), the inner Hartree space
reproduces the step's own Hartree potential from the step's density (the boundary-lift reading), and a
self-consistent orbital is a fixed point of the whole step."""
import numpy as np
import scipy.linalg as sla

from oracle import inner as OI
from oracle import linalg as olin
from oracle.correction import Level
from oracle.poisson import density_at_quad
from paper_2103_02824_gb300 import synth
from tests._cases import case
from tests.test_oracle_pins import _scf_hydrogen


def test_precomputed_route_equals_the_definition():
    """Algorithm 3 reorganises Algorithm 2's fine-mesh integrals exactly: the two routes agree to rounding, here on
    hydrogen to convergence and on the 7-orbital molecule over five inner iterations (mixing on)."""
    for name, kw in (("h_p1", dict(tol=1e-10)), ("mol4_p2_small", dict(tol=0.0, max_inner=5))):
        c = case(name)
        lv, o = c["level"], c["out"]
        phit, wt, vxc, _ = OI.correction_paper_form(lv, o["u"], c["lamH"], c["occ"], c["sigma"], o["w"], c["xc"])
        r1 = OI.inner_iteration(lv, phit, wt, vxc, c["occ"], split=False, **kw)
        r2 = OI.inner_iteration(lv, phit, wt, vxc, c["occ"], split=True, **kw)
        assert r1["iters"] == r2["iters"]
        assert np.abs(r1["lam"] - r2["lam"]).max() < 1e-12 * max(1.0, np.abs(r1["lam"]).max())
        assert np.abs(r1["X"] - r2["X"]).max() < 1e-10 * np.abs(r1["X"]).max()
        assert np.abs(r1["w"] - r2["w"]).max() < 1e-10 * np.abs(r1["w"]).max()


def test_inner_hartree_space_reproduces_the_step_potential():
    """With the density of step 6 the Galerkin solution in w_b + V_H + span{w~0} is w~ itself (w_H = 0,
    theta_1 = 1): the lift keeps the boundary values out of the test space."""
    c = case("mol4_p2_small")
    lv, o = c["level"], c["out"]
    phit, wt, vxc, _ = OI.correction_paper_form(lv, o["u"], c["lamH"], c["occ"], c["sigma"], o["w"], c["xc"])
    wH, th1, w = OI.hartree_in_W(lv, wt, density_at_quad(lv.fine, phit, c["occ"]))
    assert abs(th1 - 1.0) < 1e-9 and np.abs(wH).max() < 1e-9 * np.abs(wt).max()
    assert np.abs(w - wt).max() < 1e-9 * np.abs(wt).max()


def test_self_consistent_orbital_is_a_fixed_point_of_the_paper_step():
    """P = I and the self-consistent hydrogen orbital (Hartree + Slater exchange): the paper-form correction returns
    the orbital, the inner iteration (the full SCF, since V_H = V_h) keeps it, and the eigenvalue is unchanged."""
    c, t = synth.cube_mesh(4, 8.0)
    Z, R = synth.hydrogen()
    lv = Level(c, t, c, t, np.arange(t.shape[0]), 2, Z, R)
    u, lam, _ = _scf_hydrogen(lv, "slater")
    from oracle.poisson import hartree
    w, _ = hartree(lv.fine, density_at_quad(lv.fine, u[:, None], [1.0]), bc="multipole", tol=1e-14, K=lv.K)
    out = OI.paper_step(lv, u[:, None], [lam], [1.0], 1.0, w, "slater", tol=1e-14, inner_tol=1e-11)
    fr = lv.fine.free
    assert np.abs(out["phit"][fr, 0] - u[fr]).max() < 1e-9 * np.abs(u).max()
    assert abs(out["lam"][0] - lam) < 1e-9
    assert np.abs(out["psi"][fr, 0] - u[fr]).max() < 1e-8 * np.abs(u).max()
    assert np.abs(out["w"] - w).max() < 1e-8 * np.abs(w).max()
