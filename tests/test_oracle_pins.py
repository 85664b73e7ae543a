"""Pins of the oracle parts that every GPU parity test leans on, each against something other than the oracle
itself: golden values of the paper's printed correlation formula, the electron count and closed-form densities,
Lanczos against a library eigensolver and the interlacing of its Ritz values, and a self-consistent fixed point
of the correction step with the Hartree and exchange terms switched on (no GPU)."""
import os

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import linalg as olin
from oracle import xc
from oracle.correction import Level, correction_step
from oracle.fem import FEMesh
from oracle.poisson import density_at_quad, hartree
from paper_2103_02824_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    return vals


# ----------------------------------------------------------------------------------------------- LDA (Sec. 4)
def test_pz_golden_values_both_branches():
    """eps_c and V_c at r_s = 0.1, 0.5 (high-density branch) and 2, 5 (low-density branch) against the values
    worked out term by term from the printed formula (tests/golden/lda_pz.txt).  A typo in any printed constant
    (0.0311, 0.048, 0.0020, 0.0116, 0.1423, 1.0529, 0.3334), or two of them swapped, moves at least one value by
    more than 1e-6; the V_c closed forms are independent of the oracle's route through d eps_c / d r_s."""
    g = _golden("lda_pz.txt")
    for rs in ("0.1", "0.5", "2", "5"):
        r = float(rs)
        assert abs(float(xc.eps_c_pz(r)) - g[f"eps_c_{rs}"]) < 1e-14, rs
        rho = 3.0 / (4.0 * np.pi * r ** 3)
        assert abs(float(xc.v_c_pz(rho)) - g[f"v_c_{rs}"]) < 1e-13, rs
        # the LDA potential is Slater exchange plus this correlation
        assert abs(float(xc.v_xc(rho, "lda")) - (float(xc.v_x(rho)) + g[f"v_c_{rs}"])) < 1e-13


# ----------------------------------------------------------------------------------------------- density (Sec. 2)
def _p2_mesh(n=4, half=5.0):
    c, t = synth.cube_mesh(n, half)
    return FEMesh(c, t, 2)


def test_density_integrates_to_the_electron_count():
    """rho = sum_i f_i u_i^2: for M-normalised u_i its integral is sum_i f_i (the 27-point rule integrates the
    degree-4 products of P2 functions exactly).  A missing square or a wrong occupation weight fails."""
    m = _p2_mesh()
    M = m.assemble(m.element_mass())
    rng = np.random.default_rng(11)
    U = np.zeros((m.n_nodes, 3))
    U[m.free] = rng.standard_normal((m.n_free, 3))
    U /= np.sqrt(np.sum(U * (M @ U), axis=0))[None, :]
    occ = np.array([2.0, 2.0, 1.0])
    _, wq, _, _ = m.quad()
    rho = density_at_quad(m, U, occ)
    assert abs(np.sum(wq * rho) - occ.sum()) < 1e-12
    for i in range(3):   # one orbital at a time: its own occupation
        e = np.zeros(3)
        e[i] = occ[i]
        assert abs(np.sum(wq * density_at_quad(m, U, e)) - occ[i]) < 1e-12


def test_density_of_quadratic_interpolants_is_the_closed_form():
    """P2 interpolation is exact on quadratics, so for u_i = I_h q_i the density at every quadrature point is
    sum_i f_i q_i(x_q)^2 exactly (the points of every element, not just their sum)."""
    m = _p2_mesh(3, 4.0)
    q1 = lambda x: 1.0 + x[..., 0] - 2.0 * x[..., 1] + 0.5 * x[..., 0] * x[..., 2]
    q2 = lambda x: x[..., 1] ** 2 - x[..., 2]
    U = np.stack([q1(m.nodes), q2(m.nodes)], axis=1)
    xq, _, _, _ = m.quad()
    rho = density_at_quad(m, U, [2.0, 0.5])
    exact = 2.0 * q1(xq) ** 2 + 0.5 * q2(xq) ** 2
    assert np.abs(rho - exact).max() < 1e-12 * np.abs(exact).max()


# ----------------------------------------------------------------------------------------------- Lanczos (shift)
def _hydrogen_level(n_coarse, levels, order, half=10.0):
    cc, ct, fc, ft, par = synth.nested_cube_meshes(n_coarse, levels, half)
    Z, R = synth.hydrogen()
    return Level(cc, ct, fc, ft, par, order, Z, R)


def test_lanczos_lowest_against_library_eigensolver():
    """The lowest Ritz value of Lanczos on (K/2 + M_Vext, M): with more steps than unknowns it is the pencil's
    lowest eigenvalue (here from scipy's eigsh and LAPACK's dense eigh); for fewer steps it is an upper bound and
    it never increases with the step count (Cauchy interlacing of nested tridiagonal matrices)."""
    lv = _hydrogen_level(3, 1, 1)                        # P1, 6^3 cubes: 125 free DOF
    H = (0.5 * lv.Kff + lv.MVff).tocsr()
    lam_dense = sla.eigh(H.toarray(), lv.Mff.toarray(), eigvals_only=True)[0]
    lam_arpack = spla.eigsh(H.tocsc(), k=1, M=lv.Mff.tocsc(), sigma=-10.0, which="LM",
                            return_eigenvectors=False)[0]
    assert abs(lam_dense - lam_arpack) < 1e-10
    v0 = synth.lanczos_start(lv.fine.n_free)
    assert abs(olin.lanczos_lowest(H, lv.Mff, v0, steps=200) - lam_dense) < 1e-9
    prev = np.inf
    for k in (2, 4, 8, 16, 32):
        th = olin.lanczos_lowest(H, lv.Mff, v0, steps=k)
        assert th >= lam_dense - 1e-10
        assert th <= prev + 1e-12
        prev = th
    # the shift rule built on it makes the correction operator positive definite with margin
    sigma = olin.shift_rule(olin.lanczos_lowest(H, lv.Mff, v0, steps=60))
    assert sla.eigh((H + sigma * lv.Mff).toarray(), lv.Mff.toarray(), eigvals_only=True)[0] > 0.45


def test_lanczos_lowest_on_a_p2_mesh_converges_from_above():
    lv = _hydrogen_level(2, 1, 2)                        # P2, 4^3 cubes: 343 free DOF
    H = (0.5 * lv.Kff + lv.MVff).tocsr()
    lam = sla.eigh(H.toarray(), lv.Mff.toarray(), eigvals_only=True)[0]
    th = olin.lanczos_lowest(H, lv.Mff, synth.lanczos_start(lv.fine.n_free), steps=60)
    assert lam - 1e-10 <= th < lam + 1e-6 * abs(lam)


# ----------------------------------------------------------------------------------------------- V_Hxc term of A3
def _scf_hydrogen(lv, xc_kind, tol=1e-13, mix=0.5, maxit=400):
    """Self-consistent lowest orbital of hydrogen with Hartree (multipole boundary values) and the given exchange
    on the single mesh of lv (coarse = fine): the frozen-potential eigenproblem iterated with linear mixing of
    the potential at the quadrature points until it reproduces its own potential."""
    f = lv.fine
    fr = f.free
    Hb = (0.5 * lv.Kff + lv.MVff).toarray()
    Mff = lv.Mff.toarray()
    lam, V = sla.eigh(Hb, Mff)
    u = np.zeros(f.n_nodes)
    u[fr] = V[:, 0]
    vin = None
    for it in range(maxit):
        rho = density_at_quad(f, u[:, None], [1.0])
        w, _ = hartree(f, rho, bc="multipole", tol=1e-14, K=lv.K)
        vout = f.eval_at_quad(w) + xc.v_xc(rho, xc_kind)
        if vin is not None and np.abs(vout - vin).max() < tol * np.abs(vout).max():
            break
        vin = vout if vin is None else (1.0 - mix) * vin + mix * vout
        Mp = f.assemble(f.element_mass(vin))[fr][:, fr].toarray()
        lam, V = sla.eigh(Hb + Mp, Mff)
        u = np.zeros(f.n_nodes)
        u[fr] = V[:, 0] * np.sign(V[np.argmax(np.abs(V[:, 0])), 0])
    else:
        raise AssertionError("SCF did not converge")
    return u, lam[0], it


def test_self_consistent_orbital_is_a_fixed_point_with_hartree_and_exchange():
    """P = I (coarse mesh = fine mesh) and a self-consistent hydrogen orbital with Hartree and Slater exchange: the
    right-hand side (lambda + sigma) M u - M_{w + V_xc(rho)} u then equals (K/2 + M_Vext + sigma M) u, so the
    correction returns psi^ = u for any sigma, and the augmented problem returns the same eigenvalue (psi^ lies in
    V_H: the singular case).  A sign error on the V_Hxc term, w counted twice, the exchange dropped, or a wrong
    sign of the potential in the projected Hamiltonian each breaks one of the equalities."""
    c, t = synth.cube_mesh(4, 8.0)
    Z, R = synth.hydrogen()
    lv = Level(c, t, c, t, np.arange(t.shape[0]), 2, Z, R)
    u, lam, it = _scf_hydrogen(lv, "slater")
    fr = lv.fine.free
    # the potential is not small: the fixed point would be trivial if V_Hxc vanished
    rho = density_at_quad(lv.fine, u[:, None], [1.0])
    w, _ = hartree(lv.fine, rho, bc="multipole", tol=1e-14, K=lv.K)
    assert np.abs(w).max() > 0.1 and np.abs(xc.v_xc(rho, "slater")).max() > 0.1
    lam_bare = sla.eigh((0.5 * lv.Kff + lv.MVff).toarray(), lv.Mff.toarray(), eigvals_only=True)[0]
    assert lam - lam_bare > 0.05
    for sigma in (1.0, 4.0):
        out = correction_step(lv, u[fr][:, None], [lam], [1.0], sigma, xc="slater", hartree_bc="multipole",
                              tol=1e-14)
        assert np.abs(out["psihat"][fr, 0] - u[fr]).max() < 1e-9 * np.abs(u).max()
        assert out["status"][0] == olin.STATUS_SINGULAR_AUG
        assert abs(out["lam"][0] - lam) < 1e-10
        assert np.abs(out["psi"][fr, 0] - u[fr]).max() < 1e-9 * np.abs(u).max()


def test_fixed_point_needs_the_potential_on_the_right_hand_side():
    """The same self-consistent orbital fed to a step without the Hartree and exchange terms is no fixed point:
    the pin above depends on the V_Hxc term being applied, with its sign."""
    c, t = synth.cube_mesh(4, 8.0)
    Z, R = synth.hydrogen()
    lv = Level(c, t, c, t, np.arange(t.shape[0]), 2, Z, R)
    u, lam, _ = _scf_hydrogen(lv, "slater")
    fr = lv.fine.free
    out = correction_step(lv, u[fr][:, None], [lam], [1.0], 1.0, xc="none", hartree_bc="none", tol=1e-14)
    assert np.abs(out["psihat"][fr, 0] - u[fr]).max() > 1e-3 * np.abs(u).max()
