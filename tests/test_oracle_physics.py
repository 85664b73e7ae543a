"""Pins of the oracle's LDA, Poisson and correction step against closed forms, invariants and bounds (no GPU)."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla
from scipy.special import erf

from oracle import linalg as olin
from oracle import xc
from oracle.correction import Level, correction_step
from oracle.fem import FEMesh, coulomb
from oracle.poisson import direct_potential, hartree, multipole_moments, multipole_potential
from paper_2103_02824_gb300 import synth

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    for line in open(f"{GOLDEN}/{name}"):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    return vals


# ----------------------------------------------------------------------------------------------- LDA
def test_slater_exchange_closed_forms():
    rho = np.array([1e-6, 1e-3, 0.1, 1.0, 30.0])
    assert np.allclose(xc.v_x(rho), 4.0 / 3.0 * xc.eps_x(rho), rtol=1e-15)
    h = 1e-6 * rho
    fd = ((rho + h) * xc.eps_x(rho + h) - (rho - h) * xc.eps_x(rho - h)) / (2 * h)
    assert np.allclose(xc.v_xc(rho, "slater"), fd, rtol=1e-8)
    assert np.allclose(xc.v_xc(rho, "xalpha", alpha=2.0 / 3.0), xc.v_xc(rho, "slater"), rtol=1e-15)
    # the value at rho = pi/3 is -1 exactly: (3 rho / pi)^(1/3) = 1
    assert abs(xc.v_x(np.pi / 3.0) + 1.0) < 1e-15


def test_pz_correlation_printed_parametrisation():
    g = _golden("lda_pz.txt")
    # the two branches meet (to the printed digits) at r_s = 1
    assert abs(xc.eps_c_pz(1.0 - 1e-12) - xc.eps_c_pz(1.0)) < 1e-4
    assert abs(xc.eps_c_pz(1.0) - g["eps_c_rs1"]) < 1e-5
    # high-density limit: eps_c(r_s) - eps_c(r_s / e) -> 0.0311 (Gell-Mann--Brueckner log coefficient)
    rs = 1e-6
    assert abs(xc.eps_c_pz(rs) - xc.eps_c_pz(rs / math.e) - g["A_log"]) < 1e-6
    # V_c = d(rho eps_c)/d rho by central differences, on both branches
    for rho in [1e-4, 1e-2, 0.05, 1.0, 50.0]:
        h = 1e-6 * rho
        f = lambda r: r * xc.eps_c_pz(np.cbrt(3 / (4 * np.pi * r)))
        fd = (f(rho + h) - f(rho - h)) / (2 * h)
        assert abs(xc.v_c_pz(rho) - fd) < 1e-8 * max(1.0, abs(fd))
    assert xc.v_xc(np.array([0.0, 1e-31]), "lda").tolist() == [0.0, 0.0]


# ----------------------------------------------------------------------------------------------- Poisson
def test_gaussian_charge_poisson():
    """Normalised Gaussian charge of width s: V(r) = Q erf(r / (sqrt(2) s)) / r.  The monopole boundary value is
    exact for a centred spherical charge; the P2 solution converges to V under refinement."""
    s, Q, L = 0.8, 1.0, 6.0
    errs = []
    for n in (8, 16):
        c, t = synth.cube_mesh(n, L)
        m = FEMesh(c, t, 2)
        xq, _, _, _ = m.quad()
        r2 = np.sum(xq * xq, axis=-1)
        rhoq = Q * (2 * np.pi * s * s) ** -1.5 * np.exp(-0.5 * r2 / (s * s))
        q0, p, Qm = multipole_moments(m, rhoq)
        assert abs(q0 - Q) < 1e-3 and np.abs(p).max() < 1e-4 and np.abs(Qm).max() < 1e-3  # quadrature error only
        w, info = hartree(m, rhoq, bc="multipole")
        assert info["rel_res"] < 1e-12
        r = np.linalg.norm(m.nodes, axis=1)
        ok = r > 0.5
        exact = Q * erf(r[ok] / (math.sqrt(2) * s)) / r[ok]
        errs.append(np.abs(w[ok] - exact).max() / exact.max())
    assert errs[1] < 0.25 * errs[0] and errs[1] < 3e-3


def test_multipole_vs_direct_sum():
    c, t = synth.cube_mesh(4, 5.0)
    m = FEMesh(c, t, 1)
    xq, _, _, _ = m.quad()
    d = xq - np.array([0.7, -0.4, 0.3])
    rhoq = np.exp(-np.sum(d * d, axis=-1) / 0.6)
    bnd = m.nodes[m.boundary]
    direct = direct_potential(bnd, m, rhoq)
    mono = multipole_potential(bnd, multipole_moments(m, rhoq)[0], np.zeros(3), np.zeros((3, 3)))
    full = multipole_potential(bnd, *multipole_moments(m, rhoq))
    e_mono = np.abs(mono - direct).max() / direct.max()
    e_full = np.abs(full - direct).max() / direct.max()
    assert e_full < 5e-3 and e_full < 0.1 * e_mono   # truncation after l = 2: error ~ (a / r)^3


# ----------------------------------------------------------------------------------------------- solvers
def test_pcg_matches_direct_solve():
    lv = _level(1, 1, 1, 6.0, synth.hydrogen())
    A = lv.operator(1.0)
    b = np.random.default_rng(1).standard_normal((A.shape[0], 3))
    x, it, res = olin.pcg(A, b, tol=1e-14)
    xd = spla.spsolve(A.tocsc(), b)
    assert np.abs(x - xd).max() < 1e-11 * np.abs(xd).max() and res.max() < 1e-13


def test_pcg_breakdown_detected():
    lv = _level(2, 1, 1, 10.0, synth.hydrogen())
    A = (0.5 * lv.Kff + lv.MVff - 5.0 * lv.Mff).tocsr()        # shift far below -0.5: indefinite
    with pytest.raises(olin.Breakdown):
        olin.pcg(A, np.ones(A.shape[0]), tol=1e-12)


def _level(nc, levels, order, half, mol, vext=None):
    cc, ct, fc, ft, par = synth.nested_cube_meshes(nc, levels, half)
    return Level(cc, ct, fc, ft, par, order, mol[0], mol[1], vext=vext)


def _coarse_eigs(lv, k, vext=None):
    C = lv.coarse
    xq, _, _, _ = C.quad()
    V = coulomb(xq, lv.Z, lv.R) if vext is None else vext(xq)
    A = (0.5 * C.assemble(C.element_stiffness()) + C.assemble(C.element_mass(V)))[C.free][:, C.free].toarray()
    M = C.assemble(C.element_mass())[C.free][:, C.free].toarray()
    lam, Vec = sla.eigh(A, M)
    return lam[:k], Vec[:, :k]


def _fine_lowest(lv, k=1):
    H = (0.5 * lv.Kff + lv.MVff).tocsc()
    return np.sort(spla.eigsh(H, k=k, M=lv.Mff.tocsc(), sigma=-100.0, which="LM", return_eigenvectors=False))


# ----------------------------------------------------------------------------------------------- correction step
def test_hydrogen_correction_bounds_and_convergence():
    """Bare hydrogen (V_Hxc = 0): the corrected eigenvalue lies between the fine Galerkin eigenvalue and the coarse
    one (Rayleigh-Ritz in V_H + span{psi^}) and decreases toward -0.5 Ha as the fine mesh is refined."""
    for order, levels_list, final in ((1, (1, 2), 0.2), (2, (1,), 0.12)):
        lams = []
        for levels in levels_list:
            lv = _level(4, levels, order, 10.0, synth.hydrogen())
            lamH, psiH = _coarse_eigs(lv, 1)
            out = correction_step(lv, psiH, lamH, [1.0], sigma=1.0, xc="none", hartree_bc="none")
            lf = _fine_lowest(lv)[0]
            assert lf - 1e-10 <= out["lam"][0] <= lamH[0] + 1e-12
            assert out["lam"][0] > -0.5
            lams.append(out["lam"][0])
        assert all(b < a for a, b in zip(lams, lams[1:]))
        assert abs(lams[-1] + 0.5) < final


def test_harmonic_oscillator_spectrum():
    """V = |x|^2 / 2: eigenvalues 1.5 and 2.5 (x3).  P2 on [-6,6]^3, error falls with refinement."""
    ho = lambda x: 0.5 * np.sum(x * x, axis=-1)
    errs = []
    for levels in (0, 1):
        cc, ct, fc, ft, par = synth.nested_cube_meshes(6 * 2 ** levels, 0, 6.0)
        lv = Level(cc, ct, fc, ft, par, 2, [0.0], np.zeros((1, 3)), vext=ho)
        ev = _fine_lowest(lv, k=4)
        errs.append(np.abs(ev - [1.5, 2.5, 2.5, 2.5]).max())
    assert errs[1] < 0.15 * errs[0] and errs[1] < 0.06


def test_harmonic_oscillator_correction_recovers_fine_eigenvalue():
    ho = lambda x: 0.5 * np.sum(x * x, axis=-1)
    lv = _level(4, 1, 2, 6.0, ([0.0], np.zeros((1, 3))), vext=ho)
    lamH, psiH = _coarse_eigs(lv, 1, vext=ho)
    out = correction_step(lv, psiH, lamH, [1.0], sigma=0.0, xc="none", hartree_bc="none")
    lf = _fine_lowest(lv)[0]
    assert lf - 1e-10 <= out["lam"][0] < lamH[0]
    # one correction removes most of the coarse error
    assert out["lam"][0] - lf < 0.2 * (lamH[0] - lf)


def test_exact_eigenpair_is_a_fixed_point():
    """Coarse mesh = fine mesh (P = I): an exact eigenpair gives psi^ = psi_H (for any sigma), the augmented mass
    matrix is singular (psi^ in V_H) and the coarse Ritz pair, i.e. the same eigenpair, comes back."""
    c, t = synth.cube_mesh(4, 8.0)
    lv = Level(c, t, c, t, np.arange(t.shape[0]), 1, [1.0], np.zeros((1, 3)))
    lam, vec = _coarse_eigs(lv, 2)
    for sigma in (1.0, 3.0):
        out = correction_step(lv, vec, lam, [1.0, 1.0], sigma=sigma, xc="none", hartree_bc="none", tol=1e-14)
        assert np.abs(out["psihat"][lv.fine.free] - vec).max() < 1e-10
        assert np.all(out["status"] == olin.STATUS_SINGULAR_AUG)
        assert np.allclose(out["lam"], lam, rtol=1e-12, atol=1e-12)


def test_arrowhead_route_agrees_and_interlaces():
    wl = synth.workload("mol4_p2_small")
    lv = _level(wl["n_coarse"], wl["levels"], wl["order"], wl["half"], (wl["Z"], wl["R"]))
    N = synth.n_orbitals(wl["Z"])
    lamH, psiH = _coarse_eigs(lv, N)
    occ = synth.occupations(wl["Z"])
    out = correction_step(lv, psiH, lamH, occ, sigma=8.0, xc="lda", hartree_bc="multipole")
    assert out["cg_res"].max() < 1e-12
    G = out["gramA"]
    assert np.allclose(G, G.T, atol=1e-10 * np.abs(G).max())
    assert np.all(np.linalg.eigvalsh(out["gramM"]) > 0)
    ritz = sla.eigh(out["AH"], out["MH"], eigvals_only=True)
    for i in range(N):
        l2, c2, s2 = olin.arrowhead_select(out["AH"], out["MH"], out["b"][:, i], out["c"][:, i],
                                           out["beta"][i], out["gamma"][i])
        assert abs(l2 - out["lam"][i]) < 1e-11 * max(1, abs(l2))
        assert np.abs(c2 - out["coef"][:, i]).max() < 1e-9
        # selected eigenvalue k of the augmented pencil is <= the k-th coarse Ritz value (interlacing)
        full = np.sort(sla.eigh(*_aug(out, i), eigvals_only=True))
        k = int(np.argmin(np.abs(full - out["lam"][i])))
        assert k >= len(ritz) or full[k] <= ritz[k] + 1e-10
    # A8: orbitals are M-normalised
    Mff = lv.Mff
    psi = out["psi"][lv.fine.free]
    assert np.allclose(np.sum(psi * (Mff @ psi), axis=0), 1.0, atol=1e-10)


def _aug(out, i):
    n = out["AH"].shape[0]
    A = np.zeros((n + 1, n + 1))
    M = np.zeros((n + 1, n + 1))
    A[:n, :n], A[:n, n], A[n, :n], A[n, n] = out["AH"], out["b"][:, i], out["b"][:, i], out["beta"][i]
    M[:n, :n], M[:n, n], M[n, :n], M[n, n] = out["MH"], out["c"][:, i], out["c"][:, i], out["gamma"][i]
    return A, M


def test_singular_augmented_returns_coarse_ritz_pair():
    rng = np.random.default_rng(3)
    n = 12
    X = rng.standard_normal((n, n))
    MH = X @ X.T + n * np.eye(n)
    AH = rng.standard_normal((n, n))
    AH = AH + AH.T
    t = rng.standard_normal(n)
    lam, coef, st, _ = olin.augmented_select(AH, MH, AH @ t, MH @ t, t @ AH @ t, t @ MH @ t)
    assert st == olin.STATUS_SINGULAR_AUG and coef[-1] == 0.0
    ev = sla.eigh(AH, MH, eigvals_only=True)
    assert np.min(np.abs(ev - lam)) < 1e-12


def test_selection_prefers_alignment_not_theta():
    """The selected eigenvector maximises |(x, phi~)_M|; selecting by |theta_2| instead would pick the high,
    fine-scale eigenvector (theta_2 ~ 1/||u||), far above the physical one."""
    wl = synth.workload("h_p1")
    lv = _level(wl["n_coarse"], wl["levels"], 1, wl["half"], (wl["Z"], wl["R"]))
    lamH, psiH = _coarse_eigs(lv, 1)
    out = correction_step(lv, psiH, lamH, [1.0], sigma=1.0, xc="none", hartree_bc="none")
    A, M = _aug(out, 0)
    lam, X = sla.eigh(A, M)
    k_theta = int(np.argmax(np.abs(X[-1])))
    assert lam[k_theta] > out["lam"][0] + 1.0
    assert abs(out["lam"][0] - lam[0]) < 1e-12
