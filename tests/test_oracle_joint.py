"""Pins of the oracle's joint augmented space V_H + span{psi^_1..psi^_N} (no GPU): Ritz bounds against the coarse
and the fine Galerkin eigenvalues and against every one-orbital augmented space, M-orthonormal Ritz vectors, the
exact fixed point, and a near-degenerate spectrum."""
import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import linalg as olin
from oracle.correction import Level, correction_step
from oracle.fem import coulomb
from paper_2103_02824_gb300 import synth


def _coarse(lv, k, vext=None):
    C = lv.coarse
    xq, _, _, _ = C.quad()
    V = coulomb(xq, lv.Z, lv.R) if vext is None else vext(xq)
    A = (0.5 * C.assemble(C.element_stiffness()) + C.assemble(C.element_mass(V)))[C.free][:, C.free].toarray()
    M = C.assemble(C.element_mass())[C.free][:, C.free].toarray()
    lam, vec = sla.eigh(A, M)
    return lam[:k], vec[:, :k]


def _joint(out, k):
    return olin.joint_ritz(out["AH"], out["MH"], out["b"], out["c"], out["gramA"], out["gramM"], k)


def test_joint_space_ritz_bounds_on_a_molecule():
    wl = synth.workload("mol4_p2_small")
    cc, ct, fc, ft, par = synth.workload_meshes(wl)
    lv = Level(cc, ct, fc, ft, par, wl["order"], wl["Z"], wl["R"])
    N = synth.n_orbitals(wl["Z"])
    lamH, psiH = _coarse(lv, N)
    out = correction_step(lv, psiH, lamH, synth.occupations(wl["Z"]), sigma=20.0, xc="lda", tol=1e-12)
    lam, X = _joint(out, N)
    # the frozen Hamiltonian of the step on V_h and its Ritz values on V_H
    fr = lv.fine.free
    H = (0.5 * lv.Kff + lv.MVff + out["Mpot"][fr][:, fr]).tocsc()
    lam_h = np.sort(spla.eigsh(H, k=N, M=lv.Mff.tocsc(), sigma=-100.0, which="LM", return_eigenvectors=False))
    lam_H = sla.eigh(out["AH"], out["MH"], eigvals_only=True)[:N]
    assert np.all(lam_h - 1e-9 <= lam) and np.all(lam <= lam_H + 1e-9)
    # every one-orbital space V_H + span{psi^_i} is a subspace of the joint one
    for i in range(N):
        A1 = np.block([[out["AH"], out["b"][:, i:i + 1]], [out["b"][:, i:i + 1].T, out["gramA"][i:i + 1, i:i + 1]]])
        M1 = np.block([[out["MH"], out["c"][:, i:i + 1]], [out["c"][:, i:i + 1].T, out["gramM"][i:i + 1, i:i + 1]]])
        lam1 = sla.eigh(A1, M1, eigvals_only=True)[:N]
        assert np.all(lam <= lam1 + 1e-9)
    # M-orthonormal Ritz vectors
    M = np.block([[out["MH"], out["c"]], [out["c"].T, out["gramM"]]])
    assert np.abs(X.T @ M @ X - np.eye(N)).max() < 1e-9


def test_joint_space_fixed_point():
    """Coarse mesh = fine mesh (P = I): every psi^ lies in V_H, the extra directions are dropped, and the joint Ritz
    values are the coarse (= fine) eigenvalues."""
    c, t = synth.cube_mesh(4, 8.0)
    lv = Level(c, t, c, t, np.arange(t.shape[0]), 1, [1.0], np.zeros((1, 3)))
    lam, vec = _coarse(lv, 2)
    out = correction_step(lv, vec, lam, [1.0, 1.0], sigma=1.0, xc="none", hartree_bc="none", tol=1e-14)
    lj, _ = _joint(out, 2)
    assert np.allclose(lj, lam, rtol=1e-10, atol=1e-10)


def test_joint_space_on_a_near_degenerate_spectrum():
    """Harmonic oscillator V = |x|^2 / 2 (1.5 and a triplet at 2.5, split slightly by the meshes' anisotropy): the
    joint space returns four M-orthonormal Ritz vectors whose values lie between the fine and the coarse Galerkin
    values, at or below every one-orbital result, and much closer to the exact spectrum than the coarse values."""
    ho = lambda x: 0.5 * np.sum(x * x, axis=-1)
    cc, ct, fc, ft, par = synth.nested_cube_meshes(4, 1, 6.0)
    lv = Level(cc, ct, fc, ft, par, 2, [0.0], np.zeros((1, 3)), vext=ho)
    lamH, psiH = _coarse(lv, 4, vext=ho)
    out = correction_step(lv, psiH, lamH, [1.0] * 4, sigma=0.0, xc="none", hartree_bc="none", tol=1e-12)
    lj, X = _joint(out, 4)
    H = (0.5 * lv.Kff + lv.MVff).tocsc()
    lf = np.sort(spla.eigsh(H, k=4, M=lv.Mff.tocsc(), sigma=-1.0, which="LM", return_eigenvectors=False))
    assert np.all(lf - 1e-9 <= lj) and np.all(lj <= lamH + 1e-9)
    assert np.all(lj <= np.sort(out["lam"]) + 1e-9)
    M = np.block([[out["MH"], out["c"]], [out["c"].T, out["gramM"]]])
    assert np.abs(X.T @ M @ X - np.eye(4)).max() < 1e-9
    exact = np.array([1.5, 2.5, 2.5, 2.5])
    assert np.abs(lj - exact).max() < 0.25 * np.abs(lamH - exact).max()
