"""One eigenpairwise fine-mesh correction step (oracle side), in the paper's order.

Algorithm 1, steps 5-7, in the form where the frozen Hartree-exchange-correlation potential of the coarse density
rho_H sits on the right-hand side (the boundary-value problem of the original multilevel correction scheme):

  A1  u_i = P psi_{H,i}                           (V_H subset V_h, coarse function on the fine mesh)
  A2  (grad w, grad v) = 4 pi (rho_H, v)          (Sec. 2, Eq. (W_h_equation) with rho_H = sum_i f_i u_i^2)
  A3  b_i(v) = (lambda_{H,i} + sigma)(u_i, v) - ((w + V_xc(rho_H)) u_i, v)
  A4  (1/2)(grad psi^_i, grad v) + (V_ext psi^_i, v) + sigma (psi^_i, v) = b_i(v)     (Eq. (Aux_Linear_Problem))
  A6  A_H = P^T H P, M_H = P^T M P, b_i = P^T H psi^_i, c_i = P^T M psi^_i, beta_i, gamma_i  (Eqs. (Adef)-(betadef))
      with H = K/2 + M_{V_ext} + M_{w + V_xc(rho_H)} the Hamiltonian at the frozen density
  A7  Eq. (Eigenvalue_H_h) per orbital, eigenvector with the largest component along psi^_i (Algorithm 2 (a))
  A8  psi_i = P phi_{i,H} + theta_{2,i} psi^_i  (Algorithm 3, output)

Readings (the paper is silent or garbled here): a(.,.) = (1/2)(grad, grad) with V_ext added once; the shift sigma
keeps the operator positive definite (an exact eigenpair is a fixed point for any sigma); rho = sum_i f_i phi_i^2
with the occupation numbers f_i; the augmented eigenproblem itself is unshifted.
"""
from __future__ import annotations

import numpy as np

from .fem import FEMesh, coulomb, interpolation
from .linalg import STATUS_OK, augmented_select, pcg
from .poisson import density_at_quad, hartree
from .xc import v_xc


class Level:
    """A fine/coarse pair with the assembled operators that do not depend on the density.  `vext`, if given, is a
    closed-form potential x [.., 3] -> V [..] replacing the nuclear Coulomb potential (used by the pins)."""

    def __init__(self, coarse_coords, coarse_tets, fine_coords, fine_tets, parent, order, Z, R, vext=None):
        self.fine = FEMesh(fine_coords, fine_tets, order)
        self.coarse = FEMesh(coarse_coords, coarse_tets, order)
        self.parent = np.asarray(parent, dtype=np.int64)
        self.Z, self.R = np.asarray(Z, dtype=np.float64), np.asarray(R, dtype=np.float64)
        f = self.fine
        self.P = interpolation(self.coarse, f, self.parent)           # [n_nodes fine, n_nodes coarse]
        self.Pf = self.P[f.free][:, self.coarse.free].tocsr()         # free rows, free columns
        self.K = f.assemble(f.element_stiffness())
        self.M = f.assemble(f.element_mass())
        xq, _, _, _ = f.quad()
        Vq = coulomb(xq, self.Z, self.R) if vext is None else vext(xq)
        self.MV = f.assemble(f.element_mass(Vq))
        fr = f.free
        self.Kff = self.K[fr][:, fr].tocsr()
        self.Mff = self.M[fr][:, fr].tocsr()
        self.MVff = self.MV[fr][:, fr].tocsr()

    def prolong(self, psiH_free: np.ndarray) -> np.ndarray:
        """A1: coarse free-DOF coefficients [N_H, N] -> fine nodal values on all nodes [n_nodes, N]."""
        return self.P[:, self.coarse.free] @ psiH_free

    def operator(self, sigma: float):
        """K/2 + M_{V_ext} + sigma M on the free DOF (the operator of A4)."""
        return (0.5 * self.Kff + self.MVff + sigma * self.Mff).tocsr()


def potential_matrix(level: Level, U, occ, w, xc: str):
    """M_{w + V_xc(rho_H)} (all nodes) with rho_H from nodal values U."""
    f = level.fine
    rho = density_at_quad(f, U, occ)
    fq = f.eval_at_quad(w) + v_xc(rho, xc)
    return f.assemble(f.element_mass(fq)), rho


def correction_step(level: Level, psiH, lamH, occ, sigma: float, xc: str = "lda", hartree_bc: str = "multipole",
                    tol: float = 1e-13, x0=None):
    """Runs A1-A8 and returns every intermediate result (fine vectors on all nodes)."""
    f = level.fine
    fr = f.free
    psiH = np.asarray(psiH, dtype=np.float64)
    N = psiH.shape[1]
    lamH = np.asarray(lamH, dtype=np.float64)
    out = {}
    U = level.prolong(psiH)                                            # A1
    out["u"] = U
    rho = density_at_quad(f, U, occ)
    if hartree_bc == "none":                                           # A2
        w = np.zeros(f.n_nodes)
        out["poisson"] = dict(iters=0, rel_res=0.0)
    else:
        w, info = hartree(f, rho, bc=hartree_bc, tol=tol, K=level.K)
        out["poisson"] = info
    out["w"] = w
    Mpot, _ = potential_matrix(level, U, occ, w, xc)                   # A3
    out["Mpot"] = Mpot
    Mpot_ff = Mpot[fr][:, fr].tocsr()
    Uf = U[fr]
    B = (level.Mff @ Uf) * (lamH + sigma)[None, :] - Mpot_ff @ Uf
    rhs = np.zeros((f.n_nodes, N))
    rhs[fr] = B
    out["rhs"] = rhs
    A = level.operator(sigma)                                          # A4
    X0 = Uf if x0 is None else x0[fr]
    Xf, iters, res = pcg(A, B, X0=X0, tol=tol)
    psihat = np.zeros((f.n_nodes, N))
    psihat[fr] = Xf
    out["psihat"], out["cg_iters"], out["cg_res"] = psihat, iters, res
    H = (0.5 * level.Kff + level.MVff + Mpot_ff).tocsr()               # A6
    Pf = level.Pf
    HX, MX = H @ Xf, level.Mff @ Xf
    out["AH"] = (Pf.T @ (H @ Pf)).toarray()
    out["MH"] = (Pf.T @ (level.Mff @ Pf)).toarray()
    out["b"] = Pf.T @ HX
    out["c"] = Pf.T @ MX
    out["gramA"] = Xf.T @ HX
    out["gramM"] = Xf.T @ MX
    out["beta"] = np.diag(out["gramA"]).copy()
    out["gamma"] = np.diag(out["gramM"]).copy()
    lam = np.zeros(N)                                                  # A7
    coef = np.zeros((out["AH"].shape[0] + 1, N))
    status = np.zeros(N, dtype=np.int64)
    scores = []
    for i in range(N):
        lam[i], coef[:, i], status[i], s = augmented_select(out["AH"], out["MH"], out["b"][:, i], out["c"][:, i],
                                                            out["beta"][i], out["gamma"][i])
        scores.append(s)
    out["lam"], out["coef"], out["status"], out["scores"] = lam, coef, status, scores
    psi = np.zeros((f.n_nodes, N))                                     # A8
    psi[fr] = Pf @ coef[:-1] + Xf * coef[-1][None, :]
    sgn = np.sign(np.sum(psi[fr] * (level.Mff @ Uf), axis=0))
    sgn[sgn == 0] = 1.0
    out["psi"] = psi * sgn[None, :]
    return out


def assemble_orbitals(level: Level, coef, psihat, U):
    """A8 on its own: psi_i = P phi_{i,H} + theta_{2,i} psi^_i with the sign fixed by (psi_i, P psi_{H,i})_M > 0."""
    fr = level.fine.free
    psi = np.zeros_like(psihat)
    psi[fr] = level.Pf @ coef[:-1] + psihat[fr] * coef[-1][None, :]
    sgn = np.sign(np.sum(psi[fr] * (level.Mff @ U[fr]), axis=0))
    sgn[sgn == 0] = 1.0
    return psi * sgn[None, :]


__all__ = ["Level", "correction_step", "assemble_orbitals", "potential_matrix", "STATUS_OK"]
