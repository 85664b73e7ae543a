"""The paper's own correction step with its inner iteration (oracle side): Algorithm 1, steps 5-7, in the form the
paper writes them, with the nonlinear eigenproblem of step 7 solved by the SCF iteration of Algorithm 2, either by
assembling every inner iteration's matrices on the fine mesh (`split=False`, the definition) or with the
precomputations of Algorithm 3 (`split=True`), after which an inner iteration touches only coarse-sized data.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Step 5 (Eq. (Aux_Linear_Problem)): a(phi^_i, g) + (w^ phi^_i, g) + (V_xc(rho^l) phi^_i, g) = lambda_i (phi_i, g), with
  the frozen Hartree potential w^ and exchange-correlation potential of the step's input orbitals on the left; solved
  with the shift sigma (an exact eigenpair is a fixed point for any sigma, as for the right-hand-side form).
Step 6 (Eq. (W_h_equation)): (grad w~, grad v) = 4 pi sum_i f_i (phi~_i^2, v), multipole boundary values.
Step 7 (Eq. (Nonlinear_Eig_Hh_Full)), Algorithm 2: for s = 1, 2, ...
  (a) for every orbital the eigenproblem in S_i = V_H + span{phi~_i} with the Hamiltonian of the current Hartree
      potential w and the frozen V_xc, selecting the eigenvector with the largest component along phi~_i;
  (b) the Hartree potential in W = V_H + span{w~} from the density of the new orbitals;
  (c) stop when the orbitals no longer change.
Readings (the paper is silent or garbled here):
  * The density of (b) is sum_i f_i (phi_{i,H} + theta_{2,i} phi~_i)^2; the paper's expansion of the square drops the
    theta_{2,i}^2 of its last term (Eqs. (fH), (gdef)), a typo.
  * w~ carries the Dirichlet values of the multipole expansion, so it is no test function of the Hartree equation.
    The boundary values stay fixed during the inner iteration (Remark after Algorithm 3): w~ = w_b + w~0 with w_b the
    boundary values (zero at interior nodes) and w~0 zero on the boundary; the inner Hartree potential is
    w = w_b + w_H + theta_1 w~0, Galerkin in V_H + span{w~0}.  It reproduces w~ when the density is that of step 6.
    When w~0 already lies in V_H (its Schur complement zeta - d^T C_H^-1 d at most 1e-12 zeta) the extra direction is
    dropped (theta_1 = 0), as the augmented eigenproblem drops a correction that lies in V_H.
  * Convergence of (c): the largest change of any orbital's coefficients (phi_{i,H}, theta_{2,i}) in the max norm.
  * The plain iteration (a)-(b) oscillates on molecules with near-degenerate orbitals (the orbitals trade places and
    the Hartree potential sloshes); the paper gives no mixing rule.  Reading: linear mixing of the inner Hartree
    coefficients, (w_H, theta_1) <- (1 - mix) old + mix new, mix = 0.5 (the fixed point does not depend on it).
  * All integrals are fine-mesh quadratures (the 27-point rule).  Algorithm 3's coarse-space terms that are quadratic
    or cubic in coarse functions ((w_H psi_k, psi_j), (phi_H^2, psi_j)) use, per fine element, the tensor of its
    parent's coarse basis functions (psi_a psi_b, psi_c) on that rule, so an inner iteration costs O(N_H) and equals
    the fine-mesh assembly.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .linalg import augmented_select, pcg
from .poisson import density_at_quad, hartree
from .xc import v_xc


def _mass_with(f, fq):
    """M_{f} (all nodes) for a function given at the quadrature points."""
    return f.assemble(f.element_mass(fq))


def _coarse_local_basis(level):
    """The coarse basis functions of each fine element's parent, at the fine element's quadrature points:
    Bq [E_fine, Q, n_loc], and the coarse free DOF of the parent's local nodes, dof [E_fine, n_loc] (-1 on the
    boundary)."""
    from .fem import basis, ref_to_bary
    f, C = level.fine, level.coarse
    xq, _, _, _ = f.quad()
    T = level.parent
    s = np.einsum("eij,eqj->eqi", C.Jinv[T], xq - C.x0[T][:, None, :])
    Bq = basis(C.order, ref_to_bary(s))
    free_of = np.full(C.n_nodes, -1, dtype=np.int64)
    free_of[C.free] = np.arange(C.n_free)
    return Bq, free_of[C.elem[T]]


def _scatter_matrix(local, dof, n):
    """Dense [n, n] from element blocks local [E, a, b] with global indices dof [E, a] (-1 dropped)."""
    E, na = dof.shape
    r = np.repeat(dof, na, axis=1).ravel()
    c = np.tile(dof, (1, na)).ravel()
    keep = (r >= 0) & (c >= 0)
    return sp.coo_matrix((local.ravel()[keep], (r[keep], c[keep])), shape=(n, n)).toarray()


def _scatter_vector(local, dof, n):
    keep = dof.ravel() >= 0
    out = np.zeros(n)
    np.add.at(out, dof.ravel()[keep], local.ravel()[keep])
    return out


def correction_paper_form(level, U, lam, occ, sigma, w_prev, xc, tol=1e-13):
    """Steps 5 and 6: the corrections phi~_i and the Hartree potential w~ of their density.  U [n_nodes, N] the
    step's input orbitals (fine nodal values), w_prev the Hartree potential of the previous outer step."""
    f = level.fine
    fr = f.free
    rho_l = density_at_quad(f, U, occ)
    vxc = v_xc(rho_l, xc)
    Mw = _mass_with(f, f.eval_at_quad(w_prev) + vxc)[fr][:, fr]
    A = (0.5 * level.Kff + level.MVff + Mw + sigma * level.Mff).tocsr()
    B = (level.Mff @ U[fr]) * (np.asarray(lam, dtype=np.float64) + sigma)[None, :]
    X, iters, res = pcg(A, B, X0=U[fr], tol=tol)
    phit = np.zeros_like(U)
    phit[fr] = X
    rho_t = density_at_quad(f, phit, occ)
    wt, info = hartree(f, rho_t, bc="multipole", tol=tol, K=level.K)
    return phit, wt, vxc, dict(cg_iters=iters, cg_res=res, poisson=info)


def _select_all(AH, MH, b, c, beta, gamma):
    N = b.shape[1]
    lam = np.zeros(N)
    X = np.zeros((AH.shape[0] + 1, N))
    for i in range(N):
        lam[i], X[:, i], _, _ = augmented_select(AH, MH, b[:, i], c[:, i], beta[i], gamma[i])
    return lam, X


def inner_iteration(level, phit, wt, vxc, occ, tol=1e-10, max_inner=200, split=True, mix=0.5):
    """Step 7 by Algorithm 2, from w = w~ (w_H = 0, theta_1 = 1).  Returns dict(lam, X [N_H+1, N], wH, theta1,
    psi [n_nodes, N] (the output orbitals P phi_H + theta_2 phi~, sign with (psi_i, phi~_i)_M >= 0), w, iters)."""
    f, C = level.fine, level.coarse
    fr, bnd = f.free, f.boundary
    Pf = level.Pf                                    # [n_free fine, N_H]
    NH, N = Pf.shape[1], phit.shape[1]
    occ = np.asarray(occ, dtype=np.float64)
    wb = np.where(bnd, wt, 0.0)
    w0 = np.where(bnd, 0.0, wt)
    Kff = level.Kff
    Mff = level.Mff
    Ptf = phit[fr]
    # fixed blocks of the augmented eigenproblems and of the Hartree system in W
    MH = (Pf.T @ (Mff @ Pf)).toarray()
    c = Pf.T @ (Mff @ Ptf)
    gamma = np.sum(Ptf * (Mff @ Ptf), axis=0)
    CH = (Pf.T @ (Kff @ Pf)).toarray()
    d = Pf.T @ (Kff @ w0[fr])
    zeta = w0[fr] @ (Kff @ w0[fr])
    KIB = level.K[fr][:, np.nonzero(bnd)[0]]
    lift_H = Pf.T @ (KIB @ wb[bnd])                  # (grad w_b, grad psi_j)
    lift_0 = w0[fr] @ (KIB @ wb[bnd])                # (grad w_b, grad w~0)
    # w~0 already in V_H (its Schur complement vanishes, e.g. P = I): the extra direction is dropped, theta_1 = 0
    CHc = sla.cho_factor(CH)
    schur = zeta - d @ sla.cho_solve(CHc, d)
    w_in_VH = not (schur > 1e-12 * zeta)
    Wchol = None if w_in_VH else sla.cho_factor(np.block([[CH, d[:, None]], [d[None, :], np.array([[zeta]])]]))
    wq0, wqb = f.eval_at_quad(w0), f.eval_at_quad(wb)
    xq, wquad, _, _ = f.quad()
    if split:
        # Algorithm 3, step 1: everything that stays fixed during the inner iteration, on the fine mesh
        H1 = (0.5 * Kff + level.MVff + _mass_with(f, vxc + wqb)[fr][:, fr]).tocsr()   # static part, w_b included
        M3 = _mass_with(f, wq0)[fr][:, fr]                                               # the w~0 term
        A1 = (Pf.T @ (H1 @ Pf)).toarray()
        A3 = (Pf.T @ (M3 @ Pf)).toarray()                                               # = G of Eq. (FG)
        b1 = Pf.T @ (H1 @ Ptf)
        b3 = Pf.T @ (M3 @ Ptf)                                                          # = F_i of Eq. (FG)
        beta1 = np.sum(Ptf * (H1 @ Ptf), axis=0)
        beta3 = np.sum(Ptf * (M3 @ Ptf), axis=0)
        phq = f.eval_at_quad(phit)                                                       # [E, Q, N]
        Bq, dof = _coarse_local_basis(level)                                             # [E, Q, n_loc]
        # Eq. (Ah4def): (phi~_i psi_k, psi_j); Eq. (rhsdef): (phi~_i^2, psi_j); (phi~_i^2, w~0)
        Ah4 = [_scatter_matrix(np.einsum("eq,eqa,eqb->eab", wquad * phq[:, :, i], Bq, Bq), dof, NH) for i in range(N)]
        rhs = np.stack([_scatter_vector(np.einsum("eq,eqa->ea", wquad * phq[:, :, i] ** 2, Bq), dof, NH)
                        for i in range(N)], axis=1)
        g3 = np.einsum("eq,eqi->i", wquad * wq0, phq * phq)
        # the coarse basis tensor (psi_a psi_b, psi_c) of every fine element, for the terms quadratic and cubic in
        # coarse functions (A_H2 = (w_H psi_k, psi_j), (phi_H^2, psi_j))
        T = np.einsum("eq,eqa,eqb,eqc->eabc", wquad, Bq, Bq, Bq)

        def coarse_vals(v):  # a coarse free-DOF vector at each fine element's parent nodes
            return np.where(dof >= 0, v[np.maximum(dof, 0)], 0.0)
    wH, th1 = np.zeros(NH), 1.0
    Xprev = None
    lam = None
    for it in range(1, max_inner + 1):
        # (a) the per-orbital augmented eigenproblems with the current Hartree potential
        if split:
            AH = A1 + _scatter_matrix(np.einsum("eabc,ec->eab", T, coarse_vals(wH)), dof, NH) + th1 * A3
            b = b1 + np.stack([Ah4[i] @ wH for i in range(N)], axis=1) + th1 * b3
            beta = beta1 + rhs.T @ wH + th1 * beta3
        else:
            w = wb + level.P[:, C.free] @ wH + th1 * w0
            H = (0.5 * Kff + level.MVff + _mass_with(f, f.eval_at_quad(w) + vxc)[fr][:, fr]).tocsr()
            AH = (Pf.T @ (H @ Pf)).toarray()
            b = Pf.T @ (H @ Ptf)
            beta = np.sum(Ptf * (H @ Ptf), axis=0)
        lam, X = _select_all(AH, MH, b, c, beta, gamma)
        # (b) the Hartree potential in W from the density of the new orbitals
        ph, th2 = X[:-1], X[-1]
        if split:
            fH = np.zeros(NH)
            g = 0.0
            for i in range(N):
                pc = coarse_vals(ph[:, i])
                fH += occ[i] * (_scatter_vector(np.einsum("eabc,eb,ec->ea", T, pc, pc), dof, NH)
                                + 2.0 * th2[i] * (Ah4[i] @ ph[:, i]) + th2[i] ** 2 * rhs[:, i])
                g += occ[i] * (ph[:, i] @ (A3 @ ph[:, i]) + 2.0 * th2[i] * (b3[:, i] @ ph[:, i]) + th2[i] ** 2 * g3[i])
        else:
            orb = np.zeros((f.n_nodes, N))
            orb[fr] = Pf @ ph + Ptf * th2[None, :]
            rho = density_at_quad(f, orb, occ)
            load = f.assemble_vector(np.einsum("eq,qa->ea", wquad * rho, f.quad()[2]))
            fH = Pf.T @ load[fr]
            g = np.sum(wquad * rho * wq0)
        if w_in_VH:
            sol = np.concatenate([sla.cho_solve(CHc, 4.0 * np.pi * fH - lift_H), [0.0]])
        else:
            sol = sla.cho_solve(Wchol, np.concatenate([4.0 * np.pi * fH - lift_H, [4.0 * np.pi * g - lift_0]]))
        wH, th1 = (1.0 - mix) * wH + mix * sol[:-1], (1.0 - mix) * th1 + mix * sol[-1]
        # (c)
        done = Xprev is not None and np.abs(X - Xprev).max() < tol
        Xprev = X
        if done:
            break
    psi = np.zeros((f.n_nodes, N))
    psi[fr] = Pf @ Xprev[:-1] + Ptf * Xprev[-1][None, :]
    w = wb + level.P[:, C.free] @ wH + th1 * w0
    return dict(lam=lam, X=Xprev, wH=wH, theta1=th1, psi=psi, w=w, iters=it)


def paper_step(level, U, lam, occ, sigma, w_prev, xc, tol=1e-13, inner_tol=1e-10, max_inner=200, split=True,
               mix=0.5):
    """Algorithm 1, steps 5-7, in the paper's form with Algorithm 2 (split=False) or Algorithm 3 (split=True)."""
    phit, wt, vxc, info = correction_paper_form(level, U, lam, occ, sigma, w_prev, xc, tol=tol)
    out = inner_iteration(level, phit, wt, vxc, occ, tol=inner_tol, max_inner=max_inner, split=split, mix=mix)
    out.update(phit=phit, wt=wt, vxc=vxc, info=info)
    return out


def hartree_in_W(level, wt, rhoq):
    """The Galerkin Hartree potential in w_b + V_H + span{w~0} for a density rho given at the fine quadrature points
    (step (b) of Algorithm 2 with the lift reading): returns (w_H, theta_1, w)."""
    f, C = level.fine, level.coarse
    fr, bnd = f.free, f.boundary
    Pf, Kff = level.Pf, level.Kff
    wb = np.where(bnd, wt, 0.0)
    w0 = np.where(bnd, 0.0, wt)
    KIB = level.K[fr][:, np.nonzero(bnd)[0]]
    CH = (Pf.T @ (Kff @ Pf)).toarray()
    d = Pf.T @ (Kff @ w0[fr])
    Wsys = np.block([[CH, d[:, None]], [d[None, :], np.array([[w0[fr] @ (Kff @ w0[fr])]])]])
    _, wquad, phi, _ = f.quad()
    load = f.assemble_vector(np.einsum("eq,qa->ea", wquad * rhoq, phi))
    rhs = np.concatenate([4.0 * np.pi * (Pf.T @ load[fr]) - Pf.T @ (KIB @ wb[bnd]),
                          [4.0 * np.pi * np.sum(wquad * rhoq * f.eval_at_quad(w0)) - w0[fr] @ (KIB @ wb[bnd])]])
    sol = np.linalg.solve(Wsys, rhs)
    return sol[:-1], sol[-1], wb + level.P[:, C.free] @ sol[:-1] + sol[-1] * w0
