"""The outer AFEM loop's Estimate and Mark steps (Sec. 2), oracle side: the residual a posteriori error indicator
of the eigenpair approximation and Dorfler's marking.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

For the approximation (Lambda_h, Phi_h) of the occupied orbitals, with H = -1/2 Laplacian + V the Kohn-Sham
Hamiltonian (V = V_ext + w + V_xc at the density of Phi_h):
  element residual  R_T = (H phi_i - lambda_i phi_i)_i                      in T,
  jump residual     J_e = (1/2 grad phi_i|T+ . nu+ + 1/2 grad phi_i|T- . nu-)_i  on an interior face e = T+ ^ T-,
  indicator         eta^2(T) = h_T^2 ||R_T||_{0,T}^2 + sum over the interior faces e of T of h_e ||J_e||_{0,e}^2,
and Dorfler's strategy marks a set M of elements with sum_M eta^2 >= theta sum_T eta^2.
Readings (the paper does not fix them):
  * The norm of an orbital vector is the l2 sum over orbitals (no occupation weights).
  * h_T and h_e are the longest edges of the element and of the face.
  * ||R_T||^2 by the 27-point element rule; ||J_e||^2 by the 3-point rule at the face's edge midpoints, exact here
    because J_e is linear on a face for P2 (constant for P1), so J_e^2 is at most quadratic.
  * M is the smallest such set: elements in order of decreasing eta^2 (ties: lower element index first) until the
    sum reaches theta times the total.
"""
from __future__ import annotations

import numpy as np

from .fem import FACES, basis, basis_grad, ref_to_bary

_FACE_EDGES = [(0, 1), (0, 2), (1, 2)]   # the edges of a face, by the face's local vertex positions


def _bary_grads(f):
    """Physical gradients of the four barycentric coordinates of every element [E, 4, 3]."""
    G = np.zeros((f.n_elems, 4, 3))
    G[:, 1:, :] = f.Jinv                      # lambda_k = xi_k, xi = J^-1 (x - x0)
    G[:, 0, :] = -f.Jinv.sum(axis=1)
    return G


def _laplacians(f):
    """Laplacian of every basis function on every element [E, nloc] (constant per element)."""
    if f.order == 1:
        return np.zeros((f.n_elems, 4))
    G = _bary_grads(f)
    dots = np.einsum("eai,ebi->eab", G, G)
    vals = [4.0 * dots[:, a, a] for a in range(4)]                 # lambda_a (2 lambda_a - 1)
    vals += [8.0 * dots[:, a, b] for (a, b) in [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]]  # 4 la lb
    return np.stack(vals, axis=1)


def _longest_edge(P):
    """Longest edge of each simplex with vertices P [E, k, 3]."""
    k = P.shape[1]
    d = [np.linalg.norm(P[:, a] - P[:, b], axis=1) for a in range(k) for b in range(a + 1, k)]
    return np.max(np.stack(d, axis=1), axis=1)


def interior_faces(f):
    """Interior faces as rows (T+, face slot in T+, T-, face slot in T-), T+ < T-; face slot k is the face opposite
    local vertex k."""
    E = f.n_elems
    fv = np.sort(np.stack([f.tets[:, list(F)] for F in FACES], axis=1), axis=2)   # [E, 4, 3]
    nv = f.n_vertices
    key = ((fv[..., 0] * nv + fv[..., 1]) * nv + fv[..., 2]).ravel()
    order = np.argsort(key, kind="stable")
    ks = key[order]
    same = np.nonzero(ks[1:] == ks[:-1])[0]
    a, b = order[same], order[same + 1]
    rows = np.stack([a // 4, a % 4, b // 4, b % 4], axis=1)
    swap = rows[:, 0] > rows[:, 2]
    rows[swap] = rows[swap][:, [2, 3, 0, 1]]
    return rows[np.argsort(rows[:, 0] * 4 + rows[:, 1], kind="stable")]


def _grad_at(f, e, x, u):
    """grad of the FE function(s) u [n_nodes, N] on elements e [F] at physical points x [F, 3] -> [F, 3, N]."""
    s = np.einsum("fij,fj->fi", f.Jinv[e], x - f.x0[e])
    lam = ref_to_bary(s)
    dref = basis_grad(f.order, lam)                        # [F, nloc, 3] reference gradients
    dphys = np.einsum("fak,fkj->faj", dref, f.Jinv[e])     # grad_x phi_a = J^-T grad_xi phi_a (row form)
    return np.einsum("faj,fan->fjn", dphys, u[f.elem[e]])


def indicators(f, psi, lam, Vq):
    """eta^2 [E] for orbitals psi [n_nodes, N], eigenvalues lam [N], the potential V at the quadrature points
    Vq [E, Q] (V_ext + w + V_xc)."""
    psi = np.asarray(psi, dtype=np.float64)
    if psi.ndim == 1:
        psi = psi[:, None]
    lam = np.asarray(lam, dtype=np.float64)
    xq, wq, phi, _ = f.quad()
    uq = np.einsum("qa,ean->eqn", phi, psi[f.elem])                       # orbitals at the points
    lap = np.einsum("ea,ean->en", _laplacians(f), psi[f.elem])            # Laplacians (constant per element)
    R = -0.5 * lap[:, None, :] + (Vq[:, :, None] - lam[None, None, :]) * uq
    hT = _longest_edge(f.coords[f.tets])
    eta2 = hT ** 2 * np.einsum("eq,eqn->e", wq, R * R)
    rows = interior_faces(f)
    if rows.size:
        ep, kp, em, km = rows.T
        V = f.coords[f.tets[ep]]                                            # [F, 4, 3] vertices of T+
        fidx = np.array(FACES)[kp]                                          # [F, 3] local vertices of the face
        fvx = np.take_along_axis(V, fidx[:, :, None], axis=1)               # [F, 3, 3]
        nrm = np.cross(fvx[:, 1] - fvx[:, 0], fvx[:, 2] - fvx[:, 0])
        area = 0.5 * np.linalg.norm(nrm, axis=1)
        nu = nrm / (2.0 * area)[:, None]
        opp = V[np.arange(len(ep)), kp]                                     # the vertex of T+ off the face
        flip = np.einsum("fi,fi->f", nu, fvx[:, 0] - opp) < 0               # outward from T+
        nu[flip] = -nu[flip]
        he = _longest_edge(fvx)
        jj = np.zeros(len(ep))
        for (a, b) in _FACE_EDGES:
            x = 0.5 * (fvx[:, a] + fvx[:, b])
            gp = _grad_at(f, ep, x, psi)
            gm = _grad_at(f, em, x, psi)
            J = 0.5 * np.einsum("fj,fjn->fn", nu, gp - gm)                  # nu- = -nu+
            jj += np.sum(J * J, axis=1) * area / 3.0
        val = he * jj
        eta2 += np.bincount(ep, weights=val, minlength=f.n_elems) + np.bincount(em, weights=val, minlength=f.n_elems)
    return eta2


def ks_potential(level, psi, occ, w, xc):
    """V = V_ext + w + V_xc(rho(psi)) at the fine quadrature points [E, Q]."""
    from .fem import coulomb
    from .poisson import density_at_quad
    from .xc import v_xc
    f = level.fine
    xq, _, _, _ = f.quad()
    return coulomb(xq, level.Z, level.R) + f.eval_at_quad(w) + v_xc(density_at_quad(f, psi, occ), xc)


def dorfler(eta2, theta):
    """Dorfler's marking: boolean [E], the smallest set in order of decreasing eta^2 (ties to the lower index) whose
    indicators sum to at least theta times the total."""
    eta2 = np.asarray(eta2, dtype=np.float64)
    order = np.lexsort((np.arange(eta2.size), -eta2))
    c = np.cumsum(eta2[order])
    k = int(np.searchsorted(c, theta * c[-1], side="left")) + 1 if eta2.size else 0
    mark = np.zeros(eta2.size, dtype=bool)
    mark[order[:min(k, eta2.size)]] = True
    return mark
