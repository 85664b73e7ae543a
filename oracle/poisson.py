"""Hartree potential by a Poisson solve on the fine mesh (oracle side).

Sec. 2: -Delta V_Har = 4 pi rho with a Dirichlet condition; Eq. (Mixed_Eigenvalue_Problem_Discrete) uses the
weak form (grad w, grad v) = 4 pi (rho, v) for all v in V_h, and Eq. (W_h_equation) solves it on the fine mesh.
The boundary values are those of the free-space potential int rho(y)/|x-y| dy (definition of V_Gamma); the paper
takes them from a multipole expansion (Remark after Algorithm 3) without stating its order.  Reading: expansion
about the origin through the quadrupole (l <= 2), moments by the fine-mesh quadrature of rho.
"""
from __future__ import annotations

import numpy as np

from .fem import FEMesh
from .linalg import pcg


def density_at_quad(mesh: FEMesh, U: np.ndarray, occ) -> np.ndarray:
    """rho(x_q) = sum_i f_i u_i(x_q)^2 for nodal values U [n_nodes, N]  ->  [E, Q]."""
    uq = mesh.eval_at_quad(U)
    return np.einsum("eqn,n->eq", uq * uq, np.asarray(occ, dtype=np.float64))


def multipole_moments(mesh: FEMesh, rhoq: np.ndarray):
    """Total charge, dipole and traceless quadrupole Q_ij = int rho (3 y_i y_j - |y|^2 delta_ij)."""
    xq, wq, _, _ = mesh.quad()
    w = wq * rhoq
    q0 = w.sum()
    p = np.einsum("eq,eqi->i", w, xq)
    r2 = np.sum(xq * xq, axis=-1)
    Q = 3.0 * np.einsum("eq,eqi,eqj->ij", w, xq, xq) - np.eye(3) * np.sum(w * r2)
    return q0, p, Q


def multipole_potential(x: np.ndarray, q0, p, Q) -> np.ndarray:
    """q0/r + p.x/r^3 + (1/2) x^T Q x / r^5 at points x [n, 3]."""
    r2 = np.sum(x * x, axis=1)
    r = np.sqrt(r2)
    return q0 / r + (x @ p) / (r2 * r) + 0.5 * np.einsum("ni,ij,nj->n", x, Q, x) / (r2 * r2 * r)


def direct_potential(x: np.ndarray, mesh: FEMesh, rhoq: np.ndarray) -> np.ndarray:
    """The definition: sum_q rho(y_q) w_q / |x - y_q| (for small meshes in tests)."""
    xq, wq, _, _ = mesh.quad()
    y = xq.reshape(-1, 3)
    w = (wq * rhoq).ravel()
    out = np.empty(len(x))
    for i, xi in enumerate(x):
        out[i] = np.sum(w / np.sqrt(np.sum((y - xi) ** 2, axis=1)))
    return out


def hartree(mesh: FEMesh, rhoq: np.ndarray, bc: str = "multipole", tol: float = 1e-13, K=None):
    """Solve (grad w, grad v) = 4 pi (rho, v) for free v, w = g on the boundary nodes.
    bc: 'multipole' (boundary values from the l <= 2 expansion) or 'zero'.  Returns (w [n_nodes], info)."""
    if K is None:
        K = mesh.assemble(mesh.element_stiffness())
    _, wq, phi, _ = mesh.quad()
    F = mesh.assemble_vector(np.einsum("eq,qa->ea", wq * rhoq, phi))
    w = np.zeros(mesh.n_nodes)
    bnd = np.nonzero(mesh.boundary)[0]
    if bc == "multipole":
        w[bnd] = multipole_potential(mesh.nodes[bnd], *multipole_moments(mesh, rhoq))
    elif bc != "zero":
        raise ValueError(bc)
    fr = mesh.free
    rhs = 4.0 * np.pi * F[fr] - K[fr][:, bnd] @ w[bnd]
    wf, it, res = pcg(K[fr][:, fr], rhs, tol=tol)
    w[fr] = wf
    return w, dict(iters=int(it[0]), rel_res=float(res[0]))
