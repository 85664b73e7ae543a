"""Tetrahedral P1/P2 Lagrange finite elements, assembled (oracle side).

Sec. 2 of the paper builds V_h, the Lagrange finite element space on a conforming, shape-regular tetrahedral
mesh T_h, with zero Dirichlet data.  The paper uses linear elements; P2 is added for the larger workloads.
Conventions fixed here and checked bit-for-bit against the CUDA side's mesh upload:

* P2 node numbering: the mesh vertices first, then one node per edge, numbered in order of first appearance when
  the tetrahedra are scanned in index order and their local edges in the order (01, 02, 03, 12, 13, 23).
* Boundary nodes: nodes that lie on a boundary face (a face that belongs to exactly one tetrahedron).
  Free DOF = the other nodes, in increasing node index.
* Element colouring: greedy, elements in index order, each taking the smallest colour not used by an
  earlier element that shares a vertex with it (sharing any P2 node implies sharing a vertex).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .quadrature import tet_rule

EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
FACES = [(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)]


def barycentric_grad_ref():
    """Gradients of the four barycentric coordinates with respect to reference coordinates."""
    return np.array([[-1.0, -1.0, -1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])


def basis(order: int, lam: np.ndarray) -> np.ndarray:
    """Lagrange basis values from barycentrics lam [..., 4] -> [..., nloc]."""
    if order == 1:
        return lam.copy()
    vals = [lam[..., a] * (2.0 * lam[..., a] - 1.0) for a in range(4)]
    vals += [4.0 * lam[..., a] * lam[..., b] for (a, b) in EDGES]
    return np.stack(vals, axis=-1)


def basis_grad(order: int, lam: np.ndarray) -> np.ndarray:
    """Reference-coordinate gradients of the basis at barycentrics lam [..., 4] -> [..., nloc, 3]."""
    G = barycentric_grad_ref()
    shp = lam.shape[:-1]
    if order == 1:
        return np.broadcast_to(G, shp + (4, 3)).copy()
    out = []
    for a in range(4):
        out.append((4.0 * lam[..., a] - 1.0)[..., None] * G[a])
    for (a, b) in EDGES:
        out.append(4.0 * (lam[..., b][..., None] * G[a] + lam[..., a][..., None] * G[b]))
    return np.stack(out, axis=-2)


def ref_to_bary(xi: np.ndarray) -> np.ndarray:
    return np.concatenate([1.0 - xi.sum(axis=-1, keepdims=True), xi], axis=-1)


def local_node_bary(order: int) -> np.ndarray:
    """Barycentric coordinates of the element's local nodes [nloc, 4]."""
    I = np.eye(4)
    if order == 1:
        return I
    return np.vstack([I] + [0.5 * (I[a] + I[b]) for (a, b) in EDGES])


class FEMesh:
    """Mesh + DOF map + geometry for one level (oracle side)."""

    def __init__(self, coords, tets, order: int):
        self.coords = np.asarray(coords, dtype=np.float64)
        self.tets = np.asarray(tets, dtype=np.int64)
        self.order = order
        self.nloc = 4 if order == 1 else 10
        nv, E = self.coords.shape[0], self.tets.shape[0]
        self.n_vertices, self.n_elems = nv, E
        elem = np.empty((E, self.nloc), dtype=np.int64)
        elem[:, :4] = self.tets
        nodes = [self.coords]
        if order == 2:
            pa = np.stack([self.tets[:, a] for (a, b) in EDGES], axis=1)
            pb = np.stack([self.tets[:, b] for (a, b) in EDGES], axis=1)
            lo, hi = np.minimum(pa, pb), np.maximum(pa, pb)
            key = (lo * nv + hi).ravel()
            uniq, first, inv = np.unique(key, return_index=True, return_inverse=True)
            rank = np.empty(len(uniq), dtype=np.int64)
            rank[np.argsort(first, kind="stable")] = np.arange(len(uniq))
            elem[:, 4:] = (nv + rank[inv]).reshape(E, 6)
            ea = np.empty(len(uniq), dtype=np.int64)
            eb = np.empty(len(uniq), dtype=np.int64)
            ea[rank] = uniq // nv
            eb[rank] = uniq % nv
            nodes.append(0.5 * (self.coords[ea] + self.coords[eb]))
            self.edges = np.stack([ea, eb], axis=1)
        self.elem = elem
        self.nodes = np.vstack(nodes)
        self.n_nodes = self.nodes.shape[0]
        # boundary faces: faces that occur once
        fv = np.sort(np.stack([self.tets[:, list(f)] for f in FACES], axis=1).reshape(-1, 3), axis=1)
        fkey = (fv[:, 0] * nv + fv[:, 1]) * nv + fv[:, 2]
        u, cnt = np.unique(fkey, return_counts=True)
        bkeys = u[cnt == 1]
        bfaces = np.stack([bkeys // (nv * nv), (bkeys // nv) % nv, bkeys % nv], axis=1)
        bnd = np.zeros(self.n_nodes, dtype=bool)
        bnd[bfaces.ravel()] = True
        if order == 2:
            ekey = self.edges[:, 0] * nv + self.edges[:, 1]
            bedge = np.concatenate([np.minimum(bfaces[:, a], bfaces[:, b]) * nv + np.maximum(bfaces[:, a], bfaces[:, b])
                                    for (a, b) in [(0, 1), (0, 2), (1, 2)]])
            bnd[nv + np.nonzero(np.isin(ekey, bedge))[0]] = True
        self.boundary = bnd
        self.free = np.nonzero(~bnd)[0]
        self.n_free = len(self.free)
        # affine geometry x = x0 + J xi
        x = self.coords[self.tets]
        self.J = np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=2)
        self.det = np.linalg.det(self.J)
        self.Jinv = np.linalg.inv(self.J)
        self.x0 = x[:, 0]

    # ------------------------------------------------------------------ colouring
    def colouring(self) -> np.ndarray:
        """Greedy vertex-conflict colouring, elements in index order."""
        E, nv = self.n_elems, self.n_vertices
        order = np.argsort(self.tets.ravel(), kind="stable")
        vstart = np.searchsorted(self.tets.ravel()[order], np.arange(nv + 1))
        v2e = order // 4
        colour = np.full(E, -1, dtype=np.int64)
        for e in range(E):
            used = set()
            for v in self.tets[e]:
                for f in v2e[vstart[v]:vstart[v + 1]]:
                    c = colour[f]
                    if c >= 0:
                        used.add(c)
            c = 0
            while c in used:
                c += 1
            colour[e] = c
        return colour

    # ------------------------------------------------------------------ quadrature
    def quad(self, n: int = 3):
        """Physical quadrature points [E, Q, 3], weights*|det J| [E, Q], basis [Q, nloc], ref gradients [Q, nloc, 3]."""
        xi, w = tet_rule(n)
        lam = ref_to_bary(xi)
        phi = basis(self.order, lam)
        dphi = basis_grad(self.order, lam)
        xq = self.x0[:, None, :] + np.einsum("eij,qj->eqi", self.J, xi)
        wq = np.abs(self.det)[:, None] * w[None, :]
        return xq, wq, phi, dphi

    def element_stiffness(self) -> np.ndarray:
        """K_e[a,b] = int_e grad phi_a . grad phi_b  [E, nloc, nloc]."""
        xi, w = tet_rule(3)
        dphi = basis_grad(self.order, ref_to_bary(xi))
        Ke = np.zeros((self.n_elems, self.nloc, self.nloc))
        for q in range(len(w)):
            G = np.einsum("aj,ejk->eak", dphi[q], self.Jinv)  # physical gradients (row vectors)
            Ke += w[q] * np.einsum("eak,ebk->eab", G, G)
        return Ke * np.abs(self.det)[:, None, None]

    def element_mass(self, fq=None) -> np.ndarray:
        """M_e[a,b] = int_e f phi_a phi_b for f given at the quadrature points [E, Q] (f = 1 if None)."""
        xq, wq, phi, _ = self.quad()
        ww = wq if fq is None else wq * fq
        return np.einsum("eq,qa,qb->eab", ww, phi, phi)

    def assemble(self, Me) -> sp.csr_matrix:
        """Global matrix (all nodes) from element matrices [E, nloc, nloc]."""
        r = np.repeat(self.elem, self.nloc, axis=1).ravel()
        c = np.tile(self.elem, (1, self.nloc)).ravel()
        return sp.coo_matrix((Me.ravel(), (r, c)), shape=(self.n_nodes, self.n_nodes)).tocsr()

    def assemble_vector(self, be) -> np.ndarray:
        """Global vector(s) from element vectors [E, nloc] or [E, nloc, k]."""
        out = np.zeros((self.n_nodes,) + be.shape[2:])
        np.add.at(out, self.elem.ravel(), be.reshape((-1,) + be.shape[2:]))
        return out

    def eval_at_quad(self, u: np.ndarray) -> np.ndarray:
        """FE function(s) with nodal values u [n_nodes] or [n_nodes, k] at quadrature points -> [E, Q(, k)]."""
        _, _, phi, _ = self.quad()
        return np.einsum("qa,ea...->eq...", phi, u[self.elem])


def coulomb(xq: np.ndarray, Z, R, rmin: float = 1e-8) -> np.ndarray:
    """V_ext(x) = -sum_k Z_k / |x - R_k| (Sec. 2), with |x - R_k| clamped below at rmin."""
    V = np.zeros(xq.shape[:-1])
    for z, r in zip(Z, R):
        d = np.sqrt(np.sum((xq - r) ** 2, axis=-1))
        V -= z / np.maximum(d, rmin)
    return V


def interpolation(coarse: FEMesh, fine: FEMesh, parent) -> sp.csr_matrix:
    """Coarse-to-fine prolongation P [fine n_nodes, coarse n_nodes]: the coarse function evaluated at the fine
    nodes, exact because V_H is a subspace of V_h on nested meshes (Sec. 2, V_H subset V_h)."""
    parent = np.asarray(parent, dtype=np.int64)
    flat = fine.elem.ravel()
    _, first = np.unique(flat, return_index=True)
    e = first // fine.nloc
    node = flat[first]
    T = parent[e]
    x = fine.nodes[node]
    s = np.einsum("nij,nj->ni", coarse.Jinv[T], x - coarse.x0[T])
    vals = basis(coarse.order, ref_to_bary(s))
    rows = np.repeat(node, coarse.nloc)
    cols = coarse.elem[T].ravel()
    v = vals.ravel()
    keep = np.abs(v) > 1e-12
    return sp.csr_matrix((v[keep], (rows[keep], cols[keep])), shape=(fine.n_nodes, coarse.n_nodes))
