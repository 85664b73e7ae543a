"""Pins of the oracle's quadrature, meshes and finite elements against closed forms (no GPU)."""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.fem import FEMesh, interpolation
from oracle.quadrature import gauss_jacobi, gauss_jacobi01, tet_rule
from paper_2103_02824_gb300 import synth


def test_gauss_legendre_matches_numpy():
    for n in range(1, 7):
        x, w = gauss_jacobi(n, 0.0, 0.0)
        xr, wr = np.polynomial.legendre.leggauss(n)
        assert np.allclose(np.sort(x), xr, atol=1e-14) and np.allclose(w[np.argsort(x)], wr, atol=1e-14)


@pytest.mark.parametrize("a", [0.0, 1.0, 2.0])
def test_gauss_jacobi01_moments(a):
    # int_0^1 x^k (1-x)^a dx = B(k+1, a+1), exact up to degree 2n-1
    n = 3
    x, w = gauss_jacobi01(n, a)
    for k in range(2 * n):
        exact = math.gamma(k + 1) * math.gamma(a + 1) / math.gamma(k + a + 2)
        assert abs(np.sum(w * x ** k) - exact) < 1e-15 * max(1.0, exact) * 10


def test_tet_rule_exact_to_degree_5_and_not_6():
    pts, w = tet_rule(3)
    assert len(w) == 27 and abs(w.sum() - 1.0 / 6.0) < 1e-16 * 10
    assert np.all(pts >= 0) and np.all(pts.sum(axis=1) <= 1)
    for a in range(6):
        for b in range(6 - a):
            for c in range(6 - a - b):
                exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 3)
                got = np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
                assert abs(got - exact) < 1e-15, (a, b, c)
    exact6 = math.factorial(6) / math.factorial(9)
    assert abs(np.sum(w * pts[:, 0] ** 6) - exact6) > 1e-8


@pytest.mark.parametrize("n,order", [(2, 1), (3, 2), (4, 2)])
def test_mesh_counts_and_geometry(n, order):
    L = 1.5
    c, t = synth.cube_mesh(n, L)
    assert c.shape == ((n + 1) ** 3, 3) and t.shape == (6 * n ** 3, 4)
    m = FEMesh(c, t, order)
    assert np.all(m.det > 0)
    assert abs(np.sum(m.det) / 6.0 - (2 * L) ** 3) < 1e-12
    if order == 2:
        assert m.n_nodes == (2 * n + 1) ** 3
        # P2 nodes of a Kuhn mesh are exactly the points of the half-step grid
        g = np.round((m.nodes + L) / (L / n)).astype(int)
        assert len({tuple(r) for r in g}) == m.n_nodes and g.min() == 0 and g.max() == 2 * n
        assert m.n_free == (2 * n - 1) ** 3
    else:
        assert m.n_free == (n - 1) ** 3
    assert np.all(np.isclose(np.abs(m.nodes[m.boundary]).max(axis=1), L))
    assert np.all(np.abs(m.nodes[~m.boundary]).max(axis=1) < L - 1e-12)


def test_colouring_valid_and_greedy():
    c, t = synth.cube_mesh(3, 1.0)
    m = FEMesh(c, t, 2)
    col = m.colouring()
    E = m.n_elems
    sets = [set(tt) for tt in t.tolist()]
    for e in range(E):
        nb = [f for f in range(E) if f != e and sets[e] & sets[f]]
        assert all(col[f] != col[e] for f in nb)
        earlier = {col[f] for f in nb if f < e}
        assert col[e] == min(set(range(len(earlier) + 1)) - earlier)
    assert col.max() + 1 >= 24  # 24 tetrahedra meet at an interior vertex of a Kuhn mesh


def test_parent_map_nested():
    cc, ct, fc, ft, par = synth.nested_cube_meshes(2, 2, 1.0)
    C, F = FEMesh(cc, ct, 1), FEMesh(fc, ft, 1)
    assert np.all(np.bincount(par, minlength=C.n_elems) == 64)
    s = np.einsum("eij,ekj->eki", C.Jinv[par], fc[ft] - C.x0[par][:, None, :])
    lam = np.concatenate([1 - s.sum(axis=2, keepdims=True), s], axis=2)
    assert lam.min() > -1e-12 and lam.max() < 1 + 1e-12
    vol = np.bincount(par, weights=F.det, minlength=C.n_elems)
    assert np.allclose(vol, C.det, rtol=1e-13)


def _quad_poly(x):
    return 1.0 + 0.5 * x[:, 0] - 0.25 * x[:, 1] + 0.3 * x[:, 0] * x[:, 2] - 0.2 * x[:, 1] ** 2 + 0.1 * x[:, 2] ** 2


@pytest.mark.parametrize("order", [1, 2])
def test_patch_tests(order):
    L = 1.0
    c, t = synth.cube_mesh(3, L)
    m = FEMesh(c, t, order)
    K = m.assemble(m.element_stiffness())
    M = m.assemble(m.element_mass())
    one = np.ones(m.n_nodes)
    assert np.abs(K @ one).max() < 1e-12                      # K annihilates constants
    assert abs(one @ (M @ one) - (2 * L) ** 3) < 1e-12         # 1^T M 1 = |Omega|
    assert abs(K - K.T).max() < 1e-14 and abs(M - M.T).max() < 1e-16 * 100
    Me = m.element_mass()
    rows = Me.sum(axis=2) / m.det[:, None]                     # int_e phi_a / |det J|
    if order == 1:
        assert np.allclose(rows, 1.0 / 24.0, atol=1e-15)        # vol/4 with vol = |det J|/6
    else:
        assert np.allclose(rows[:, :4], -1.0 / 120.0, atol=1e-15)   # -vol/20
        assert np.allclose(rows[:, 4:], 1.0 / 30.0, atol=1e-15)     # vol/5
    fr = m.free
    assert spla.eigsh(M[fr][:, fr], k=1, which="SA", return_eigenvectors=False)[0] > 0
    assert spla.eigsh(K[fr][:, fr], k=1, which="SA", return_eigenvectors=False)[0] > 0


def test_p2_reproduces_quadratic_integrals():
    # u = x^2 + y z, v = y^2 are in V_h (P2): u^T M v and u^T K v must equal the exact integrals over [-1,1]^3
    c, t = synth.cube_mesh(2, 1.0)
    m = FEMesh(c, t, 2)
    x = m.nodes
    u = x[:, 0] ** 2 + x[:, 1] * x[:, 2]
    v = x[:, 1] ** 2
    M = m.assemble(m.element_mass())
    K = m.assemble(m.element_stiffness())
    # int x^2 y^2 = (2/3)^2 * 2 ; int y z y^2 = 0
    assert abs(u @ (M @ v) - 8.0 / 9.0) < 1e-13
    # grad u = (2x, z, y), grad v = (0, 2y, 0): int 2 y z = 0 ; uu: int 4x^2 + z^2 + y^2 = 6*(2/3)*4 = 16
    assert abs(u @ (K @ v)) < 1e-13
    assert abs(u @ (K @ u) - 16.0) < 1e-12


@pytest.mark.parametrize("order", [1, 2])
def test_interpolation_exact_and_galerkin(order):
    cc, ct, fc, ft, par = synth.nested_cube_meshes(2, 1, 1.0)
    C, F = FEMesh(cc, ct, order), FEMesh(fc, ft, order)
    P = interpolation(C, F, par)
    if order == 2:
        assert np.abs(P @ _quad_poly(C.nodes) - _quad_poly(F.nodes)).max() < 1e-14
    else:
        lin = lambda x: 1 + x[:, 0] - 2 * x[:, 1] + 0.5 * x[:, 2]
        assert np.abs(P @ lin(C.nodes) - lin(F.nodes)).max() < 1e-14
    # Galerkin identity on nested spaces: P^T K_h P = K_H and P^T M_h P = M_H
    for build in ("element_stiffness", "element_mass"):
        Ah = F.assemble(getattr(F, build)())
        AH = C.assemble(getattr(C, build)())
        assert abs((P.T @ Ah @ P) - AH).max() < 1e-12
