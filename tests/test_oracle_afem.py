"""Pins of the oracle's a posteriori error indicator and Dorfler marking (oracle/afem.py), no GPU: a global
quadratic (no jumps; the element residual is its Laplacian), the kink of |x| across a mesh plane (residual zero,
every jump -1 on the plane), the face structure, and Dorfler's set against brute force."""
import itertools

import numpy as np

from oracle import afem
from oracle.fem import FEMesh
from paper_2103_02824_gb300 import synth


def _vol(f):
    return np.abs(f.det) / 6.0


def test_quadratic_has_no_jumps_and_its_laplacian_as_residual():
    """u = x^2 + 2y^2 - z + 3 lies in P2: its gradient is continuous (no jump), and with V = lambda the residual is
    -1/2 Laplacian u = -3 everywhere, so eta^2 = 9 h_T^2 |T|."""
    c, t = synth.cube_mesh(2, 1.0)
    f = FEMesh(c, t, 2)
    x = f.nodes
    u = x[:, 0] ** 2 + 2 * x[:, 1] ** 2 - x[:, 2] + 3
    Vq = np.full((f.n_elems, 27), 0.7)
    eta2 = afem.indicators(f, u, [0.7], Vq)
    hT = afem._longest_edge(f.coords[f.tets])
    assert np.allclose(eta2, 9.0 * hT ** 2 * _vol(f), rtol=1e-12, atol=1e-14)


def test_kink_across_a_mesh_plane():
    """u = |x| on a mesh with x = 0 a plane of faces: linear on every element (residual 0 with V = lambda), gradient
    jump -2 across the plane, so J = -1 there and eta^2(T) = sum over T's faces in the plane of h_e |e|."""
    for order in (1, 2):
        c, t = synth.cube_mesh(4, 1.0)
        f = FEMesh(c, t, order)
        u = np.abs(f.nodes[:, 0])
        Vq = np.full((f.n_elems, 27), -0.3)
        eta2 = afem.indicators(f, np.stack([u, 2 * u], axis=1), [-0.3, -0.3], Vq)
        expect = np.zeros(f.n_elems)
        for e in range(f.n_elems):
            for fc in [(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)]:
                P = f.coords[f.tets[e, list(fc)]]
                if np.all(np.abs(P[:, 0]) < 1e-14):
                    area = 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
                    he = max(np.linalg.norm(P[a] - P[b]) for a, b in [(0, 1), (0, 2), (1, 2)])
                    expect[e] += (1.0 + 4.0) * he * area      # two orbitals: u and 2u
        assert expect.sum() > 0
        assert np.allclose(eta2, expect, rtol=1e-12, atol=1e-13)


def test_interior_faces_count_and_pairing():
    """4E = 2 (interior faces) + boundary faces, every pair shares its three vertices, T+ < T-."""
    c, t = synth.cube_mesh(3, 1.0)
    f = FEMesh(c, t, 1)
    rows = afem.interior_faces(f)
    n_boundary = 2 * 6 * 3 * 3          # 6 box faces, 3 x 3 squares, 2 triangles each
    assert 2 * rows.shape[0] + n_boundary == 4 * f.n_elems
    fl = [(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)]
    for ep, kp, em, km in rows:
        assert ep < em
        assert set(f.tets[ep, list(fl[kp])]) == set(f.tets[em, list(fl[km])])


def test_dorfler_is_the_smallest_set_and_breaks_ties_by_index():
    rng = np.random.default_rng(3)
    for trial in range(20):
        n = 9
        eta2 = rng.random(n) ** 3
        if trial % 4 == 0:
            eta2[[2, 5]] = eta2[7]                 # ties
        theta = [0.1, 0.4, 0.7, 1.0][trial % 4]
        mark = afem.dorfler(eta2, theta)
        tot = eta2.sum()
        assert eta2[mark].sum() >= theta * tot
        best = min(k for k in range(1, n + 1) for S in itertools.combinations(range(n), k)
                   if eta2[list(S)].sum() >= theta * tot)
        assert mark.sum() == best
        # every marked value is at least every unmarked one, and a tie at the cut goes to the lower index
        if mark.sum() < n:
            assert eta2[mark].min() >= eta2[~mark].max()
            cut = eta2[mark].min()
            tied = np.nonzero(eta2 == cut)[0]
            assert np.all(np.diff(mark[tied].astype(int)) <= 0)
