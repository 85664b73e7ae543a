"""Pins of the graded (locally bisected) meshes that stand in for the paper's adaptive meshes (no GPU): conformity,
nesting in the coarse mesh, shape regularity, the grading rule, the finite-element identities of the oracle on them,
and the physical effect of grading (hydrogen's ground state)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.correction import Level
from oracle.fem import FEMesh, interpolation
from paper_2103_02824_gb300 import synth

PAIRS = np.array([(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)])


def _small():
    return synth.graded_mesh(2, 1.0, [[0.31, -0.22, 0.13]], h_min=0.15, alpha=0.3)


def _volumes(X, T):
    P = X[T]
    return np.einsum("ij,ij->i", np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), P[:, 3] - P[:, 0]) / 6.0


def test_conforming_nested_and_shape_regular():
    half = 1.0
    cc, ct, fc, ft, par = _small()
    assert ft.shape[0] > 10 * ct.shape[0]
    # conformity: an interior face belongs to exactly two tetrahedra, a face on the box to one
    F = np.sort(np.concatenate([ft[:, [1, 2, 3]], ft[:, [0, 2, 3]], ft[:, [0, 1, 3]], ft[:, [0, 1, 2]]]), axis=1)
    u, cnt = np.unique(F, axis=0, return_counts=True)
    X = fc[u]
    onb = np.zeros(len(u), dtype=bool)
    for ax in range(3):
        for side in (-half, half):
            onb |= np.all(np.abs(X[:, :, ax] - side) < 1e-12, axis=1)
    assert np.all(cnt[~onb] == 2) and np.all(cnt[onb] == 1)
    # no duplicated vertices
    assert np.unique(np.round(fc, 12), axis=0).shape[0] == fc.shape[0]
    # positive orientation, volumes tile the box and each coarse parent
    vol = _volumes(fc, ft)
    assert vol.min() > 0 and abs(vol.sum() - (2 * half) ** 3) < 1e-12
    assert np.allclose(np.bincount(par, weights=vol, minlength=ct.shape[0]), _volumes(cc, ct), rtol=1e-12)
    # every fine tetrahedron lies in its parent
    C = FEMesh(cc, ct, 1)
    s = np.einsum("eij,ekj->eki", C.Jinv[par], fc[ft] - C.x0[par][:, None, :])
    lam = np.concatenate([1 - s.sum(axis=2, keepdims=True), s], axis=2)
    assert lam.min() > -1e-12
    # bisection of Kuhn tetrahedra produces three similarity classes only
    P = fc[ft]
    diam = np.sqrt(((P[:, PAIRS[:, 0]] - P[:, PAIRS[:, 1]]) ** 2).sum(axis=2)).max(axis=1)
    assert len(np.unique(np.round(diam ** 3 / vol, 8))) <= 3


def test_grading_rule_and_determinism():
    centre = np.array([0.31, -0.22, 0.13])
    m1, m2 = _small(), _small()
    for a, b in zip(m1, m2):
        assert np.array_equal(a, b)
    _, _, fc, ft, _ = m1
    P = fc[ft]
    diam = np.sqrt(((P[:, PAIRS[:, 0]] - P[:, PAIRS[:, 1]]) ** 2).sum(axis=2)).max(axis=1)
    dist = np.linalg.norm(P.mean(axis=1) - centre, axis=1)
    assert np.all(diam <= np.maximum(0.15, 0.3 * dist) * (1 + 1e-12))
    assert diam[dist < 0.1].max() <= 0.15 and diam.max() > 3 * 0.15      # fine near the centre, coarse far away
    # fewer elements than a uniform mesh at the finest size (Kuhn cube of side 0.15/sqrt(3))
    uniform = 6 * (2.0 / (0.15 / np.sqrt(3))) ** 3
    assert ft.shape[0] < 0.5 * uniform


@pytest.mark.parametrize("order", [1, 2])
def test_fem_identities_on_graded_mesh(order):
    cc, ct, fc, ft, par = _small()
    Cm, Fm = FEMesh(cc, ct, order), FEMesh(fc, ft, order)
    K = Fm.assemble(Fm.element_stiffness())
    M = Fm.assemble(Fm.element_mass())
    one = np.ones(Fm.n_nodes)
    assert np.abs(K @ one).max() < 1e-11
    assert abs(one @ (M @ one) - 8.0) < 1e-11
    P = interpolation(Cm, Fm, par)
    f = (lambda x: 1.0 + 0.5 * x[:, 0] - 0.25 * x[:, 1] + 0.3 * x[:, 0] * x[:, 2] - 0.2 * x[:, 1] ** 2) if order == 2 \
        else (lambda x: 1.0 + x[:, 0] - 2.0 * x[:, 1] + 0.5 * x[:, 2])
    assert np.abs(P @ f(Cm.nodes) - f(Fm.nodes)).max() < 1e-13
    KH = Cm.assemble(Cm.element_stiffness())
    assert abs((P.T @ K @ P) - KH).max() < 1e-11


def test_grading_lowers_hydrogen_error_with_fewer_unknowns():
    Z, R = np.array([1.0]), np.zeros((1, 3))

    def lowest(mesh):
        lv = Level(*mesh, 1, Z, R)
        H = (0.5 * lv.Kff + lv.MVff).tocsc()
        w = spla.eigsh(H, k=1, M=lv.Mff.tocsc(), sigma=-0.6, which="LM", return_eigenvectors=False)[0]
        return w, lv.fine.n_free

    lu, nu = lowest(synth.nested_cube_meshes(4, 2, 10.0))
    lg, ng = lowest(synth.graded_mesh(4, 10.0, R, h_min=0.6, alpha=0.5))
    assert ng < nu
    assert -0.5 - 1e-3 < lg < lu                       # closer to the exact -1/2 Ha from above
    assert (lg + 0.5) < 0.3 * (lu + 0.5)


def test_correction_step_on_graded_mesh_keeps_the_ritz_bounds():
    """Bare hydrogen on the graded mesh (V_Hxc = 0): the corrected eigenvalue lies between the fine Galerkin
    eigenvalue and the coarse one (Rayleigh-Ritz in V_H + span{psi^}), as on the uniform meshes, and it is closer to
    -1/2 Ha than the corrected eigenvalue on the uniform 16^3 mesh, which has more unknowns."""
    import scipy.linalg as sla
    from oracle.correction import correction_step
    from oracle.fem import coulomb

    Z, R = np.array([1.0]), np.zeros((1, 3))

    def run(mesh):
        lv = Level(*mesh, 1, Z, R)
        C = lv.coarse
        xq, _, _, _ = C.quad()
        A = (0.5 * C.assemble(C.element_stiffness()) + C.assemble(C.element_mass(coulomb(xq, Z, R))))
        Mc = C.assemble(C.element_mass())
        lamH, psiH = sla.eigh(A[C.free][:, C.free].toarray(), Mc[C.free][:, C.free].toarray())
        out = correction_step(lv, psiH[:, :1], lamH[:1], [1.0], sigma=1.0, xc="none", hartree_bc="none")
        H = (0.5 * lv.Kff + lv.MVff).tocsc()
        lf = spla.eigsh(H, k=1, M=lv.Mff.tocsc(), sigma=-100.0, which="LM", return_eigenvectors=False)[0]
        return out["lam"][0], lf, lamH[0], lv.fine.n_free

    lg, lfg, lHg, ng = run(synth.graded_mesh(4, 10.0, R, h_min=0.6, alpha=0.5))
    lu, _, _, nu = run(synth.nested_cube_meshes(4, 2, 10.0))
    assert lfg - 1e-10 <= lg <= lHg + 1e-12 and lg > -0.5
    assert ng < nu and (lg + 0.5) < (lu + 0.5)


def test_cube_hierarchy_is_nested():
    """The intermediate levels of the multigrid hierarchy: 6 n^3 tetrahedra per level, and every element's
    vertices lie in its parent (barycentric coordinates in [0, 1]) down the whole chain."""
    meshes, parents = synth.cube_hierarchy(2, 3, 5.0)
    cc, ct = synth.cube_mesh(2, 5.0)
    fc, ft = synth.cube_mesh(16, 5.0)
    chain = [(cc, ct)] + meshes + [(fc, ft)]
    assert [t.shape[0] for _, t in chain] == [6 * n ** 3 for n in (2, 4, 8, 16)]
    for (pc, pt), (c, t), par in zip(chain[:-1], chain[1:], parents):
        x = pc[pt[par]]                                   # parent vertices [E, 4, 3]
        J = np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=2)
        for k in range(4):
            s = np.linalg.solve(J, (c[t[:, k]] - x[:, 0])[..., None])[..., 0]
            lam = np.concatenate([1.0 - s.sum(axis=1, keepdims=True), s], axis=1)
            assert lam.min() > -1e-12 and lam.max() < 1.0 + 1e-12


def test_graded_hierarchy_is_nested():
    """The multigrid levels of a graded mesh (refinement passes about 4x apart in size): the chain coarse -> levels -> fine is
    nested (every element's vertices lie in its parent), the children of every parent tile its volume, the levels
    grow, and the fine mesh is the graded mesh itself."""
    Z, R = synth.molecule(5, 3)
    cc, ct, fc, ft, _ = synth.graded_mesh(2, 5.0, R, h_min=0.6, alpha=0.5)
    meshes, parents = synth.graded_hierarchy(2, 5.0, R, h_min=0.6, alpha=0.5)
    assert len(meshes) >= 2
    chain = [(cc, ct)] + meshes + [(fc, ft)]
    sizes = [t.shape[0] for _, t in chain]
    assert all(a < b for a, b in zip(sizes[:-1], sizes[1:])), sizes

    def vol(c, t):
        x = c[t]
        return np.abs(np.einsum("ij,ij->i", np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]), x[:, 3] - x[:, 0])) / 6
    for (pc, pt), (c, t), par in zip(chain[:-1], chain[1:], parents):
        assert par.shape[0] == t.shape[0] and par.min() >= 0 and par.max() < pt.shape[0]
        x = pc[pt[par]]
        J = np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=2)
        for k in range(4):
            s = np.linalg.solve(J, (c[t[:, k]] - x[:, 0])[..., None])[..., 0]
            lam = np.concatenate([1.0 - s.sum(axis=1, keepdims=True), s], axis=1)
            assert lam.min() > -1e-12 and lam.max() < 1.0 + 1e-12
        summed = np.bincount(par, weights=vol(c, t), minlength=pt.shape[0])
        assert np.allclose(summed, vol(pc, pt), rtol=1e-12, atol=0)
