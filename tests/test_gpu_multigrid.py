"""The multigrid V(1,1) preconditioner of the Hartree Poisson solve on the nested hierarchy (coarse 4^3 cubes, the
intermediate uniform refinements, the fine mesh): the solution against the oracle's Hartree potential, fewer FCG
iterations than the two-level form and than Jacobi, and the argument checks of the hierarchy."""
import numpy as np
import pytest

from tests._cases import case, maxrel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def ctx(torch):
    from paper_2103_02824_gb300 import build, mk
    build.build()
    c = mk.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("name", ["mol4_p2_small", "mol4_p2_mid"])
def test_multigrid_poisson_matches_oracle(ctx, torch, name):
    from paper_2103_02824_gb300 import mk, synth
    c = case(name)
    wl = c["wl"]
    cc, ct, fc, ft, par = c["meshes"]
    m = mk.Mesh(ctx, fc, ft, cc, ct, par, 2)
    meshes, parents = synth.cube_hierarchy(wl["n_coarse"], wl["levels"], wl["half"])
    assert len(meshes) == wl["levels"] - 1
    m.set_hierarchy(meshes, parents)
    N, ld = c["N"], 8
    u = np.zeros((m.info["n_nodes"], ld))
    u[:, :N] = c["out"]["u"]
    u = torch.from_numpy(u).cuda()
    its = {}
    for label, kw in (("jacobi", dict(precision="fp64")), ("twolevel", dict(precision="mixed", coarse=True)),
                      ("multigrid", dict(precision="mixed", coarse="multigrid"))):
        w = torch.zeros(m.info["n_nodes"], dtype=torch.float64, device="cuda")
        rep = mk.mk_hartree_poisson(ctx, m, u, c["occ"], N, w, opt=mk.opts(rtol=1e-12, check_every=5, **kw))
        assert rep["max_rel_residual"] <= 1e-12
        assert maxrel(w.cpu().numpy(), c["out"]["w"]) < 1e-9
        its[label] = rep["iterations"]
    # with no intermediate level the V-cycle is the two-level form; with one or more it needs fewer iterations
    assert its["multigrid"] <= its["twolevel"] < its["jacobi"], its
    if meshes:
        assert its["multigrid"] < its["twolevel"], its
    print(f"\n{name}: Poisson iterations to 1e-12 {its}")
    m.close()


def test_multigrid_poisson_on_a_graded_mesh(ctx, torch):
    """The V-cycle over the refinement passes of the graded 12-nucleus mesh (levels about 4x apart) against the
    oracle's Hartree potential, with fewer iterations than Jacobi and than the two-level form."""
    from paper_2103_02824_gb300 import mk, synth
    c = case("cluster12_p2_small")
    wl = c["wl"]
    cc, ct, fc, ft, par = c["meshes"]
    m = mk.Mesh(ctx, fc, ft, cc, ct, par, 2)
    meshes, parents = synth.graded_hierarchy(wl["n_coarse"], wl["half"], wl["R"], h_min=wl["h_min"],
                                             alpha=wl["alpha"])
    assert len(meshes) >= 1
    m.set_hierarchy(meshes, parents)
    N = c["N"]
    ld = (N + 3) // 4 * 4
    u = np.zeros((m.info["n_nodes"], ld))
    u[:, :N] = c["out"]["u"]
    u = torch.from_numpy(u).cuda()
    its = {}
    for label, kw in (("jacobi", dict(precision="fp64")), ("twolevel", dict(precision="mixed", coarse=True)),
                      ("multigrid", dict(precision="mixed", coarse="multigrid"))):
        w = torch.zeros(m.info["n_nodes"], dtype=torch.float64, device="cuda")
        rep = mk.mk_hartree_poisson(ctx, m, u, c["occ"], N, w, opt=mk.opts(rtol=1e-12, check_every=5, **kw))
        assert rep["max_rel_residual"] <= 1e-12
        assert maxrel(w.cpu().numpy(), c["out"]["w"]) < 1e-9
        its[label] = rep["iterations"]
    print(f"\ncluster12_p2_small: Poisson iterations to 1e-12 {its}")
    assert its["multigrid"] < its["twolevel"] and its["multigrid"] < its["jacobi"], its
    m.close()


def test_hierarchy_arguments(ctx, torch):
    from paper_2103_02824_gb300 import mk, synth
    c = case("mol4_p2_mid")
    wl = c["wl"]
    cc, ct, fc, ft, par = c["meshes"]
    m = mk.Mesh(ctx, fc, ft, cc, ct, par, 2)
    N = c["N"]
    u = np.zeros((m.info["n_nodes"], 8))
    u[:, :N] = c["out"]["u"]
    u = torch.from_numpy(u).cuda()
    w = torch.zeros(m.info["n_nodes"], dtype=torch.float64, device="cuda")
    with pytest.raises(mk.MkError) as e:          # multigrid before a hierarchy exists
        mk.mk_hartree_poisson(ctx, m, u, c["occ"], N, w, opt=mk.opts(precision="mixed", coarse="multigrid"))
    assert e.value.code == mk.MK_ERR_INVALID_ARG
    meshes, parents = synth.cube_hierarchy(wl["n_coarse"], wl["levels"], wl["half"])
    bad = [parents[0], np.roll(parents[1], 1)]    # fine elements assigned to the wrong parents
    with pytest.raises(mk.MkError) as e:
        m.set_hierarchy(meshes, bad)
    assert e.value.code == mk.MK_ERR_INVALID_ARG
    m.set_hierarchy(meshes, parents)              # the right one is accepted after the failure
    rep = mk.mk_hartree_poisson(ctx, m, u, c["occ"], N, w, opt=mk.opts(precision="mixed", coarse="multigrid",
                                                                       rtol=1e-10))
    assert rep["max_rel_residual"] <= 1e-10
    m.close()
