"""The step on the other workload kinds, chained on the GPU against the oracle: the 12-nucleus cluster on a mesh
graded toward its nuclei by newest-vertex bisection (the adaptive-mesh workload, 28 orbitals, topology of the
graded mesh bit-exact), and an 8-nucleus evaluation molecule of the learned preconditioner (learned FCG, two-level
Poisson).  Both sides solve to 1e-12 / 1e-13."""
import numpy as np
import pytest

from tests._cases import case, maxrel, rel

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


def _check_step(st, c, N):
    o = c["out"]
    lam = st.lam.cpu().numpy()
    assert np.abs(lam - o["lam"]).max() < 1e-6      # the target
    assert np.abs(lam - o["lam"]).max() < 1e-9      # observed: rounding level
    psi = st.psi.cpu().numpy()[:, :N]
    for i in range(N):
        assert rel(psi[:, i], o["psi"][:, i]) < 1e-6 and maxrel(psi[:, i], o["psi"][:, i]) < 1e-6
    return float(np.abs(lam - o["lam"]).max())


def test_graded_cluster_step_matches_oracle(ctx, torch):
    from paper_2103_02824_gb300 import mk
    from paper_2103_02824_gb300.step import CorrectionStep
    c = case("cluster12_p2_small")
    lv = c["level"]
    cc, ct, fc, ft, par = c["meshes"]
    m = mk.Mesh(ctx, fc, ft, cc, ct, par, 2)
    for level, L in ((0, lv.fine), (1, lv.coarse)):
        nodes, bnd, elem, col = m.topology(level)
        assert np.array_equal(nodes, L.nodes) and np.array_equal(bnd, L.boundary) and np.array_equal(elem, L.elem)
        if level == 0:
            assert np.array_equal(col, L.colouring())
    N = c["N"]
    assert N == 28
    for prec in ("mixed", "fp64"):
        st = CorrectionStep(ctx, m, c["wl"]["Z"], c["wl"]["R"], N)
        st.run(c["psiH"], c["lamH"], c["occ"], c["sigma"], xc=c["xc"], hartree_bc="multipole",
               solve_opts=mk.opts(precision=prec, rtol=1e-12, check_every=10),
               poisson_opts=mk.opts(precision=prec, rtol=1e-12, check_every=10, coarse=prec == "mixed"))
        torch.cuda.synchronize()
        err = _check_step(st, c, N)
        print(f"\ngraded cluster ({prec}): max |lambda - oracle| = {err:.3e} Ha")
    m.close()


def test_eval_molecule_learned_step_matches_oracle(ctx, torch):
    from paper_2103_02824_gb300 import mk, synth
    from paper_2103_02824_gb300.step import CorrectionStep
    c = case("mol8_p2_small")
    cc, ct, fc, ft, par = c["meshes"]
    m = mk.Mesh(ctx, fc, ft, cc, ct, par, 2)
    N = c["N"]
    mlp = mk.Mlp(ctx, 10, synth.mlp_init(10, 0))
    st = CorrectionStep(ctx, m, c["wl"]["Z"], c["wl"]["R"], N)
    st.run(c["psiH"], c["lamH"], c["occ"], c["sigma"], xc=c["xc"], hartree_bc="multipole",
           solve_opts=mk.opts(precision="mixed", precond="learned", mlp=mlp, rtol=1e-12, check_every=10),
           poisson_opts=mk.opts(precision="mixed", rtol=1e-12, check_every=10, coarse=True))
    torch.cuda.synchronize()
    err = _check_step(st, c, N)
    print(f"\neval molecule (learned FCG, N = {N}): max |lambda - oracle| = {err:.3e} Ha")
    mlp.close()
    m.close()
