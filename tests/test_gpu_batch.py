"""Batched correction solves (many molecules, uneven meshes and orbital counts, shared launches) and the patch
autotuner, against the single-problem solver.  The batched kernels run the single-problem kernel bodies with the
same block maps and summation orders, so every problem's result must be bit-identical to its own solve."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def env(torch):
    from paper_2103_02824_gb300 import build, mk, synth
    from paper_2103_02824_gb300.step import upload_workload
    build.build()
    ctx = mk.Context(0)
    small = [upload_workload(ctx, synth.workload("mol4_p2_small"))[0] for _ in range(2)]
    mid = upload_workload(ctx, synth.workload("mol4_p2_mid"))[0]
    yield ctx, small, mid
    for m in small + [mid]:
        m.close()
    ctx.close()


def test_batch_matches_single_solves(env, torch):
    from paper_2103_02824_gb300 import learned, mk, synth
    ctx, small, mid = env
    meshes = [small[0], small[1], mid]
    probs = [learned.Problem(ctx, m, *synth.molecule(seed, 4)) for m, seed in zip(meshes, (3, 5, 4))]
    assert len({p.N for p in probs}) > 1, "want uneven orbital counts"
    opt = mk.opts(precision="mixed", rtol=1e-10, inner_rtol=1e-4, check_every=5)
    singles = []
    for p in probs:
        x, rep = p.solve(opt)
        assert rep["max_rel_residual"] <= 1e-10
        singles.append(x)
    xs = [p.u.clone() for p in probs]
    reps = mk.mk_batch_correction_solve(ctx, meshes, [p.mol for p in probs], [p.sigma for p in probs],
                                        [p.rhs for p in probs], xs, [p.N for p in probs], opt=opt)
    torch.cuda.synchronize()
    for p, x, xb, r in zip(probs, singles, xs, reps):
        assert r["max_rel_residual"] <= 1e-10 and r["status"] == 0
        assert torch.equal(x, xb), float((x - xb).abs().max())
    print("\nbatched problems: N", [p.N for p in probs], "inner iterations", [r["iterations"] for r in reps])


def test_batch_with_32_columns_matches_single_solves(env, torch):
    """A 22-orbital molecule in a 32-column problem beside a narrow one: one register-staged launch covers all 32
    columns, and the results are bit-identical to the single solves."""
    from paper_2103_02824_gb300 import learned, mk, synth
    ctx, small, mid = env
    wide = learned.Problem(ctx, small[0], *synth.molecule(2002, 8))
    narrow = learned.Problem(ctx, small[1], *synth.molecule(3, 4))
    assert 16 < wide.N <= 32

    def padded(t, ld):
        out = torch.zeros((t.shape[0], ld), dtype=t.dtype, device=t.device)
        out[:, :t.shape[1]] = t
        return out
    rhs = [padded(wide.rhs, 32), narrow.rhs]
    x0 = [padded(wide.u, 32), narrow.u]
    opt = mk.opts(precision="mixed", rtol=1e-10, inner_rtol=1e-4, check_every=5)
    singles = []
    for p, r, x in zip((wide, narrow), rhs, x0):
        xs = x.clone()
        rep = mk.mk_correction_solve(ctx, p.mesh, p.mol, p.sigma, r, xs, p.N, opt=opt)
        assert rep["max_rel_residual"] <= 1e-10
        singles.append(xs)
    xb = [x.clone() for x in x0]
    reps = mk.mk_batch_correction_solve(ctx, [wide.mesh, narrow.mesh], [wide.mol, narrow.mol],
                                        [wide.sigma, narrow.sigma], rhs, xb, [wide.N, narrow.N], opt=opt)
    torch.cuda.synchronize()
    for x, y, r in zip(singles, xb, reps):
        assert r["max_rel_residual"] <= 1e-10 and torch.equal(x, y), float((x - y).abs().max())


def test_autotune_patches(env, torch):
    from paper_2103_02824_gb300 import mk, synth
    ctx, small, mid = env
    mol = mk.Molecule(*synth.molecule(2, 4))
    n = mid.info["n_nodes"]
    g = torch.Generator(device="cuda").manual_seed(3)
    x = torch.randn((n, 8), generator=g, device="cuda", dtype=torch.float32)
    y0, y1 = torch.empty_like(x), torch.empty_like(x)
    mk.mk_operator_apply(ctx, mid, mol, 5.0, x, y0)
    best, ms = mk.mk_autotune_patches(ctx, mid, 8)
    assert best in (64, 96, 128, 192) and all(t > 0 for t in ms)
    mk.mk_operator_apply(ctx, mid, mol, 5.0, x, y1)
    torch.cuda.synchronize()
    assert torch.allclose(y1, y0, rtol=1e-5, atol=1e-5 * float(y0.abs().max()))
    mk.mk_mesh_set_patch_elems(mid, 128)
    print("\nautotune: best", best, "ms per application", ms)
