"""Pins of the learned-preconditioner oracle (oracle/learned.py) against mathematics that does not depend on it:
finite differences of the forward pass, the closed-form first Adam steps, the reduction of FCG(1) with a fixed
Jacobi preconditioner to textbook PCG, and brute-force element loops for the assembly and the training samples."""
import numpy as np
import pytest

from oracle import learned as LO
from oracle.fem import FEMesh
from oracle.linalg import pcg
from paper_2103_02824_gb300 import synth


def small_mesh(order=2, n=2, half=1.0):
    coords, tets = synth.cube_mesh(n, half)
    return FEMesh(coords, tets, order)


def params_for(nloc, seed=3, bias=0.1):
    nin, nh, _, nout = LO.sizes(nloc)
    p = LO.unflatten(synth.mlp_init(nloc, seed).astype(np.float64), nin, nh, nout)
    rng = np.random.default_rng(seed + 100)
    for k in ("b1", "b2", "b3"):
        p[k] = p[k] + bias * rng.standard_normal(p[k].shape)
    return p


def test_flatten_roundtrip():
    p = params_for(10)
    v = LO.flatten(p)
    assert v.size == 64 * 22 + 64 + 64 * 64 + 64 + 10 * 64 + 10
    q = LO.unflatten(v, 22, 64, 10)
    for k in LO.PARAM_ORDER:
        assert np.array_equal(p[k], q[k])


@pytest.mark.parametrize("nloc", [4, 10])
def test_backward_matches_central_differences(nloc):
    p = params_for(nloc)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((9, nloc + 12))
    dY = rng.standard_normal((9, nloc))
    _, cache = LO.forward(p, X)
    g = LO.flatten(LO.backward(p, cache, dY))
    v = LO.flatten(p)
    nin, nh, _, nout = LO.sizes(nloc)

    def f(vec):
        y, _ = LO.forward(LO.unflatten(vec, nin, nh, nout), X)
        return float(np.sum(dY * y))

    h = 1e-6
    for k in rng.choice(v.size, 60, replace=False):
        e = np.zeros_like(v)
        e[k] = h
        fd = (f(v + e) - f(v - e)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_loss_gradient_matches_central_differences():
    p = params_for(10, seed=5)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((12, 22))
    U = np.abs(rng.standard_normal(12)) + 0.1
    E = rng.standard_normal((12, 10))
    loss, g = LO.loss_and_grad(p, X, U, E)
    # the loss is its definition: sum ||u y - e||^2 / sum u^2
    y, _ = LO.forward(p, X)
    assert loss == pytest.approx(np.sum((U[:, None] * y - E) ** 2) / np.sum(U * U), rel=1e-14)
    gv, v = LO.flatten(g), LO.flatten(p)

    def f(vec):
        return LO.loss_and_grad(LO.unflatten(vec, 22, 64, 10), X, U, E)[0]

    h = 1e-6
    for k in rng.choice(v.size, 60, replace=False):
        e = np.zeros_like(v)
        e[k] = h
        fd = (f(v + e) - f(v - e)) / (2 * h)
        assert abs(fd - gv[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, gv[k])


def test_adam_first_steps_closed_form():
    """With zero moments and a constant gradient g the bias-corrected moments are g and g^2, so each of the
    first steps moves every weight by lr * g / (|g| + eps)."""
    p = params_for(4)
    rng = np.random.default_rng(2)
    g = {k: rng.standard_normal(p[k].shape) for k in LO.PARAM_ORDER}
    st = {}
    lr, eps = 1e-3, 1e-8
    q = LO.adam_step(p, g, st, lr, eps=eps)
    q2 = LO.adam_step(q, g, st, lr, eps=eps)
    for k in LO.PARAM_ORDER:
        step = lr * g[k] / (np.abs(g[k]) + eps)
        np.testing.assert_allclose(p[k] - q[k], step, rtol=1e-10, atol=1e-15)
        np.testing.assert_allclose(p[k] - q2[k], 2 * step, rtol=1e-9, atol=1e-15)


def test_fcg_with_jacobi_is_pcg():
    """FCG(1) with a fixed symmetric preconditioner is CG: same iterates up to rounding."""
    m = small_mesh(2, 3, 2.0)
    K = m.assemble(m.element_stiffness())
    M = m.assemble(m.element_mass())
    fr = m.free
    A = (0.5 * K + 3.0 * M)[fr][:, fr].tocsr()
    rng = np.random.default_rng(4)
    B = rng.standard_normal((len(fr), 3))
    d = A.diagonal()
    X1, it1, res1 = pcg(A, B, tol=1e-12)
    X2, it2, res2 = LO.fcg(A, B, lambda R: R / d[:, None], tol=1e-12)
    assert np.all(np.abs(it1 - it2) <= 1)
    assert res2.max() <= 1e-12
    np.testing.assert_allclose(X2, X1, rtol=0, atol=1e-10 * np.abs(X1).max())


def test_zero_network_gives_jacobi():
    m = small_mesh()
    p = params_for(10)
    p["W3"][:] = 0.0
    p["b3"][:] = 0.0
    rng = np.random.default_rng(6)
    R = rng.standard_normal((m.n_nodes, 3))
    R[m.boundary] = 0
    diag = 1.0 + rng.random(m.n_nodes)
    Z = LO.precond(m, p, diag, R)
    expect = np.where(m.boundary[:, None], 0.0, R / diag[:, None])
    assert np.array_equal(Z, expect)


def test_constant_network_assembly_brute_force():
    """W3 = 0, b3 = 1: every slot of element e receives s_e / h_e; a node gets the mean over its incidences."""
    m = small_mesh()
    p = params_for(10)
    p["W3"][:] = 0.0
    p["b3"][:] = 1.0
    rng = np.random.default_rng(7)
    R = rng.standard_normal((m.n_nodes, 2))
    R[m.boundary] = 0
    Z = LO.correction(m, p, R)
    acc = np.zeros((m.n_nodes, 2))
    cnt = np.zeros(m.n_nodes)
    for e in range(m.n_elems):
        v = m.coords[m.tets[e]]
        J = np.stack([v[1] - v[0], v[2] - v[0], v[3] - v[0]], axis=1)
        h = abs(np.linalg.det(J)) ** (1.0 / 3.0)
        for a in range(10):
            node = m.elem[e, a]
            for j in range(2):
                acc[node, j] += np.linalg.norm(R[m.elem[e], j]) / h
            cnt[node] += 1
    expect = acc / cnt[:, None]
    expect[m.boundary] = 0
    np.testing.assert_allclose(Z, expect, rtol=1e-13, atol=0)


def test_features_invariances():
    m = small_mesh()
    p = params_for(10, seed=8)
    rng = np.random.default_rng(9)
    R = rng.standard_normal((m.n_nodes, 2))
    R[m.boundary] = 0
    X1, s1, h1 = LO.features(m, R)
    X2, s2, _ = LO.features(m, 3.5 * R)
    np.testing.assert_allclose(X2, X1, rtol=1e-14, atol=1e-15)       # scale-free inputs
    np.testing.assert_allclose(s2, 3.5 * s1, rtol=1e-14)
    shifted = FEMesh(m.coords + np.array([1.25, -0.5, 2.0]), m.tets, 2)
    X3, _, h3 = LO.features(shifted, R)
    np.testing.assert_allclose(X3, X1, rtol=0, atol=1e-13)           # translation-free geometry
    np.testing.assert_allclose(h3, h1, rtol=1e-13)
    # positive homogeneity of the correction: z_nn(a r) = a z_nn(r) for a > 0
    np.testing.assert_allclose(LO.correction(m, p, 2.0 * R), 2.0 * LO.correction(m, p, R), rtol=1e-12, atol=1e-14)


def test_harvest_brute_force():
    m = small_mesh()
    rng = np.random.default_rng(10)
    Rk, Xk, Xs = (rng.standard_normal((m.n_nodes, 2)) for _ in range(3))
    X, U, E = LO.harvest(m, Rk, Xk, Xs)
    N = 2
    for e in (0, 5, m.n_elems - 1):
        v = m.coords[m.tets[e]]
        J = np.stack([v[1] - v[0], v[2] - v[0], v[3] - v[0]], axis=1)
        h = abs(np.linalg.det(J)) ** (1.0 / 3.0)
        c = v.mean(axis=0)
        for j in range(N):
            r = Rk[m.elem[e], j]
            s = np.linalg.norm(r)
            row = e * N + j
            np.testing.assert_allclose(X[row, :10], r / s, rtol=1e-13)
            np.testing.assert_allclose(X[row, 10:], ((v - c) / h).ravel(), rtol=1e-13, atol=1e-15)
            assert U[row] == pytest.approx(s / h, rel=1e-13)
            np.testing.assert_allclose(E[row], (Xs - Xk)[m.elem[e], j], rtol=1e-14)
