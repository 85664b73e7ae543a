"""Pins of the oracle's Refine step (oracle/refine.py), no GPU: bisecting every element three times reproduces the
uniform refinement of the Kuhn mesh, a single mark closes into a conforming nested mesh, and the result equals the
vectorised bisection of the input generator (synth.NVBMesh) on random marks."""
import numpy as np

from oracle import refine as R
from paper_2103_02824_gb300 import synth


def _vol(X, T):
    P = X[T]
    return np.einsum("ij,ij->i", np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), P[:, 3] - P[:, 0]) / 6.0


def test_three_full_rounds_are_the_uniform_refinement():
    """Three rounds that bisect every element halve every edge once: the vertices are exactly the lattice of half
    the spacing, every element has an eighth of a Kuhn element's volume and the Kuhn edge lengths h/2 (1, sqrt 2,
    sqrt 3), and the mesh is conforming."""
    X, T, K = R.kuhn(2, 1.0)
    for _ in range(3):
        X, T, K, _, rounds = R.refine(X, T, K, np.ones(len(T), dtype=bool))
        assert rounds == 1                              # bisecting everything leaves nothing hanging
    assert len(T) == 8 * 48 and len(X) == 5 ** 3
    g = np.linspace(-1.0, 1.0, 5)
    lattice = {(a, b, c) for a in g for b in g for c in g}
    assert {tuple(x) for x in X} == lattice
    h = 0.5
    assert np.allclose(np.abs(_vol(X, T)), h ** 3 / 6, rtol=1e-13)
    for t in T:
        d = sorted(np.linalg.norm(X[t[a]] - X[t[b]]) for a in range(4) for b in range(a + 1, 4))
        assert np.allclose(d, h * np.array([1, 1, 1, np.sqrt(2), np.sqrt(2), np.sqrt(3)]), rtol=1e-13)
    assert all(len(els) <= 2 for els in _faces(T).values())


def _faces(T):
    f = {}
    for e, t in enumerate(T):
        for k in range(4):
            key = tuple(sorted(int(t[j]) for j in range(4) if j != k))
            f.setdefault(key, []).append(e)
    return f


def test_one_mark_closes_into_a_conforming_nested_mesh():
    X0, T0, K0 = R.kuhn(3, 1.0)
    marked = np.zeros(len(T0), dtype=bool)
    marked[len(T0) // 2] = True
    X, T, K, parent, rounds = R.refine(X0, T0, K0, marked)
    assert rounds >= 2 and len(T) > len(T0) + 1       # the closure cut neighbours too
    assert set(np.unique(K)) <= {1, 2, 3}
    for key, els in _faces(T).items():
        assert len(els) <= 2
        if len(els) == 1:                             # a boundary face lies on the box boundary
            P = X[list(key)]
            assert np.any(np.all(np.abs(np.abs(P) - 1.0) < 1e-12, axis=0))
    v = np.abs(_vol(X, T))
    assert np.allclose(np.bincount(parent, weights=v, minlength=len(T0)), np.abs(_vol(X0, T0)), rtol=1e-13)
    for e in range(len(T)):                           # every child inside its parent
        P = X0[T0[parent[e]]]
        J = np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]], axis=1)
        for x in X[T[e]]:
            s = np.linalg.solve(J, x - P[0])
            assert s.min() > -1e-12 and s.sum() < 1 + 1e-12


def test_equals_the_vectorised_bisection_on_random_marks():
    rng = np.random.default_rng(4)
    nvb = synth.NVBMesh.kuhn(3, 2.0)
    X, T, K = nvb.coords().copy(), nvb.T.copy(), nvb.K.copy()
    for _ in range(4):
        marked = rng.random(len(T)) < 0.15
        Xo, To, Ko, Po, ro = R.refine(X, T, K, marked)
        nvb = synth.NVBMesh(X, T, K)
        rs = nvb.refine(np.nonzero(marked)[0])
        assert ro == rs
        assert np.array_equal(To, nvb.T) and np.array_equal(Ko, nvb.K) and np.array_equal(Po, nvb.A)
        assert np.array_equal(Xo, nvb.coords())
        X, T, K = Xo, To, Ko
