"""The outer AFEM loop's Refine step (Sec. 2: the marked elements are refined so that the mesh stays shape regular and
conforming), oracle side: newest-vertex bisection in Maubach's form with conforming closure, element by element in
plain Python (small meshes only).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

A tetrahedron (x0, x1, x2, x3) with tag k in {1, 2, 3} is cut at the midpoint z of its refinement edge x0-xk into
(x0, .., x_{k-1}, z, x_{k+1}, .., x3), which keeps its index, and (x1, .., xk, z, x_{k+1}, .., x3), appended after the
existing elements in the order of the cut ones; both take tag k - 1 (3 after 1).  The first round cuts the marked
elements; every later round cuts the elements that hold an edge already cut, until none does.  Readings (the paper
names only "refined so that the triangulation is still shape regular and conforming"): newest-vertex bisection in
this form (Maubach's), whose closure always ends on Kuhn meshes; a new midpoint is numbered after the existing
vertices in the order of the lowest-index element that cuts its edge in its round.
"""
from __future__ import annotations

import numpy as np


def refine(X, T, K, marked):
    """(X', T', K', parent, rounds) for vertices X [nv, 3], tetrahedra T [E, 4] in bisection order, tags K [E] and
    marked [E] (bool); parent[e'] = the input element that contains output element e'."""
    X = [tuple(float(c) for c in x) for x in np.asarray(X, dtype=np.float64)]
    T = [list(int(v) for v in t) for t in np.asarray(T)]
    K = [int(k) for k in np.asarray(K)]
    parent = list(range(len(T)))
    mid = {}                                    # cut edge (lo, hi) -> midpoint vertex
    cut = [e for e in range(len(T)) if marked[e]]
    rounds = 0
    while cut:
        # new midpoints, numbered in the order of the first cutting element
        for e in cut:
            a, b = T[e][0], T[e][K[e]]
            key = (min(a, b), max(a, b))
            if key not in mid:
                mid[key] = len(X)
                X.append(tuple(0.5 * (X[a][c] + X[b][c]) for c in range(3)))
        for e in cut:
            v, k = T[e], K[e]
            z = mid[(min(v[0], v[k]), max(v[0], v[k]))]
            nk = k - 1 if k > 1 else 3
            second = v[1:k + 1] + [z] + v[k + 1:]
            first = v[:k] + [z] + v[k + 1:]
            T[e], K[e] = first, nk
            T.append(second)
            K.append(nk)
            parent.append(parent[e])
        rounds += 1
        cut = [e for e in range(len(T))
               if any((min(T[e][a], T[e][b]), max(T[e][a], T[e][b])) in mid
                      for a, b in ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)))]
    return (np.array(X), np.array(T, dtype=np.int64), np.array(K, dtype=np.int64), np.array(parent, dtype=np.int64),
            rounds)


def kuhn(n: int, half: float):
    """The Kuhn mesh of n^3 cubes of [-half, half]^3 in Maubach's form: every cube split along its main diagonal into
    the six tetrahedra x0 -> x0 + e_p0 -> x0 + e_p0 + e_p1 -> x0 + (1,1,1) (vertices in path order), tag 3."""
    import itertools
    h = 2.0 * half / n
    g = np.arange(n + 1)
    I, J, Kk = np.meshgrid(g, g, g, indexing="ij")
    X = np.stack([I.ravel(order="F"), J.ravel(order="F"), Kk.ravel(order="F")], axis=1) * h - half
    vid = lambda i, j, k: i + (n + 1) * (j + (n + 1) * k)
    T = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                for p in itertools.permutations(range(3)):
                    c = [i, j, k]
                    path = [vid(*c)]
                    for d in p:
                        c[d] += 1
                        path.append(vid(*c))
                    T.append(path)
    return X, np.array(T, dtype=np.int64), np.full(len(T), 3, dtype=np.int64)
