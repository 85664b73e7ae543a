"""Seeded synthetic inputs for the fine-mesh correction step.

This module is the only code that both the CUDA path's callers (tests, bench, smoke) and the CPU oracle use.
It holds none of the method's arithmetic: box meshes made of cubes, sampled molecules, occupation numbers and
closed-form trial functions evaluated at points that the caller supplies.

Workload shapes follow the paper's experiments (Sec. 4): all-electron molecules with nuclear charges of H..O in
boxes of half-width 6..15 bohr, N = 1..64 doubly occupied orbitals, meshes of tetrahedra obtained by uniform
refinement of a cube mesh (the paper's coarsest mesh is such a mesh with 24,576 tetrahedra), or by local
bisection graded toward the nuclei (the paper's adaptive meshes are locally refined, Sec. 2).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

# Kuhn (Freudenthal) split of a cube: one tetrahedron per permutation of the axes, walking from the
# corner (0,0,0) to (1,1,1) one unit step per axis.  The six are nested under 2x refinement.
_PERMS = list(itertools.permutations((0, 1, 2)))
_PERM_SIGN = [1, -1, -1, 1, 1, -1]


def cube_mesh(n: int, half: float):
    """Kuhn triangulation of [-half, half]^3 into n^3 cubes x 6 positively oriented tetrahedra.

    Returns (coords [(n+1)^3, 3] float64, tets [6 n^3, 4] int32).  Vertex (i,j,k) has index
    i + (n+1) (j + (n+1) k); tetrahedron 6 c + p belongs to cube c = i + n (j + n k) and permutation p.
    """
    h = 2.0 * half / n
    g = np.arange(n + 1)
    k, j, i = np.meshgrid(g, g, g, indexing="ij")
    coords = np.stack([-half + i.ravel() * h, -half + j.ravel() * h, -half + k.ravel() * h], axis=1)

    def vid(ii, jj, kk):
        return ii + (n + 1) * (jj + (n + 1) * kk)

    c = np.arange(n ** 3)
    ci, cj, ck = c % n, (c // n) % n, c // (n * n)
    tets = np.empty((n ** 3, 6, 4), dtype=np.int64)
    for p, perm in enumerate(_PERMS):
        pos = [ci.copy(), cj.copy(), ck.copy()]
        path = [vid(*pos)]
        for ax in perm:
            pos[ax] = pos[ax] + 1
            path.append(vid(*pos))
        if _PERM_SIGN[p] < 0:  # swap the last two vertices to make the orientation positive
            path[2], path[3] = path[3], path[2]
        tets[:, p, :] = np.stack(path, axis=1)
    return coords, tets.reshape(-1, 4).astype(np.int32)


def nested_cube_meshes(n_coarse: int, levels: int, half: float):
    """Coarse and fine Kuhn meshes of the same box, the fine one `levels` uniform 2x refinements deeper.

    Returns (coarse_coords, coarse_tets, fine_coords, fine_tets, fine_parent) with fine_parent[e] the
    coarse tetrahedron that contains fine tetrahedron e.
    """
    cc, ct = cube_mesh(n_coarse, half)
    r = 2 ** levels
    nf = n_coarse * r
    fc, ft = cube_mesh(nf, half)
    e = np.arange(ft.shape[0])
    cube = e // 6
    fi, fj, fk = cube % nf, (cube // nf) % nf, cube // (nf * nf)
    coarse_cube = (fi // r) + n_coarse * ((fj // r) + n_coarse * (fk // r))
    # centroid of the fine tetrahedron in the unit cube of its coarse cube
    hc = 2.0 * half / n_coarse
    cen = fc[ft].mean(axis=1)
    ccorner = np.stack([-half + (fi // r) * hc, -half + (fj // r) * hc, -half + (fk // r) * hc], axis=1)
    frac = (cen - ccorner) / hc
    # the coarse Kuhn tetrahedron of permutation p is {x : x[p0] >= x[p1] >= x[p2]}
    order = np.argsort(-frac, axis=1, kind="stable")
    perm_index = {perm: p for p, perm in enumerate(_PERMS)}
    pidx = np.array([perm_index[tuple(o)] for o in order.tolist()], dtype=np.int64)
    parent = (6 * coarse_cube + pidx).astype(np.int32)
    return cc, ct, fc, ft, parent


def cube_hierarchy(n_coarse: int, levels: int, half: float):
    """The intermediate meshes between the coarse (n_coarse^3 cubes) and the fine (n_coarse 2^levels cubes per side)
    Kuhn meshes of nested_cube_meshes, coarsest first, with the parent maps of the nested chain: returns
    (meshes, parents), meshes[k] = (coords, tets) of n_coarse 2^(k+1) cubes per side for k < levels - 1,
    parents[k] the element of the next coarser mesh containing each element of meshes[k], and parents[-1] that of
    the finest intermediate mesh for each fine element."""
    meshes, parents = [], []
    for k in range(1, levels):
        _, _, c, t, par = nested_cube_meshes(n_coarse * 2 ** (k - 1), 1, half)
        meshes.append((c, t))
        parents.append(par)
    if levels >= 2:
        parents.append(nested_cube_meshes(n_coarse * 2 ** (levels - 1), 1, half)[4])
    return meshes, parents


def _edge_keys(a, b, nv_cap: int):
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    return lo.astype(np.int64) * nv_cap + hi.astype(np.int64)


class NVBMesh:
    """A tetrahedral mesh in Maubach's form for newest-vertex bisection: vertices X [nv, 3], tetrahedra T [E, 4] with
    their vertices in bisection order and tags K [E] in {1, 2, 3}.  A tetrahedron (x0, x1, x2, x3) with tag k is cut
    at the midpoint z of the edge x0-xk into (x0, .., x_{k-1}, z, x_{k+1}, .., x3), which keeps its index, and
    (x1, .., xk, z, x_{k+1}, .., x3), appended after the existing elements in the order of the cut ones; both take
    tag k - 1 (3 after 1).  A new midpoint is numbered after the existing vertices in the order of the first element
    (lowest index) that cuts its edge.  The Kuhn tetrahedra, with their vertices in path order and tag 3, are
    compatible with it: every refinement is conforming after closure (any tetrahedron that holds an edge already cut
    is cut too, until none does), the elements fall into a bounded number of similarity classes, and every
    tetrahedron lies inside the one it descends from.  A (ancestor) and B (the element of the last `mark_level`)
    track the nesting."""

    _PAIRS = np.array([(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)])
    _CAP = 1 << 31

    def __init__(self, X, T, K):
        self.V = [np.asarray(X, dtype=np.float64)]
        self.nv = self.V[0].shape[0]
        self.T = np.asarray(T, dtype=np.int64).copy()
        self.K = np.asarray(K, dtype=np.int64).copy()
        self.A = np.arange(self.T.shape[0], dtype=np.int64)
        self.B = self.A.copy()
        self.split_k = np.zeros(0, dtype=np.int64)   # sorted keys of the edges already cut
        self.split_m = np.zeros(0, dtype=np.int64)   # their midpoints

    @classmethod
    def kuhn(cls, n: int, half: float):
        """The Kuhn mesh of n^3 cubes in Maubach's form (path order, tag 3)."""
        cc, ct = cube_mesh(n, half)
        T = ct.astype(np.int64).copy()
        neg = np.array([_PERM_SIGN[p] < 0 for p in range(6)] * (T.shape[0] // 6))
        T[neg, 2], T[neg, 3] = ct[neg, 3], ct[neg, 2]
        return cls(cc, T, np.full(T.shape[0], 3, dtype=np.int64))

    def coords(self):
        if len(self.V) > 1:
            self.V = [np.concatenate(self.V, axis=0)]
        return self.V[0]

    def _midpoints(self, a, b):
        keys = _edge_keys(a, b, self._CAP)
        pos = np.searchsorted(self.split_k, keys)
        found = np.zeros(keys.size, dtype=bool)
        ok = pos < self.split_k.size
        found[ok] = self.split_k[pos[ok]] == keys[ok]
        if not found.all():
            uk, first = np.unique(keys[~found], return_index=True)
            o = np.argsort(first, kind="stable")          # in order of first appearance (element order)
            uk, first = uk[o], first[o]
            ia, ib = a[~found][first], b[~found][first]
            X = self.coords()
            self.V.append(0.5 * (X[ia] + X[ib]))
            ids = self.nv + np.arange(uk.size, dtype=np.int64)
            self.nv += uk.size
            allk = np.concatenate([self.split_k, uk])
            allm = np.concatenate([self.split_m, ids])
            srt = np.argsort(allk, kind="stable")
            self.split_k, self.split_m = allk[srt], allm[srt]
            pos = np.searchsorted(self.split_k, keys)
        return self.split_m[pos]

    def bisect(self, idx):
        """Bisect the elements idx (ascending)."""
        t, k = self.T[idx], self.K[idx]
        z = self._midpoints(t[:, 0], t[np.arange(idx.size), k])
        c1 = t.copy()
        c1[np.arange(idx.size), k] = z
        c2 = np.empty_like(t)
        for kk in (1, 2, 3):
            sel = k == kk
            if not sel.any():
                continue
            tk = t[sel]
            c2[sel] = np.concatenate([tk[:, 1:kk + 1], z[sel, None], tk[:, kk + 1:]], axis=1)
        nk = np.where(k > 1, k - 1, 3)
        self.T[idx], self.K[idx] = c1, nk
        self.T = np.concatenate([self.T, c2])
        self.K = np.concatenate([self.K, nk])
        self.A = np.concatenate([self.A, self.A[idx]])
        self.B = np.concatenate([self.B, self.B[idx]])

    def hanging(self):
        """Elements (ascending) that hold an edge already cut."""
        keys = _edge_keys(self.T[:, self._PAIRS[:, 0]], self.T[:, self._PAIRS[:, 1]], self._CAP)
        pos = np.searchsorted(self.split_k, keys)
        hit = np.zeros(keys.shape, dtype=bool)
        ok = pos < self.split_k.size
        hit[ok] = self.split_k[pos[ok]] == keys[ok]
        return np.nonzero(hit.any(axis=1))[0]

    def refine(self, idx):
        """Bisect the elements idx (ascending), then close: bisect every element holding a cut edge until none
        does.  Returns the number of bisection rounds."""
        rounds = 0
        if np.size(idx):
            self.bisect(np.asarray(idx, dtype=np.int64))
            rounds += 1
        while True:
            h = self.hanging()
            if h.size == 0:
                return rounds
            self.bisect(h)
            rounds += 1

    def mark_level(self):
        """Start a new level of the nested chain: B becomes the identity of the current elements."""
        self.B = np.arange(self.T.shape[0], dtype=np.int64)


def graded_mesh(n_coarse: int, half: float, centres, h_min: float = 0.05, alpha: float = 0.3,
                max_elems: int = 4_000_000, snapshots=None, maubach=None):
    """A conforming tetrahedral mesh of [-half, half]^3 refined toward the points `centres` [M, 3] until every
    element's longest edge is at most max(h_min, alpha * distance from its centroid to the nearest centre), nested
    in the Kuhn mesh of n_coarse^3 cubes, by newest-vertex bisection (NVBMesh): every pass bisects the elements that
    violate the rule, then closes the mesh.

    Returns (coarse_coords, coarse_tets, fine_coords, fine_tets, fine_parent) like nested_cube_meshes, with
    positively oriented tetrahedra.  Deterministic: no randomness, stable orderings.  snapshots: a list that, when
    given, receives after every refinement pass the mesh so far as (coords, tets, prev), prev the element of the
    previous snapshot (or of the coarse mesh) that contains each element: a nested chain.  maubach: a list that,
    when given, receives the final NVBMesh (its tetrahedra in bisection order, with their tags).
    """
    cc, ct = cube_mesh(n_coarse, half)
    centres = np.asarray(centres, dtype=np.float64).reshape(-1, 3)
    nvb = NVBMesh.kuhn(n_coarse, half)
    pairs = NVBMesh._PAIRS
    while True:
        X = nvb.coords()
        P = X[nvb.T]
        diam = np.sqrt(((P[:, pairs[:, 0]] - P[:, pairs[:, 1]]) ** 2).sum(axis=2)).max(axis=1)
        cen = P.mean(axis=1)
        dist = np.sqrt(((cen[:, None, :] - centres[None, :, :]) ** 2).sum(axis=2)).min(axis=1)
        mark = np.nonzero(diam > np.maximum(h_min, alpha * dist) * (1 + 1e-12))[0]
        if mark.size == 0:
            break
        if nvb.T.shape[0] + mark.size > max_elems:
            raise ValueError("graded_mesh: more than max_elems elements")
        nvb.refine(mark)
        if snapshots is not None:
            snapshots.append((nvb.coords(), _oriented(nvb.coords(), nvb.T), nvb.B.astype(np.int32)))
            nvb.mark_level()
    if maubach is not None:
        maubach.append(nvb)
    X = nvb.coords()
    return cc, ct, X, _oriented(X, nvb.T), nvb.A.astype(np.int32)


def _oriented(X, T):
    """The tetrahedra T with their last two vertices swapped where the orientation is negative (int32 copy)."""
    P = X[T]
    vol = np.einsum("ij,ij->i", np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), P[:, 3] - P[:, 0])
    T = T.copy()
    flip = vol < 0
    T[flip, 2], T[flip, 3] = T[flip, 3].copy(), T[flip, 2].copy()
    return T.astype(np.int32)


def graded_hierarchy(n_coarse: int, half: float, centres, h_min: float = 0.05, alpha: float = 0.3,
                     ratio: float = 4.0):
    """Intermediate meshes between the coarse Kuhn mesh and the graded mesh of graded_mesh (same arguments), as
    cube_hierarchy returns them: of the meshes after each refinement pass, the first with at least `ratio` times the
    elements of the last level kept (the coarse mesh to begin with), coarsest first, each with the parent map into
    the next coarser level (the coarse mesh for the first); the last parent map is that of the fine mesh into the
    finest intermediate mesh."""
    snaps = []
    graded_mesh(n_coarse, half, centres, h_min=h_min, alpha=alpha, snapshots=snaps)
    return hierarchy_from_snapshots(snaps, ratio)


def hierarchy_from_snapshots(snaps, ratio: float = 4.0):
    """(meshes, parents) of graded_hierarchy from the snapshots graded_mesh recorded."""
    meshes, parents = [], []
    comp = None
    kept = snaps[0][2].max() + 1 if snaps else 0   # elements of the coarse mesh
    for k, (X, T, prev) in enumerate(snaps):
        comp = prev if comp is None else comp[prev]
        if k == len(snaps) - 1:
            parents.append(comp.astype(np.int32))
        elif T.shape[0] >= ratio * kept:
            meshes.append((X, T))
            parents.append(comp.astype(np.int32))
            kept = T.shape[0]
            comp = None
    return meshes, parents


def molecule(seed: int, n_nuclei: int, zmax: int = 8, half: float = 3.0, dmin: float = 1.5):
    """Nuclei with charges uniform in {1..zmax}, positions uniform in [-half, half]^3 by sequential
    rejection so that every pair is at least dmin bohr apart.  Returns (Z [M], R [M,3])."""
    rng = np.random.default_rng(seed)
    Z = rng.integers(1, zmax + 1, size=n_nuclei).astype(np.float64)
    R = []
    while len(R) < n_nuclei:
        p = rng.uniform(-half, half, size=3)
        if all(np.linalg.norm(p - q) >= dmin for q in R):
            R.append(p)
    return Z, np.array(R, dtype=np.float64).reshape(n_nuclei, 3)


def occupations(Z) -> np.ndarray:
    """Spin-unpolarised filling: N = ceil(sum Z / 2) orbitals, each holding 2 electrons except that the
    last one holds the remainder (1 when the electron count is odd)."""
    ne = int(round(float(np.sum(Z))))
    n = (ne + 1) // 2
    f = np.full(n, 2.0)
    f[-1] = ne - 2 * (n - 1)
    return f


# Shells used for trial orbitals, in filling order: (principal n, angular polynomial selector)
_SHELLS = [(1, "s"), (2, "s"), (2, "x"), (2, "y"), (2, "z"), (3, "s"), (3, "x"), (3, "y"), (3, "z")]


def trial_orbitals(points, Z, R, n_orb: int, width: float = 1.25):
    """Closed-form smooth trial orbitals (Gaussian-damped atomic-like shapes) evaluated at `points` [P,3].

    Orbital k sits on nucleus k mod M (nuclei ordered by decreasing charge) with shell k // M of the list
    above; the Gaussian width grows with the shell so that coarse meshes resolve the function.
    Returns (values [P, n_orb], guess eigenvalues [n_orb]).  They stand in for the coarse-mesh eigenpairs
    that the method takes as its starting point; they are not eigenfunctions of anything.
    """
    points = np.asarray(points, dtype=np.float64)
    order = np.argsort(-np.asarray(Z), kind="stable")
    M = len(Z)
    vals = np.zeros((points.shape[0], n_orb))
    lam = np.zeros(n_orb)
    for k in range(n_orb):
        m = order[k % M]
        nsh, kind = _SHELLS[min(k // M, len(_SHELLS) - 1)]
        w = width * (1.0 + 0.35 * (nsh - 1))
        d = points - R[m]
        r2 = np.sum(d * d, axis=1)
        g = np.exp(-0.5 * r2 / (w * w))
        if kind == "s":
            poly = 1.0 - (nsh - 1) * 0.5 * r2 / (w * w)
        else:
            poly = d[:, "xyz".index(kind)] / w
        vals[:, k] = poly * g
        lam[k] = -0.5 * Z[m] / (nsh * nsh) - 0.05 * k
    return vals, lam


def hydrogen():
    """One proton at the origin."""
    return np.array([1.0]), np.zeros((1, 3))


def lanczos_start(n: int, seed: int = 7) -> np.ndarray:
    """Seeded start vector for an extreme-eigenvalue Lanczos estimate."""
    return np.random.default_rng(seed).standard_normal(n)


def mlp_init(nloc: int, seed: int, nh: int = 64, out_scale: float = 0.1) -> np.ndarray:
    """Seeded initial parameters of the learned preconditioner's network, float32, flattened in the order
    W1 [nh][nloc+12], b1 [nh], W2 [nh][nh], b2 [nh], W3 [nloc][nh], b3 [nloc] (row-major): He-normal weights,
    zero biases, the last layer scaled by out_scale so that the untrained correction is small."""
    rng = np.random.default_rng(seed)
    nin, nout = nloc + 12, nloc
    W1 = rng.standard_normal((nh, nin)) * np.sqrt(2.0 / nin)
    W2 = rng.standard_normal((nh, nh)) * np.sqrt(2.0 / nh)
    W3 = rng.standard_normal((nout, nh)) * np.sqrt(2.0 / nh) * out_scale
    parts = [W1.ravel(), np.zeros(nh), W2.ravel(), np.zeros(nh), W3.ravel(), np.zeros(nout)]
    return np.concatenate(parts).astype(np.float32)


def workload(name: str, seed: int = 2000):
    """Named workloads of the paper's kind, with their sizes.

    'h_p1'  : hydrogen, box [-10,10]^3, P1, coarse 4^3 cubes, fine 16^3 cubes (24,576 tetrahedra).
    'mol4_p2': 4 nuclei (seed 2), box [-15,15]^3, P2, coarse 4^3 cubes, fine 32^3 cubes (196,608
               tetrahedra, 250,047 free fine DOF), N = ceil(sum Z / 2) <= 16, LDA.
    'mol4_p2_small': the same molecule on fine 8^3 cubes (parity-test size).
    'cluster12_p2': 12 nuclei (seed 5), box [-15,15]^3, P2, coarse 4^3 cubes, fine mesh graded toward the nuclei
               (graded_mesh, longest edge <= max(0.05, 0.3 r): about 0.87 M tetrahedra), N <= 48, LDA.
    'cluster12_p2_small': the same cluster graded with h_min = 1.5, alpha = 1.0 (9,782 tetrahedra).
    'mol8_p2'     : the evaluation molecules of the learned preconditioner: 8 nuclei (molecule(seed, 8), seeds
               2000-2015; `seed` picks one), box [-15,15]^3, P2, coarse 6^3 cubes (N_H = 1,331), fine 48^3 cubes
               (663,552 tetrahedra, 857,375 free DOF), N = ceil(sum Z / 2) <= 32, LDA.
    'mol8_p2_small': the same molecules on fine 12^3 cubes (10,368 tetrahedra, 12,167 free DOF).
    """
    if name == "h_p1":
        Z, R = hydrogen()
        return dict(name=name, Z=Z, R=R, order=1, half=10.0, n_coarse=4, levels=2, xc="slater")
    if name in ("mol4_p2", "mol4_p2_small", "mol4_p2_mid"):
        Z, R = molecule(2, 4)
        lv = {"mol4_p2": 3, "mol4_p2_mid": 2, "mol4_p2_small": 1}[name]
        return dict(name=name, Z=Z, R=R, order=2, half=15.0, n_coarse=4, levels=lv, xc="lda")
    if name in ("cluster12_p2", "cluster12_p2_small"):
        Z, R = molecule(5, 12)
        # nuclei on the lattice of the Kuhn mesh refined 6 times (spacing 30 / 4 / 64 = 0.117 bohr), so that the
        # graded mesh has a vertex at every nucleus and no quadrature point falls next to a Coulomb singularity
        step = 2 * 15.0 / 4 / 2 ** 6
        R = np.round(R / step) * step
        h_min, alpha = {"cluster12_p2": (0.05, 0.3), "cluster12_p2_small": (1.5, 1.0)}[name]
        return dict(name=name, Z=Z, R=R, order=2, half=15.0, n_coarse=4, mesh="graded", h_min=h_min, alpha=alpha,
                    xc="lda")
    if name in ("mol8_p2", "mol8_p2_small"):
        Z, R = molecule(seed, 8)
        return dict(name=name, Z=Z, R=R, order=2, half=15.0, n_coarse=6, levels=3 if name == "mol8_p2" else 1,
                    xc="lda", seed=seed)
    raise KeyError(name)


EVAL_SEEDS = tuple(range(2000, 2016))  # molecules the learned preconditioner is evaluated on (never trained on)


def workload_meshes(wl):
    """(coarse_coords, coarse_tets, fine_coords, fine_tets, fine_parent) of a workload: the uniformly refined cube
    meshes, or the mesh graded toward its nuclei."""
    if wl.get("mesh") == "graded":
        return graded_mesh(wl["n_coarse"], wl["half"], wl["R"], h_min=wl["h_min"], alpha=wl["alpha"])
    return nested_cube_meshes(wl["n_coarse"], wl["levels"], wl["half"])


def n_orbitals(Z) -> int:
    return int(math.ceil(float(np.sum(Z)) / 2.0))
