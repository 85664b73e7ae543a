"""Shared parity cases: synthetic inputs and the oracle's results on them (computed once per process)."""
import functools

import numpy as np
import scipy.linalg as sla

from oracle import linalg as olin
from oracle.correction import Level, correction_step
from oracle.fem import coulomb
from oracle.poisson import density_at_quad
from oracle.xc import v_xc
from paper_2103_02824_gb300 import synth


def coarse_eigs(lv, k):
    C = lv.coarse
    xq, _, _, _ = C.quad()
    A = (0.5 * C.assemble(C.element_stiffness()) + C.assemble(C.element_mass(coulomb(xq, lv.Z, lv.R))))
    A = A[C.free][:, C.free].toarray()
    M = C.assemble(C.element_mass())[C.free][:, C.free].toarray()
    lam, V = sla.eigh(A, M)
    return lam[:k], V[:, :k]


@functools.lru_cache(maxsize=None)
def case(name: str, trial: bool = False):
    """Oracle level + inputs + full oracle step for a named workload.  trial=True uses the closed-form trial
    orbitals of synth instead of coarse eigenvectors."""
    wl = synth.workload(name)
    cc, ct, fc, ft, par = synth.workload_meshes(wl)
    lv = Level(cc, ct, fc, ft, par, wl["order"], wl["Z"], wl["R"])
    N = synth.n_orbitals(wl["Z"])
    occ = synth.occupations(wl["Z"])
    if trial:
        vals, lamH = synth.trial_orbitals(lv.coarse.nodes[lv.coarse.free], wl["Z"], wl["R"], N)
        psiH = vals
    else:
        lamH, psiH = coarse_eigs(lv, N)
    H = (0.5 * lv.Kff + lv.MVff).tocsr()
    v0 = synth.lanczos_start(lv.fine.n_free)
    theta = olin.lanczos_lowest(H, lv.Mff, v0, steps=60)
    sigma = olin.shift_rule(theta)
    xc = wl["xc"]
    out = correction_step(lv, psiH, lamH, occ, sigma, xc=xc, hartree_bc="multipole", tol=1e-13)
    rho = density_at_quad(lv.fine, out["u"], occ)
    vq = lv.fine.eval_at_quad(out["w"]) + v_xc(rho, xc)
    return dict(wl=wl, meshes=(cc, ct, fc, ft, par), level=lv, N=N, occ=occ, psiH=np.ascontiguousarray(psiH),
                lamH=np.asarray(lamH), sigma=sigma, theta=theta, v0=v0, xc=xc, out=out, vq=vq)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def maxrel(a, b):
    """Element-wise: max |a - b| over all entries, relative to max |b| (a local error cannot hide under a norm)."""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
