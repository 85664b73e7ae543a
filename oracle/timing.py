"""Times the oracle's correction step on a workload (test infrastructure: used by bench.py's cpu_baseline and
--impl reference legs only).  Run as `python -m oracle.timing <workload> <steps> <warmup>` in a fresh process; prints
one JSON line.  The oracle is timed as it stands: assembled scipy.sparse matrices, plain Jacobi-PCG, dense
LAPACK eigensolves.  Static assembly (K, M, M_Vext, P) is done once before timing, as the GPU path's mesh upload
is; everything that depends on the density is inside every timed step."""
from __future__ import annotations

import json
import os
import sys
import time


def main():
    name = sys.argv[1]
    steps = int(sys.argv[2])
    warmup = int(sys.argv[3])
    import numpy as np
    import scipy.linalg as sla
    from oracle.correction import Level, correction_step
    from oracle.fem import coulomb
    from oracle import linalg as olin
    from paper_2103_02824_gb300 import synth
    wl = synth.workload(name)
    cc, ct, fc, ft, par = synth.workload_meshes(wl)
    t0 = time.perf_counter()
    lv = Level(cc, ct, fc, ft, par, wl["order"], wl["Z"], wl["R"])
    t_setup = time.perf_counter() - t0
    N = synth.n_orbitals(wl["Z"])
    occ = synth.occupations(wl["Z"])
    # inputs: lowest coarse eigenpairs of the Galerkin bare Hamiltonian (as the GPU bench's setup computes them)
    Hff = (0.5 * lv.Kff + lv.MVff).tocsr()
    AH = (lv.Pf.T @ (Hff @ lv.Pf)).toarray()
    MH = (lv.Pf.T @ (lv.Mff @ lv.Pf)).toarray()
    lamH, V = sla.eigh(AH, MH)
    psiH, lamH = V[:, :N], lamH[:N]
    if len(sys.argv) > 4:        # the shift the GPU run used (same input on both sides)
        sigma = float(sys.argv[4])
    else:
        theta = olin.lanczos_lowest(Hff, lv.Mff, synth.lanczos_start(lv.fine.n_free), steps=60)
        sigma = olin.shift_rule(theta)
    times = []
    res = None
    for k in range(warmup + steps):
        t0 = time.perf_counter()
        out = correction_step(lv, psiH, lamH, occ, sigma, xc=wl["xc"], hartree_bc="multipole", tol=1e-8)
        dt = time.perf_counter() - t0
        if k >= warmup:
            times.append(dt)
        res = out
    threads = int(os.environ.get("OMP_NUM_THREADS", "0") or 0) or os.cpu_count()
    print(json.dumps(dict(workload=name, n_free=int(lv.fine.n_free), n_elems=int(lv.fine.n_elems),
                          n_free_coarse=int(lv.coarse.n_free), N=N, sigma=sigma, setup_s=t_setup,
                          step_s=times, lam=[float(x) for x in res["lam"]],
                          cg_iters=[int(x) for x in res["cg_iters"]], poisson_iters=res["poisson"]["iters"],
                          threads=threads)))


if __name__ == "__main__":
    main()
