"""Training and use of the learned element-patch preconditioner through the C ABI.

The data come from the correction solves themselves: a problem of Algorithm 1, step 5 (frozen density, shifted
operator) is solved by plain FP64 PCG with its iterates traced; every traced iterate x_k with residual r_k and
the converged x* gives one sample per (element, orbital) (mk_mlp_harvest).  Training draws seeded minibatches of
those samples and takes Adam steps (mk_mlp_train_step).  Every computation runs in the CUDA library; this module
only allocates device buffers (torch) and passes pointers.
"""
from __future__ import annotations

import numpy as np

from . import mk, synth


class Problem:
    """One correction boundary-value problem on `mesh` for the molecule (Z, R): the library's own stages give
    the coarse eigenpairs, the shift sigma (60 Lanczos steps), the Hartree potential and the right-hand side."""

    def __init__(self, ctx, mesh, Z, R, xc="lda", lanczos_seed=7):
        import torch
        from .step import coarse_eigenpairs
        self.ctx, self.mesh, self.Z, self.R = ctx, mesh, np.asarray(Z, float), np.asarray(R, float)
        info = mesh.info
        self.N = synth.n_orbitals(self.Z)
        self.ld = 4 if self.N <= 4 else 8 if self.N <= 8 else 16 if self.N <= 16 else (self.N + 3) // 4 * 4
        self.mol = mk.Molecule(self.Z, self.R)
        occ = synth.occupations(self.Z)
        _, self.sigma = mk.mk_correction_shift(ctx, mesh, self.mol, synth.lanczos_start(info["n_free"], lanczos_seed),
                                               steps=60)
        psiH, lamH = coarse_eigenpairs(ctx, mesh, self.Z, self.R, self.N)
        f64 = dict(dtype=torch.float64, device="cuda")
        n, NH = info["n_nodes"], info["n_free_coarse"]
        ph = torch.zeros((NH, self.ld), **f64)
        ph[:, : self.N] = torch.from_numpy(psiH).cuda()
        self.u = torch.zeros((n, self.ld), **f64)
        w = torch.zeros(n, **f64)
        self.rhs = torch.zeros((n, self.ld), **f64)
        vq = torch.zeros((info["n_elems"], info["n_quad"]), **f64)
        mk.mk_prolongate(ctx, mesh, ph, self.N, self.u)
        mk.mk_hartree_poisson(ctx, mesh, self.u, occ, self.N, w, opt=mk.opts(rtol=1e-10))
        mk.mk_assemble_rhs(ctx, mesh, self.u, lamH, occ, self.N, w, self.sigma, xc, self.rhs, vq)
        torch.cuda.synchronize()

    def solve(self, opt, x0=None):
        """Solves from x0 (default: the prolonged coarse orbitals); returns (x, report)."""
        x = (self.u if x0 is None else x0).clone()
        rep = mk.mk_correction_solve(self.ctx, self.mesh, self.mol, self.sigma, self.rhs, x, self.N, opt=opt)
        return x, rep


def harvest(problem: Problem, every=2, cap=12, rtol=1e-10):
    """Samples (X [S, n_in], U [S], E [S, n_loc], device float32) from a traced FP64 PCG solve of `problem`."""
    import torch
    info = problem.mesh.info
    n, ld, N = info["n_nodes"], problem.ld, problem.N
    f64 = dict(dtype=torch.float64, device="cuda")
    xb, rb = torch.zeros((cap, n, ld), **f64), torch.zeros((cap, n, ld), **f64)
    xs, rep = problem.solve(mk.opts(precision="fp64", rtol=rtol, trace=(every, xb, rb)))
    k = rep["n_traced"]
    E, nloc = info["n_elems"], info["nloc"]
    f32 = dict(dtype=torch.float32, device="cuda")
    X = torch.empty((k, E * N, nloc + 12), **f32)
    U = torch.empty((k, E * N), **f32)
    Er = torch.empty((k, E * N, nloc), **f32)
    for i in range(k):
        mk.mk_mlp_harvest(problem.ctx, problem.mesh, rb[i], xb[i], xs, N, X[i], U[i], Er[i])
    torch.cuda.synchronize()
    return X.reshape(-1, nloc + 12), U.reshape(-1), Er.reshape(-1, nloc)


def train(ctx, mlp: "mk.Mlp", X, U, E, steps=2000, batch=8192, lr=1e-3, seed=0, log_every=0):
    """Adam on seeded minibatches (indices drawn on the host, copied as int32).  Returns the loss history."""
    import torch
    rng = np.random.default_rng(seed)
    S = X.shape[0]
    hist = []
    for step in range(steps):
        idx = torch.from_numpy(rng.integers(0, S, size=batch).astype(np.int32)).cuda()
        loss = mk.mk_mlp_train_step(ctx, mlp, X, U, E, idx=idx, lr=lr)
        hist.append(loss)
        if log_every and step % log_every == 0:
            print(f"train step {step} loss {loss:.6g}", flush=True)
    return hist
