"""One fine-mesh correction step (Algorithm 1, steps 5-7, frozen V_Hxc(rho_H) on the right) through the C ABI.

Holds device buffers for one mesh pair and chains mk_prolongate -> mk_hartree_poisson -> mk_assemble_rhs ->
mk_correction_solve -> mk_augmented_project -> mk_small_eigensolve -> mk_orbital_assemble.  Every step runs in the
CUDA library; this class only allocates the caller-owned device arrays (torch) and passes pointers.
"""
from __future__ import annotations

import numpy as np

from . import mk


class CorrectionStep:
    def __init__(self, ctx: "mk.Context", mesh: "mk.Mesh", Z, R, N: int, ld: int | None = None,
                 overlap: bool = True, basis=None):
        """basis: optional M_H-orthonormal device matrix [N_H, N_H] (eigenvectors of the density-independent
        coarse pencil) from which the coarse decomposition is warm-started."""
        import torch
        self.ctx, self.mesh, self.N = ctx, mesh, N
        self.overlap = overlap
        self.basis = basis
        if overlap:
            self._side = torch.cuda.Stream()
            self._ev_rhs = torch.cuda.Event()
            self._ev_dec = torch.cuda.Event()
        self.ld = ld or max(4, (N + 3) // 4 * 4)
        self.mol = mk.Molecule(Z, R)
        info = mesh.info
        n, E, NH = info["n_nodes"], info["n_elems"], info["n_free_coarse"]
        self.NH = NH
        dev = torch.device("cuda")
        f64 = dict(dtype=torch.float64, device=dev)
        self.u = torch.zeros((n, self.ld), **f64)
        self.w = torch.zeros(n, **f64)
        self.rhs = torch.zeros((n, self.ld), **f64)
        self.vq = torch.zeros((E, info["n_quad"]), **f64)
        self.rho = torch.zeros((E, info["n_quad"]), **f64)  # rho_H at the quadrature points
        self.psihat = torch.zeros((n, self.ld), **f64)
        self.AH = torch.zeros((NH, NH), **f64)
        self.MH = torch.zeros((NH, NH), **f64)
        self.b = torch.zeros((NH, N), **f64)
        self.c = torch.zeros((NH, N), **f64)
        self.beta = torch.zeros(N, **f64)
        self.gamma = torch.zeros(N, **f64)
        self.gramA = torch.zeros((N, N), **f64)
        self.gramM = torch.zeros((N, N), **f64)
        self.d = torch.zeros(NH, **f64)
        self.V = torch.zeros((NH, NH), **f64)
        self.lam = torch.zeros(N, **f64)
        self.coef = torch.zeros((NH + 1, N), **f64)
        self.status = torch.zeros(N, dtype=torch.int32, device=dev)
        self.psi = torch.zeros((n, self.ld), **f64)
        self.psiH = torch.zeros((NH, self.ld), **f64)

    def _decompose(self, stream):
        if self.basis is not None:
            mk.mk_coarse_decompose_warm(self.ctx, self.NH, self.AH, self.basis, self.d, self.V, stream=stream)
        else:
            mk.mk_coarse_decompose(self.ctx, self.mesh, self.AH, self.d, self.V, stream=stream)

    def run(self, psiH, lamH, occ, sigma, xc="lda", hartree_bc="multipole", solve_opts=None, poisson_opts=None,
            stream=None):
        """psiH: torch [N_H, >=N] (device) or numpy [N_H, N]; lamH, occ: numpy [N].  Returns reports."""
        import torch
        N = self.N
        if isinstance(psiH, np.ndarray):
            self.psiH.zero_()
            self.psiH[:, :N] = torch.from_numpy(psiH).to(self.psiH.device)
            psiH = self.psiH
        ctx, mesh = self.ctx, self.mesh
        mk.mk_prolongate(ctx, mesh, psiH, N, self.u, stream=stream)
        # rho_H at the quadrature points, once for the Poisson solve and the frozen potential
        mk.mk_density(ctx, mesh, self.u, occ, N, self.rho, stream=stream)
        reps = {}
        if hartree_bc == "none":
            self.w.zero_()
            reps["poisson"] = None
        else:
            reps["poisson"] = mk.mk_hartree_poisson(ctx, mesh, self.u, occ, N, self.w, bc=hartree_bc,
                                                    opt=poisson_opts, stream=stream, rho_q=self.rho)
        # A3 in two halves: the frozen potential vq first, so that the coarse pencil and its decomposition (which
        # need vq, not rhs or psi^) start on the side stream while the right-hand sides and the fine solve run
        mk.mk_frozen_potential(ctx, mesh, self.u, occ, N, self.w, xc, self.vq, stream=stream, rho_q=self.rho)
        main = torch.cuda.current_stream() if stream is None else torch.cuda.ExternalStream(stream)
        if self.overlap:
            self._ev_rhs.record(main)
            self._side.wait_event(self._ev_rhs)
            mk.mk_coarse_pencil(ctx, mesh, self.mol, self.vq, self.AH, None, stream=self._side.cuda_stream)
            self._decompose(self._side.cuda_stream)
            self._ev_dec.record(self._side)
        mk.mk_assemble_rhs_from_vq(ctx, mesh, self.u, lamH, N, self.vq, sigma, self.rhs, stream=stream)
        self.psihat.copy_(self.u)
        reps["solve"] = mk.mk_correction_solve(ctx, mesh, self.mol, sigma, self.rhs, self.psihat, N,
                                               opt=solve_opts, stream=stream)
        if not self.overlap:
            mk.mk_coarse_pencil(ctx, mesh, self.mol, self.vq, self.AH, None, stream=stream)
            self._decompose(stream)
        mk.mk_augmented_project(ctx, mesh, self.mol, self.vq, self.psihat, N, None, None, self.b, self.c,
                                self.beta, self.gamma, self.gramA, self.gramM, stream=stream)
        if self.overlap:
            main.wait_event(self._ev_dec)
        mk.mk_small_eigensolve_shared(ctx, self.NH, N, self.d, self.V, self.b, self.c, self.beta, self.gamma,
                                      self.lam, self.coef, self.status, stream=stream)
        mk.mk_orbital_assemble(ctx, mesh, self.coef, self.psihat, self.u, N, self.psi, stream=stream)
        return reps


def coarse_eigenpairs(ctx, mesh, Z, R, N, return_basis=False):
    """Lowest N eigenpairs of the bare coarse Hamiltonian P^T (K/2 + M_Vext) P in V_H, the frozen-potential version
    of Algorithm 1, step 1 (the initial solve on the coarse space), on the GPU.  Returns numpy (psiH, lamH), and
    with return_basis also the full M_H-orthonormal eigenbasis as a device tensor (a warm start for the step's
    coarse decomposition)."""
    import torch
    mol = mk.Molecule(Z, R)
    NH = mesh.info["n_free_coarse"]
    f64 = dict(dtype=torch.float64, device="cuda")
    AH, MH, d, V = (torch.zeros((NH, NH), **f64), torch.zeros((NH, NH), **f64), torch.zeros(NH, **f64),
                    torch.zeros((NH, NH), **f64))
    mk.mk_coarse_pencil(ctx, mesh, mol, None, AH, MH)
    mk.mk_coarse_decompose(ctx, mesh, AH, d, V)
    torch.cuda.synchronize()
    out = (V[:, :N].cpu().numpy().copy(), d[:N].cpu().numpy().copy())
    return out + (V,) if return_basis else out


def upload_workload(ctx, wl, hierarchy=True):
    """Meshes of a named synthetic workload (see synth.workload) uploaded to the device, with the intermediate levels
    of the multigrid hierarchy (mesh.multigrid True): the coarser cube meshes for the uniformly refined workloads,
    refinement passes about 4x apart in size for the graded ones."""
    from . import synth
    graded = wl.get("mesh") == "graded"
    snaps = [] if (graded and hierarchy) else None
    if graded:
        cc, ct, fc, ft, par = synth.graded_mesh(wl["n_coarse"], wl["half"], wl["R"], h_min=wl["h_min"],
                                                alpha=wl["alpha"], snapshots=snaps)
    else:
        cc, ct, fc, ft, par = synth.workload_meshes(wl)
    mesh = mk.Mesh(ctx, fc, ft, cc, ct, par, wl["order"])
    mesh.multigrid = False
    if hierarchy:
        levels = synth.hierarchy_from_snapshots(snaps) if graded else \
            synth.cube_hierarchy(wl["n_coarse"], wl["levels"], wl["half"])
        if levels[0]:
            mesh.set_hierarchy(*levels)
            mesh.multigrid = True
    return mesh, (cc, ct, fc, ft, par)


class PaperStep:
    """The correction step in the paper's own form (Algorithm 1, steps 5-7, with Algorithm 2's inner iteration and
    Algorithm 3's precomputations), through the C ABI: the frozen potential w_prev + V_xc(rho^l) of the step's input
    orbitals on the left of the correction problems (mk_correction_solve_vq), the Hartree potential w~ of the
    corrections' density (mk_hartree_poisson), then the nonlinear eigenproblem in V_H + span{phi~_i} by the inner
    SCF (mk_inner_*).  Buffers are device tensors owned here."""

    def __init__(self, ctx, mesh, Z, R, N: int, ld: int | None = None):
        import torch
        self.ctx, self.mesh, self.N = ctx, mesh, N
        self.ld = ld or max(4, (N + 3) // 4 * 4)
        self.mol = mk.Molecule(Z, R)
        info = mesh.info
        n, E, NH = info["n_nodes"], info["n_elems"], info["n_free_coarse"]
        self.NH = NH
        f64 = dict(dtype=torch.float64, device=torch.device("cuda"))
        self.u = torch.zeros((n, self.ld), **f64)
        self.zero_n = torch.zeros(n, **f64)
        self.zero_q = torch.zeros((E, info["n_quad"]), **f64)
        self.vq = torch.zeros((E, info["n_quad"]), **f64)       # w_prev + V_xc(rho^l): the operator's potential
        self.vxc = torch.zeros((E, info["n_quad"]), **f64)      # V_xc(rho^l) alone
        self.rhs = torch.zeros((n, self.ld), **f64)
        self.phit = torch.zeros((n, self.ld), **f64)
        self.wt = torch.zeros(n, **f64)
        self.lam = torch.zeros(N, **f64)
        self.coef = torch.zeros((NH + 1, N), **f64)
        self.status = torch.zeros(N, dtype=torch.int32, device=f64["device"])
        self.wH = torch.zeros(NH, **f64)
        self.w = torch.zeros(n, **f64)
        self.psi = torch.zeros((n, self.ld), **f64)
        self.inner = None

    def run(self, U, lam, occ, sigma, w_prev, xc="lda", solve_opts=None, poisson_opts=None, inner_tol=1e-10,
            max_inner=200, mix=0.5, stream=None):
        """U: device [n_nodes, >=N] or numpy [n_nodes, N] (the step's input orbitals on the fine mesh); lam, occ:
        numpy [N]; w_prev: device or numpy [n_nodes].  Returns reports."""
        import torch
        N = self.N
        if isinstance(U, np.ndarray):
            self.u.zero_()
            self.u[:, :N] = torch.from_numpy(U).to(self.u.device)
        elif U is not self.u:
            self.u.copy_(U)
        if isinstance(w_prev, np.ndarray):
            w_prev = torch.from_numpy(np.ascontiguousarray(w_prev)).to(self.u.device)
        ctx, mesh = self.ctx, self.mesh
        mk.mk_frozen_potential(ctx, mesh, self.u, occ, N, w_prev, xc, self.vq, stream=stream)
        mk.mk_frozen_potential(ctx, mesh, self.u, occ, N, self.zero_n, xc, self.vxc, stream=stream)
        # step 5: (K/2 + V_ext + w_prev + V_xc + sigma) phi~_i = (lambda_i + sigma) M u_i
        mk.mk_assemble_rhs_from_vq(ctx, mesh, self.u, lam, N, self.zero_q, sigma, self.rhs, stream=stream)
        self.phit.copy_(self.u)
        reps = {"solve": mk.mk_correction_solve_vq(ctx, mesh, self.mol, self.vq, sigma, self.rhs, self.phit, N,
                                                   opt=solve_opts, stream=stream)}
        # step 6: the Hartree potential of the corrections' density
        reps["poisson"] = mk.mk_hartree_poisson(ctx, mesh, self.phit, occ, N, self.wt, bc="multipole",
                                                opt=poisson_opts, stream=stream)
        # step 7: Algorithm 3's precomputations, then Algorithm 2's inner iteration
        if self.inner is not None:
            self.inner.close()
        self.inner = mk.Inner(ctx, mesh, self.mol, self.phit, N, self.wt, self.vxc, stream=stream)
        reps["inner"] = self.inner.run(occ, self.lam, self.coef, self.status, self.wH, tol=inner_tol,
                                       max_inner=max_inner, mix=mix, stream=stream)
        mk.mk_orbital_assemble(ctx, mesh, self.coef, self.phit, self.phit, N, self.psi, stream=stream)
        self.inner.potential(self.w, stream=stream)
        return reps

    def close(self):
        if self.inner is not None:
            self.inner.close()
            self.inner = None
