"""Benchmark of the fine-mesh correction step (all hot-path rows A1-A8) on the GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mk|reference] [--workload mol4_p2]
                [--precision mixed|fp64] [--precond learned|jacobi]

Metric: fine-mesh DOF x orbitals solved per second at 1e-8 FP64 relative residual, i.e. n_free * N per step time,
where one step = prolongation, Hartree Poisson solve, RHS, correction solve, coarse pencil + decomposition,
augmented projection, small eigensolves and orbital assembly, with inputs resident in HBM.  The working set of a
step (fine-mesh element matrices and vectors, several hundred MB) is larger than the 129 MB L2.

The headline `value` is the fastest form of the step: mixed precision (FP32 operator, FP64 refinement) with Jacobi
PCG; `compare` times the same step with the learned preconditioner (BF16 network on tcgen05, FCG(1)) and with
plain FP64 PCG, and `learned_vs_plain` compares the learned and plain solves on the 8-nucleus evaluation molecules.
The network is trained before any timing on correction solves of other seeded molecules.

--gpus N > 1 (torchrun): replicas only -- each rank solves its own copy of the workload, no collective on the data
path; value = all ranks' units / max over ranks of the timed region.
--impl reference: the CPU FP64 oracle on the host cores (rank 0 only), same workload, metric and unit.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fine-mesh DOF×orbitals solved/s at 1e-8 rel. residual; learned vs plain PCG"
# dram__bytes_read.sum + dram__bytes_write.sum of one k_apply_stream launch from an ncu capture of the same kernel
# build on the same workload (None until such a capture exists for the current kernel)
TRAFFIC = {("mol4_p2", 8): 68.16e6}  # ncu: 66.19 MB read + 1.97 MB written by one k_apply_reg launch on mol4_p2
UNIT = "DOF*orbitals/s"
OPERATOR_KERNEL = "k_apply_reg (FP32 element-by-element operator: element matrices staged in registers)"
# FP64 FMA rate of the GB300: 152 SMs x 2 FP64 FMA per clock x 2 flops x 2.07 GHz (maximum SM clock)
FP64_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP64_NOTE = "152 SMs x 2 FMA/clock x 2 flop x 2.07 GHz = 1.26 TFLOP/s; a probe measured 1.196"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mk", choices=["mk", "reference"])
    ap.add_argument("--workload", default="mol4_p2")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--precond", default="jacobi", choices=["learned", "jacobi"],
                    help="inner preconditioner of the headline mixed-precision correction solve (learned: FCG(1))")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip training the network (and so the learned form in compare and learned_vs_plain)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-solve measurement")
    ap.add_argument("--no-paper", action="store_true", help="skip the paper-form step (inner SCF) measurement")
    ap.add_argument("--no-eval", action="store_true",
                    help="skip the learned-vs-plain evaluation on the 16 unseen 8-nucleus molecules")
    ap.add_argument("--patch-kernel", default="reg", choices=["reg", "pipelined", "single"],
                    help="--mode apply: the FP32 register-staged kernel (default), the two-group pipelined kernel, "
                         "or the one-patch-per-CTA kernel")
    ap.add_argument("--mode", default="step", choices=["step", "apply", "learned", "stiffness", "decompose", "serve"],
                    help="apply: time the FP32 element-by-element operator alone (kernel-level roofline); "
                         "learned: the learned preconditioner (BF16 network) alone; stiffness: the matrix-free "
                         "Poisson operator K alone (one column); decompose: the warm coarse decomposition of the "
                         "step's pencil alone")
    return ap.parse_args()


def apply_mode(a):
    """Times mk_operator_apply's FP32 patch operator (y = A x, all orbital columns) on the workload's mesh."""
    import torch
    from paper_2103_02824_gb300 import build, mk, synth
    from paper_2103_02824_gb300.step import upload_workload
    build.build()
    wl = synth.workload(a.workload)
    ctx = mk.Context(0)
    mesh, _ = upload_workload(ctx, wl)
    info = mesh.info
    N = synth.n_orbitals(wl["Z"])
    ld = max(4, (N + 3) // 4 * 4)
    mol = mk.Molecule(wl["Z"], wl["R"])
    mk.ctx_set_option(ctx, mk.MK_OPT_PATCH_PIPELINE, {"reg": 1, "pipelined": 2, "single": 0}[a.patch_kernel])
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn((info["n_nodes"], ld), generator=g, device="cuda", dtype=torch.float32)
    y = torch.empty_like(x)
    for _ in range(a.warmup):
        mk.mk_operator_apply(ctx, mesh, mol, 18.0, x, y)
    mk.profile_enable(ctx, True)
    torch.cuda.synchronize()
    for _ in range(a.steps):
        mk.mk_operator_apply(ctx, mesh, mol, 18.0, x, y)
    torch.cuda.synchronize()
    ms, n = mk.profile_read(ctx, mk.PROF_APPLY32)
    hms, hn = mk.profile_read(ctx, mk.PROF_HALO)
    nloc, E = info["nloc"], info["n_elems"]
    npack = nloc * (nloc + 1) // 2
    nbytes = 2.0 * info["n_nodes"] * ld * 4 + E * (npack * 4 + nloc * 4 + 2 * nloc)
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6780.7) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6780.7
    gbs = nbytes / (ms / n * 1e-3) / 1e9
    print(json.dumps({"mode": "apply", "kernel": a.patch_kernel, "workload": a.workload, "ld": ld, "applications": n,
                      "patch_ms": ms / n, "halo_ms": hms / max(hn, 1), "bytes_per_application": nbytes,
                      "achieved_gbs": gbs, "peak_gbs": peak, "frac": gbs / peak}))


def learned_mode(a):
    """Times mk_learned_precond (BF16 tensor-core network, untrained seeded weights) on the workload's mesh."""
    import torch
    from paper_2103_02824_gb300 import build, mk, synth
    from paper_2103_02824_gb300.step import upload_workload
    build.build()
    wl = synth.workload(a.workload)
    ctx = mk.Context(0)
    mesh, _ = upload_workload(ctx, wl)
    info = mesh.info
    N = synth.n_orbitals(wl["Z"])
    ld = max(4, (N + 3) // 4 * 4)
    mol = mk.Molecule(wl["Z"], wl["R"])
    mlp = mk.Mlp(ctx, info["nloc"], synth.mlp_init(info["nloc"], 0))
    g = torch.Generator(device="cuda").manual_seed(5)
    r = torch.randn((info["n_nodes"], ld), generator=g, device="cuda", dtype=torch.float32)
    z = torch.empty_like(r)
    for _ in range(a.warmup):
        mk.mk_learned_precond(ctx, mesh, mlp, mol, 18.0, r, z, N)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        mk.mk_learned_precond(ctx, mesh, mlp, mol, 18.0, r, z, N)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.steps
    rows = info["n_elems"] * N
    flops = 2.0 * (22 * 64 + 64 * 64 + 64 * 10) * rows if info["nloc"] == 10 else 2.0 * (16 * 64 + 64 * 64 + 64 * 4) * rows
    print(json.dumps({"mode": "learned", "workload": a.workload, "N": N, "ms_per_application": ms,
                      "note": "includes the operator diagonal (element matrices + assembly) recomputed per call",
                      "network_tflops": flops / (ms * 1e-3) / 1e12}))


def stiffness_mode(a):
    """Times mk_operator_apply with no molecule: the matrix-free FP32 stiffness operator K on one column."""
    import torch
    from paper_2103_02824_gb300 import build, mk, synth
    from paper_2103_02824_gb300.step import upload_workload
    build.build()
    wl = synth.workload(a.workload)
    ctx = mk.Context(0)
    mesh, _ = upload_workload(ctx, wl)
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn(mesh.info["n_nodes"], generator=g, device="cuda", dtype=torch.float32)
    y = torch.empty_like(x)
    for _ in range(a.warmup):
        mk.mk_operator_apply(ctx, mesh, None, 0.0, x, y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        mk.mk_operator_apply(ctx, mesh, None, 0.0, x, y)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"mode": "stiffness", "workload": a.workload, "ms_per_application": e0.elapsed_time(e1) / a.steps,
                      "note": "stiffness kernel and halo pass"}))


def decompose_mode(a):
    """Times the warm coarse decomposition (block Jacobi) of the step's coarse pencil alone: one Jacobi-form step
    fills A_H, then the decomposition is repeated on it."""
    import torch
    from paper_2103_02824_gb300 import build, mk, synth
    from paper_2103_02824_gb300.step import CorrectionStep, coarse_eigenpairs, upload_workload
    build.build()
    wl = synth.workload(a.workload)
    ctx = mk.Context(0)
    mesh, _ = upload_workload(ctx, wl)
    N, occ = synth.n_orbitals(wl["Z"]), synth.occupations(wl["Z"])
    psiH, lamH, basis = coarse_eigenpairs(ctx, mesh, wl["Z"], wl["R"], N, return_basis=True)
    st = CorrectionStep(ctx, mesh, wl["Z"], wl["R"], N, overlap=False, basis=basis)
    _, sigma = mk.mk_correction_shift(ctx, mesh, st.mol, synth.lanczos_start(mesh.info["n_free"]), steps=60)
    st.run(psiH, lamH, occ, sigma, xc=wl["xc"], hartree_bc="multipole",
           solve_opts=mk.opts(precision="mixed", precond="jacobi", rtol=1e-8, check_every=10),
           poisson_opts=mk.opts(precision="mixed", rtol=1e-8, check_every=10, coarse=True))
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(a.warmup):
        st._decompose(stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        st._decompose(stream)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"mode": "decompose", "workload": a.workload, "N_H": st.NH,
                      "ms_per_decomposition": e0.elapsed_time(e1) / a.steps}))


def eval_learned(ctx, mlp, max_molecules=16):
    """The learned preconditioner against plain PCG on the molecules it is evaluated on (never trained on): the
    correction solves of 16 seeded 8-nucleus molecules on the 857,375-DOF P2 mesh (fine 48^3 cubes of [-15,15]^3,
    coarse 6^3), N = 13-25 orbitals, to 1e-8 FP64 relative residual, each molecule in four forms: mixed precision
    with the learned FCG(1), mixed precision with Jacobi PCG, plain FP64 Jacobi PCG, plain FP64 PCG with the
    degree-4 Chebyshev preconditioner.  One timed solve per molecule and form (CUDA events), after one untimed solve
    of each form on the first molecule.  Returns DOF x orbitals / s over all molecules per form, with iterations."""
    import numpy as np
    import torch
    from paper_2103_02824_gb300 import learned, mk, synth
    from paper_2103_02824_gb300.step import upload_workload
    t0 = time.perf_counter()
    mesh, _ = upload_workload(ctx, synth.workload("mol8_p2"))
    forms = {"learned_mixed": mk.opts(precision="mixed", precond="learned", mlp=mlp, rtol=1e-8, check_every=10),
             "jacobi_mixed": mk.opts(precision="mixed", precond="jacobi", rtol=1e-8, check_every=10),
             "jacobi_fp64": mk.opts(precision="fp64", precond="jacobi", rtol=1e-8, check_every=10),
             "chebyshev_fp64": mk.opts(precision="fp64", precond="chebyshev", rtol=1e-8, check_every=10)}
    res = {k: {"ms": 0.0, "units": 0.0, "iterations": []} for k in forms}
    Ns = []
    n_free = mesh.info["n_free"]
    for i, seed in enumerate(synth.EVAL_SEEDS[:max_molecules]):
        prob = learned.Problem(ctx, mesh, *synth.molecule(seed, 8))
        Ns.append(prob.N)
        for name, o in forms.items():
            if i == 0:
                prob.solve(o)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, rep = prob.solve(o)
            e1.record()
            torch.cuda.synchronize()
            assert rep["max_rel_residual"] <= 1e-8, (name, seed, rep["max_rel_residual"])
            r = res[name]
            r["ms"] += e0.elapsed_time(e1)
            r["units"] += float(n_free) * prob.N
            r["iterations"].append(rep["iterations"])
        del prob
    mesh.close()
    out = {"workload": f"mol8_p2: synthetic 8-nucleus molecules synth.molecule(seed, 8), seeds "
                       f"{synth.EVAL_SEEDS[0]}-{synth.EVAL_SEEDS[max_molecules - 1]}, P2 tetrahedra, box [-15,15]^3, "
                       f"fine 48^3 cubes (663,552 tets, {n_free} free DOF), coarse 6^3 cubes (N_H=1331), LDA",
           "orbitals": Ns, "rtol": 1e-8, "unit": UNIT, "seconds": time.perf_counter() - t0}
    for name, r in res.items():
        out[name] = {"value": r["units"] / (r["ms"] * 1e-3), "ms_total": r["ms"],
                     "mean_iterations": float(np.mean(r["iterations"])), "iterations": r["iterations"]}
    out["learned_over_jacobi_mixed"] = out["learned_mixed"]["value"] / out["jacobi_mixed"]["value"]
    out["learned_over_jacobi_fp64"] = out["learned_mixed"]["value"] / out["jacobi_fp64"]["value"]
    return out


def whole_job_ms(ms, dist, device):
    """The timed region of the whole job: the largest of the ranks' own durations (ms), since the job ends when its
    slowest rank does; ms itself on one rank (dist None)."""
    if dist is None:
        return ms
    import torch
    tt = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def workload_config(wl, N, n_free, NH, E):
    Z = ",".join(str(int(z)) for z in wl["Z"])
    if wl.get("mesh") == "graded":
        fine = (f"fine mesh bisected toward the nuclei to longest edge <= max({wl['h_min']:g}, {wl['alpha']:g} r) "
                f"({E} tets, {n_free} free DOF)")
        mol = f"synthetic {len(wl['Z'])}-nucleus cluster (seed 5, Z={Z})"
    else:
        fine = f"fine {wl['n_coarse'] * 2 ** wl['levels']}^3 cubes ({E} tets, {n_free} free DOF)"
        mol = f"synthetic {len(wl['Z'])}-nucleus molecule (seed 2, Z={Z})"
    return {
        "workload": f"{wl['name']}: {mol}, P{wl['order']} tetrahedra, box [-{wl['half']:g},{wl['half']:g}]^3, "
                    f"{fine}, coarse {wl['n_coarse']}^3 cubes (N_H={NH}), N={N} orbitals, {wl['xc'].upper()}, "
                    f"multipole Hartree BC",
        "n_free": n_free, "orbitals": N, "N_H": NH,
    }


def host_cpu():
    """The host's CPU model (lscpu) and core count, recorded beside the CPU baseline."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"model": model, "nproc": os.cpu_count(), "threads_used": 1}


def run_oracle(workload, steps, warmup, sigma=None, timeout=1800):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1", PYTHONPATH=ROOT)
    cmd = [sys.executable, "-m", "oracle.timing", workload, str(steps), str(warmup)]
    if sigma is not None:
        cmd.append(repr(float(sigma)))
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError("oracle timing failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.dev = device_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        smax = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": reasons, "samples": len(rows)}


TRAIN_SEEDS = tuple(range(1000, 1064))  # 64 seeded 4-nucleus molecules (never the benchmark or evaluation ones)


def train_network(ctx, order, seeds=TRAIN_SEEDS, steps=1500, batch=8192):
    """The learned preconditioner's network, trained before any timing on correction solves of other seeded
    molecules (never the benchmark molecule nor the evaluation molecules) on the mid-size mesh of the same kind (the
    inputs are resolution-free)."""
    import numpy as np
    from paper_2103_02824_gb300 import learned, mk, synth
    from paper_2103_02824_gb300.step import upload_workload
    t0 = time.perf_counter()
    wl = synth.workload("mol4_p2_mid")
    mesh, _ = upload_workload(ctx, wl)
    data = [learned.harvest(learned.Problem(ctx, mesh, *synth.molecule(s, 4)), every=4, cap=5) for s in seeds]
    import torch
    X, U, E = (torch.cat([d[k] for d in data]) for k in range(3))
    mlp = mk.Mlp(ctx, 10 if order == 2 else 4, synth.mlp_init(10 if order == 2 else 4, 0))
    hist = learned.train(ctx, mlp, X, U, E, steps=steps, batch=batch, lr=1e-3, seed=1)
    del X, U, E, data
    mesh.close()
    return mlp, {"molecules": f"synth.molecule(seed, 4), seeds {seeds[0]}-{seeds[-1]} ({len(seeds)} molecules), on "
                              f"mol4_p2_mid (fine 16^3 cubes)",
                 "samples_from": "FP64 PCG iterates 0, 4, ..., 16 of each correction solve",
                 "steps": steps, "batch": batch, "loss_first50": float(np.mean(hist[:50])),
                 "loss_last50": float(np.mean(hist[-50:])), "train_s": time.perf_counter() - t0}


# the serving sweep: 32 molecules (seeds 5000-5031, 1-16 nuclei), each on its own uniform mesh chosen log-uniformly
# between about 50k and 900k free DOF, every orbital's correction problem solved
SERVE_MESHES = ((5, 2), (6, 2), (4, 3), (5, 3), (6, 3))   # (coarse cubes per side, levels): 20^3 .. 48^3 fine cubes


def serve_mode(a):
    """The correction solves (A4) of 32 molecules of uneven size in shared launches (the batched solve, orbitals in
    blocks of at most 32 columns per problem, every block of a molecule on the same mesh and shift) against the same
    solves one molecule after another (mixed precision, and plain FP64 PCG), and the molecules' Hartree Poisson solves
    (A2, multigrid, one after another).  Inputs: each molecule's coarse ground state of the bare Hamiltonian, its
    shift, the Hartree potential of its coarse density and its right-hand sides (setup, untimed)."""
    import numpy as np
    import torch
    from paper_2103_02824_gb300 import build, learned, mk, synth
    from paper_2103_02824_gb300.step import upload_workload
    build.build()
    ctx = mk.Context(0)
    mols, meshes, probs = [], [], []
    t0 = time.perf_counter()
    for k in range(32):
        rng = np.random.default_rng(5000 + k)
        n_nuc = int(rng.integers(1, 17))
        target = float(np.exp(rng.uniform(np.log(5e4), np.log(1.5e6))))
        dofs = [(2 * nc * 2 ** lv - 1) ** 3 for nc, lv in SERVE_MESHES]
        nc, lv = SERVE_MESHES[int(np.argmin([abs(np.log(d / target)) for d in dofs]))]
        Z, R = synth.molecule(5000 + k, n_nuc)
        wl = dict(name=f"serve{k}", Z=Z, R=R, order=2, half=15.0, n_coarse=nc, levels=lv, xc="lda")
        mesh, _ = upload_workload(ctx, wl)
        meshes.append(mesh)
        probs.append(learned.Problem(ctx, mesh, Z, R))
        mols.append(dict(seed=5000 + k, nuclei=n_nuc, N=probs[-1].N, free_dof=mesh.info["n_free"]))
    setup_s = time.perf_counter() - t0
    units = sum(float(p.mesh.info["n_free"]) * p.N for p in probs)
    # orbital blocks of <= 32 columns: one batch problem each
    blocks = []
    for p in probs:
        for c0 in range(0, p.N, 32):
            nb = min(32, p.N - c0)
            ldb = 4 if nb <= 4 else 8 if nb <= 8 else 16 if nb <= 16 else 32
            rb = torch.zeros((p.u.shape[0], ldb), dtype=torch.float64, device="cuda")
            rb[:, :nb] = p.rhs[:, c0:c0 + nb]
            xb = torch.zeros_like(rb)
            xb[:, :nb] = p.u[:, c0:c0 + nb]
            blocks.append((p, rb, xb, nb))
    bopt = mk.opts(precision="mixed", rtol=1e-8, check_every=10)
    fopt = mk.opts(precision="fp64", rtol=1e-8)

    def batched():
        xs = [xb.clone() for (_, _, xb, _) in blocks]
        return mk.mk_batch_correction_solve(ctx, [p.mesh for (p, _, _, _) in blocks], [p.mol for (p, _, _, _) in blocks],
                                            [p.sigma for (p, _, _, _) in blocks], [rb for (_, rb, _, _) in blocks], xs,
                                            [nb for (_, _, _, nb) in blocks], opt=bopt)

    def timed(fn, reps=2):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    ms_b, reps_b = timed(batched)
    ms_m, _ = timed(lambda: [p.solve(bopt) for p in probs])
    ms_f, reps_f = timed(lambda: [p.solve(fopt) for p in probs], reps=1)
    # the Hartree Poisson solves, multigrid, one molecule after another
    occs = [synth.occupations(p.Z) for p in probs]
    ws = [torch.zeros(p.u.shape[0], dtype=torch.float64, device="cuda") for p in probs]
    popt = mk.opts(precision="mixed", rtol=1e-8, check_every=10, coarse="multigrid")
    ms_p, _ = timed(lambda: [mk.mk_hartree_poisson(ctx, p.mesh, p.u, o, p.N, w, opt=popt)
                             for p, o, w in zip(probs, occs, ws)])
    line = {"mode": "serve", "molecules": len(probs), "batch_problems": len(blocks),
            "orbitals": [m["N"] for m in mols], "free_dof": [m["free_dof"] for m in mols],
            "unit": UNIT, "dof_orbitals": units, "setup_s": setup_s,
            "correction_solves_batched_ms": ms_b, "value_batched": units / (ms_b * 1e-3),
            "correction_solves_sequential_mixed_ms": ms_m, "value_sequential_mixed": units / (ms_m * 1e-3),
            "correction_solves_sequential_fp64_ms": ms_f, "value_sequential_fp64": units / (ms_f * 1e-3),
            "max_rel_residual_batched": max(r["max_rel_residual"] for r in reps_b),
            "hartree_solves_sequential_multigrid_ms": ms_p,
            "note": "A4 batched; the A2 Poisson solves run one after another (not batched)"}
    print(json.dumps(line))
    for m in meshes:
        m.close()


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        return reference(a, rank, world)
    if a.mode == "apply":
        return apply_mode(a)
    if a.mode == "learned":
        return learned_mode(a)
    if a.mode == "stiffness":
        return stiffness_mode(a)
    if a.mode == "serve":
        return serve_mode(a)
    if a.mode == "decompose":
        return decompose_mode(a)
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2103_02824_gb300 import build, mk, synth
    from paper_2103_02824_gb300.step import CorrectionStep, coarse_eigenpairs, upload_workload
    build.build()
    wl = synth.workload(a.workload)
    ctx = mk.Context(local)
    precond = "jacobi" if a.precision == "fp64" else a.precond
    mlp, train_info = (None, None)
    if precond == "learned" or not a.no_learned:
        mlp, train_info = train_network(ctx, wl["order"])
    mesh, _ = upload_workload(ctx, wl)
    info = mesh.info
    N, occ = synth.n_orbitals(wl["Z"]), synth.occupations(wl["Z"])
    n_free, NH, E = info["n_free"], info["n_free_coarse"], info["n_elems"]
    mol = mk.Molecule(wl["Z"], wl["R"])
    theta, sigma = mk.mk_correction_shift(ctx, mesh, mol, synth.lanczos_start(n_free), steps=60)
    psiH, lamH, basis = coarse_eigenpairs(ctx, mesh, wl["Z"], wl["R"], N, return_basis=True)
    st = CorrectionStep(ctx, mesh, wl["Z"], wl["R"], N, basis=basis)
    psiH_dev = torch.zeros((NH, st.ld), dtype=torch.float64, device="cuda")
    psiH_dev[:, :N] = torch.from_numpy(psiH).cuda()

    def arm_opts(kind):
        prec = "fp64" if kind == "fp64" else "mixed"
        pc = "learned" if kind == "learned" else "jacobi"
        so = mk.opts(precision=prec, precond=pc, mlp=mlp if pc == "learned" else None, rtol=1e-8, check_every=10)
        # the Hartree Poisson solve of the mixed forms uses the multigrid V-cycle on the mesh hierarchy (the
        # two-level coarse-space preconditioner where the mesh has no hierarchy)
        pc = ("multigrid" if mesh.multigrid else True) if prec == "mixed" else False
        po = mk.opts(precision=prec, rtol=1e-8, check_every=10, coarse=pc)
        return so, po

    def make_step(kind):
        so, po = arm_opts(kind)
        return lambda: st.run(psiH_dev, lamH, occ, sigma, xc=wl["xc"], hartree_bc="multipole", solve_opts=so,
                              poisson_opts=po)

    head_kind = "fp64" if a.precision == "fp64" else precond
    step = make_step(head_kind)
    # the shift rule takes theta from 60 Lanczos steps, an upper bound of the lowest eigenvalue; where it is not
    # low enough the correction operator is indefinite and PCG reports breakdown: sigma is doubled (setup)
    sigma_doublings = 0
    while True:
        try:
            reps = step()
            break
        except mk.MkError as ex:
            if ex.code != mk.MK_ERR_BREAKDOWN or sigma_doublings >= 10:
                raise
            sigma *= 2.0
            sigma_doublings += 1
    for _ in range(a.warmup):
        reps = step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    launches0 = mk.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record()
    for _ in range(a.steps):
        reps = step()
    e1.record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if dist:
        dist.barrier()
    launches = mk.launch_count() - launches0
    ms_total = e0.elapsed_time(e1)
    clk = clocks.stop()
    t_max = whole_job_ms(ms_total, dist, "cuda")
    units = float(n_free) * N * a.steps * world
    value = units / (t_max * 1e-3)
    lam_head = st.lam.cpu().numpy().copy()

    # the dominant kernel's duration, from CUDA events around each application on the launching stream, over a
    # second pass of the same steps (the events are kept out of the timed region above)
    mk.profile_enable(ctx, True)
    for _ in range(a.steps):
        step()
    torch.cuda.synchronize()
    prof = {k: mk.profile_read(ctx, k) for k in (mk.PROF_APPLY64, mk.PROF_APPLY32, mk.PROF_HALO, mk.PROF_LEARNED,
                                                 mk.PROF_STIFF, mk.PROF_PAIRS)}
    # the refinement residuals of the mixed solves on FP32 pairs against the FP64 operator applications of the same
    # steps (the right-hand sides and the projection); both kernels take 4 columns per launch
    pairs_vs_fp64 = None
    if a.precision == "mixed":
        (mp, n_p), (m64, n64) = prof[mk.PROF_PAIRS], prof[mk.PROF_APPLY64]
        pairs_vs_fp64 = {"pairs_us_per_launch": 1e3 * mp / n_p if n_p else None, "pairs_launches_per_step": n_p / a.steps,
                         "fp64_us_per_launch": 1e3 * m64 / n64 if n64 else None, "fp64_launches_per_step": n64 / a.steps,
                         "note": "CUDA events inside the overlapped steps; k_apply_pair (FP32 pairs, about 48 "
                                 "significant bits) for the solves' residuals, k_apply_patch<10,double> for the rest"}
    mk.profile_enable(ctx, False)

    # end to end through the C ABI with host buffers: pinned psi_H in, eigenvalues, coefficients, orbitals out
    h_psiH = torch.zeros((NH, st.ld), dtype=torch.float64).pin_memory()
    h_psiH[:, :N] = torch.from_numpy(psiH)
    h_lam = torch.zeros(N, dtype=torch.float64).pin_memory()
    h_coef = torch.zeros((NH + 1, N), dtype=torch.float64).pin_memory()
    h_psi = torch.zeros(st.psi.shape, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        psiH_dev.copy_(h_psiH, non_blocking=True)
        step()
        h_lam.copy_(st.lam, non_blocking=True)
        h_coef.copy_(st.coef, non_blocking=True)
        h_psi.copy_(st.psi, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    h2d = h_psiH.numel() * 8
    d2h = (h_lam.numel() + h_coef.numel() + h_psi.numel()) * 8

    # the other forms of the same step on the same GPU: mixed precision with Jacobi, and plain FP64 PCG
    compare = {}
    for kind in ("learned", "jacobi", "fp64"):
        if kind == head_kind or (kind == "learned" and mlp is None):
            continue
        stp = make_step(kind)
        try:
            for _ in range(max(1, a.warmup)):
                r = stp()
        except mk.MkError as ex:   # a form that cannot solve this workload is reported, not timed
            compare[kind] = {"error": str(ex)}
            continue
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record()
        for _ in range(a.steps):
            r = stp()
        c1.record()
        torch.cuda.synchronize()
        ms = c0.elapsed_time(c1) / a.steps
        lam_k = st.lam.cpu().numpy()
        compare[kind] = {"value": float(n_free) * N / (ms * 1e-3), "ms_per_step": ms,
                         "solve_iterations": r["solve"]["iterations"],
                         "poisson_iterations": r["poisson"]["iterations"] if r["poisson"] else None,
                         "max_abs_lambda_diff_vs_headline_Ha": float(np.abs(lam_k - lam_head).max())}
        if kind == "learned":
            # the network kernel's duration inside these steps, on a second pass with events on (kept out of the
            # timed pass above)
            mk.profile_enable(ctx, True)
            for _ in range(a.steps):
                stp()
            torch.cuda.synchronize()
            prof[mk.PROF_LEARNED] = mk.profile_read(ctx, mk.PROF_LEARNED)
            mk.profile_enable(ctx, False)

    # the paper's own form of the step (Algorithm 1 steps 5-7 with Algorithm 2's inner SCF and Algorithm 3's
    # precomputations), applied to the headline step's output: its orbitals and eigenvalues, and the Hartree
    # potential of their density (a second correction on the same mesh pair, as Algorithm 1 chains its steps)
    paper = None
    if world == 1 and not a.no_paper:
        from paper_2103_02824_gb300.step import PaperStep
        pst = PaperStep(ctx, mesh, wl["Z"], wl["R"], N, ld=st.ld)
        so, po = arm_opts(head_kind)
        u_in, lam_in = st.psi.clone(), st.lam.cpu().numpy().copy()
        w_in = torch.zeros_like(st.w)
        mk.mk_hartree_poisson(ctx, mesh, u_in, occ, N, w_in, bc="multipole", opt=po)

        def paper_run():
            return pst.run(u_in, lam_in, occ, sigma, w_in, xc=wl["xc"], solve_opts=so, poisson_opts=po,
                           inner_tol=1e-10, max_inner=200)
        for _ in range(max(1, a.warmup)):
            pr = paper_run()
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record()
        for _ in range(a.steps):
            pr = paper_run()
        c1.record()
        torch.cuda.synchronize()
        p_ms = c0.elapsed_time(c1) / a.steps
        # the inner part alone: Algorithm 3's precomputations, then the inner iterations
        i0, i1, i2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        lam_p, coef_p = torch.zeros_like(pst.lam), torch.zeros_like(pst.coef)
        i0.record()
        inner = mk.Inner(ctx, mesh, pst.mol, pst.phit, N, pst.wt, pst.vxc)
        i1.record()
        ir = inner.run(occ, lam_p, coef_p, tol=1e-10, max_inner=200)
        i2.record()
        torch.cuda.synchronize()
        inner.close()
        lam_paper = pst.lam.cpu().numpy()
        pst.run(u_in, lam_in, occ, sigma, w_in, xc=wl["xc"], solve_opts=so, poisson_opts=po, inner_tol=0.0,
                max_inner=1)
        lam_first = pst.lam.cpu().numpy()
        paper = {"ms_per_step": p_ms, "value": float(n_free) * N / (p_ms * 1e-3), "unit": UNIT,
                 "inner_iterations": pr["inner"]["iters"], "inner_last_change": pr["inner"]["delta"],
                 "precompute_ms": i0.elapsed_time(i1), "inner_ms": i1.elapsed_time(i2),
                 "inner_ms_per_iteration": i1.elapsed_time(i2) / max(1, ir["iters"]),
                 "solve_iterations": pr["solve"]["iterations"], "poisson_iterations": pr["poisson"]["iterations"],
                 "lambda": [float(x) for x in lam_paper],
                 "lambda_after_one_inner_iteration": [float(x) for x in lam_first],
                 "input": "the headline step's output orbitals and eigenvalues, w = their Hartree potential",
                 "max_abs_lambda_diff_vs_headline_Ha": float(np.abs(lam_paper - lam_head).max())}
        pst.close()

    # the joint augmented space V_H + span{psi^_1..psi^_N} (the original multilevel-correction form) from the
    # headline step's blocks: Rayleigh-Ritz for the lowest N pairs, then the joint orbitals on the fine mesh
    joint = None
    if world == 1 and not a.no_paper:
        lam_j = torch.zeros(N, dtype=torch.float64, device="cuda")
        X_j = torch.zeros((NH + N, N), dtype=torch.float64, device="cuda")
        psi_j = torch.zeros_like(st.psi)
        step()
        torch.cuda.synchronize()
        j0, j1, j2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        j0.record()
        kept = mk.mk_joint_ritz(ctx, NH, N, N, st.d, st.V, st.b, st.c, st.gramA, st.gramM, lam_j, X_j)
        j1.record()
        mk.mk_joint_assemble(ctx, mesh, N, N, X_j, st.psihat, st.u, psi_j)
        j2.record()
        torch.cuda.synchronize()
        lj = lam_j.cpu().numpy()
        joint = {"ritz_ms": j0.elapsed_time(j1), "assemble_ms": j1.elapsed_time(j2), "corrections_kept": kept,
                 "lambda": [float(x) for x in lj],
                 "sum_lambda_joint_minus_per_orbital_Ha": float(lj.sum() - np.sort(lam_head).sum())}

    # the outer AFEM loop's Estimate and Mark steps on the headline step's output: the residual indicator of
    # (lambda, psi) at the potential of psi's own density, then Dorfler's marking (theta = 0.4)
    afem = None
    if world == 1 and not a.no_paper:
        w_psi = torch.zeros_like(st.w)
        vq_psi = torch.zeros_like(st.vq)
        eta2 = torch.zeros(E, dtype=torch.float64, device="cuda")
        marked = torch.zeros(E, dtype=torch.uint8, device="cuda")
        lam_np = st.lam.cpu().numpy().copy()
        _, po_a = arm_opts(head_kind)
        a0, a1, a2, a3 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
        for rep_k in range(2):          # the first pass builds the mesh's face table
            a0.record()
            mk.mk_hartree_poisson(ctx, mesh, st.psi, occ, N, w_psi, bc="multipole", opt=po_a)
            mk.mk_frozen_potential(ctx, mesh, st.psi, occ, N, w_psi, wl["xc"], vq_psi)
            a1.record()
            mk.mk_error_indicators(ctx, mesh, mol, st.psi, N, lam_np, vq_psi, eta2)
            a2.record()
            n_marked, t_cut = mk.mk_dorfler_mark(ctx, eta2, 0.4, marked)
            a3.record()
            torch.cuda.synchronize()
        afem = {"potential_ms": a0.elapsed_time(a1), "indicator_ms": a1.elapsed_time(a2),
                "dorfler_ms": a2.elapsed_time(a3), "theta": 0.4, "marked": n_marked, "elements": E,
                "eta_total": float(eta2.sum().sqrt()), "threshold": t_cut}
        # Refine: newest-vertex bisection of the marked elements with closure, on the fine mesh in Maubach's form
        # (the uniform workloads' fine mesh is the Kuhn mesh of its cubes, element for element)
        if wl.get("mesh") != "graded":
            nvb = synth.NVBMesh.kuhn(wl["n_coarse"] * 2 ** wl["levels"], wl["half"])
            nv0 = nvb.coords().shape[0]
            cap_v, cap_e = nv0 + 4 * E, 3 * E
            Xd = torch.zeros((cap_v, 3), dtype=torch.float64, device="cuda")
            Td = torch.zeros((cap_e, 4), dtype=torch.int32, device="cuda")
            Kd = torch.zeros(cap_e, dtype=torch.int8, device="cuda")
            Pd = torch.zeros(cap_e, dtype=torch.int32, device="cuda")
            times = []
            for rep_k in range(3):
                Xd[:nv0] = torch.from_numpy(nvb.coords()).cuda()
                Td[:E] = torch.from_numpy(nvb.T.astype(np.int32)).cuda()
                Kd[:E] = torch.from_numpy(nvb.K.astype(np.int8)).cuda()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                nv1, E1, rnd = mk.mk_refine(ctx, Xd, Td, Kd, Pd, marked, nv0, E)
                times.append(time.perf_counter() - t0)
            afem.update({"refine_ms": 1e3 * min(times), "refined_elements": E1, "refined_vertices": nv1,
                         "refine_rounds": rnd})

    # the same operator kernel timed alone (no concurrent stream), for comparison with its in-step duration
    iso_ms = None
    if a.precision == "mixed":
        g = torch.Generator(device="cuda").manual_seed(5)
        xa = torch.randn((info["n_nodes"], st.ld), generator=g, device="cuda", dtype=torch.float32)
        ya = torch.empty_like(xa)
        for _ in range(3):
            mk.mk_operator_apply(ctx, mesh, mol, sigma, xa, ya)
        torch.cuda.synchronize()
        mk.profile_enable(ctx, True)
        for _ in range(20):
            mk.mk_operator_apply(ctx, mesh, mol, sigma, xa, ya)
        torch.cuda.synchronize()
        ims, inn = mk.profile_read(ctx, mk.PROF_APPLY32)
        mk.profile_enable(ctx, False)
        iso_ms = ims / inn if inn else None

    # batching: the correction solves of 8 other seeded molecules on mid-size meshes, batched (shared launches)
    # against one after the other, same options
    batch = None
    if a.precision == "mixed" and world == 1 and not a.no_batch:
        from paper_2103_02824_gb300 import learned
        bw = synth.workload("mol4_p2_mid")
        bmeshes = [upload_workload(ctx, bw)[0] for _ in range(8)]
        bprobs = [learned.Problem(ctx, bm, *synth.molecule(sd, 4)) for bm, sd in zip(bmeshes, range(20, 28))]
        bopt = mk.opts(precision="mixed", rtol=1e-8, check_every=10)
        units_b = sum(float(bm.info["n_free"]) * bp.N for bm, bp in zip(bmeshes, bprobs))
        for _ in range(2):  # warm-up of both forms
            for bp in bprobs:
                bp.solve(bopt)
            mk.mk_batch_correction_solve(ctx, bmeshes, [bp.mol for bp in bprobs], [bp.sigma for bp in bprobs],
                                         [bp.rhs for bp in bprobs], [bp.u.clone() for bp in bprobs],
                                         [bp.N for bp in bprobs], opt=bopt)
        torch.cuda.synchronize()
        xs = [bp.u.clone() for bp in bprobs]
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record()
        for bp in bprobs:
            bp.solve(bopt)
        c1.record()
        torch.cuda.synchronize()
        seq_ms = c0.elapsed_time(c1)
        c0.record()
        breps = mk.mk_batch_correction_solve(ctx, bmeshes, [bp.mol for bp in bprobs], [bp.sigma for bp in bprobs],
                                             [bp.rhs for bp in bprobs], xs, [bp.N for bp in bprobs], opt=bopt)
        c1.record()
        torch.cuda.synchronize()
        bat_ms = c0.elapsed_time(c1)
        batch = {"molecules": "synth.molecule(seed, 4), seeds 20-27, each on its own mol4_p2_mid mesh (24,576 P2 tets)",
                 "orbitals": [bp.N for bp in bprobs], "correction_solves_ms_batched": bat_ms,
                 "correction_solves_ms_sequential": seq_ms,
                 "value_batched": units_b / (bat_ms * 1e-3), "value_sequential": units_b / (seq_ms * 1e-3),
                 "unit": UNIT, "max_rel_residual": max(r["max_rel_residual"] for r in breps)}
        for bm in bmeshes:
            bm.close()

    # the metric's own comparison, learned vs plain PCG, on the molecules the network is evaluated on
    evaluation = None
    if mlp is not None and world == 1 and not a.no_eval:
        evaluation = eval_learned(ctx, mlp)

    # roofline of the dominant kernel (the element-by-element operator application of the correction problems):
    # its algorithmic bytes over the average CUDA-event duration of its launches on the launching stream, every
    # application of the profiled pass (inside the graphs too), the Poisson solve's stiffness kernel excluded
    kind = mk.PROF_APPLY32 if prof[mk.PROF_APPLY32][1] > 0 else mk.PROF_APPLY64
    ms_k, n_k = prof[kind]
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    nloc = info["nloc"]
    npack = nloc * (nloc + 1) // 2
    ld = st.ld
    # the library records one event pair per launch, and a launch covers a block of columns: up to 32 (the FP32
    # register-staged operator), 8 (the learned network) or 4 (the FP64 operator); an application to all columns is
    # `passes` launches
    passes = -(-ld // (4 if kind == mk.PROF_APPLY64 else 32))
    n_k, ms_pass = n_k // passes, ms_k / n_k if n_k else None
    ms_k = ms_pass * passes * n_k if n_k else 0.0
    if iso_ms is not None:
        iso_ms *= passes
    if kind == mk.PROF_APPLY64:
        flops = 2.0 * nloc * nloc * E * N
        achieved = flops / (ms_k / n_k * 1e-3) / 1e12 if n_k else None
        peak = FP64_TFLOPS
        roof = {"kernel": "k_apply_patch<10,double> (FP64 element-by-element operator)", "bound": "alu",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak if achieved else None,
                "traffic": None, "applications": n_k, "ms_per_application": ms_k / n_k if n_k else None,
                "peak_source": f"FP64 FMA rate derived from the SM count and clock ({FP64_NOTE})"}
    else:
        nbytes = 2.0 * info["n_nodes"] * ld * 4 + E * (npack * 4 + nloc * 4 + 2 * nloc)
        achieved = nbytes / (ms_k / n_k * 1e-3) / 1e9 if n_k else None
        peak = peaks.get("hbm_gbs", 6780.7)
        roof = {"kernel": OPERATOR_KERNEL, "bound": "hbm",
                "achieved": achieved,
                "peak": peak, "unit": "GB/s", "frac": achieved / peak if achieved else None,
                "traffic": TRAFFIC.get((a.workload, ld)),
                "applications": n_k, "applications_per_step": n_k / a.steps,
                "ms_per_application": ms_k / n_k if n_k else None,
                "bytes_per_application": nbytes, "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst), of measured",
                "frac_of_nominal_8tbs": achieved / 8000.0 if achieved else None,
                "target": "0.60 of HBM (north star)", "target_met": bool(achieved and achieved / peak >= 0.60),
                "measured": "CUDA events around every application of the correction operator inside the steps",
                "isolated": None if iso_ms is None else {
                    "ms_per_application": iso_ms, "achieved": nbytes / (iso_ms * 1e-3) / 1e9,
                    "frac": nbytes / (iso_ms * 1e-3) / 1e9 / peak, "applications": 20}}
    # the Poisson solve's matrix-free stiffness operator (one column): 8 FP32 factors, 10 int32 node indices and
    # 10 uint16 incidences per element, x read and y written once
    roof_k = None
    ms_s, n_s = prof[mk.PROF_STIFF]
    if n_s:
        sbytes = 2.0 * info["n_nodes"] * 4 + E * (8 * 4 + nloc * 4 + 2 * nloc)
        sach = sbytes / (ms_s / n_s * 1e-3) / 1e9
        speak = peaks.get("hbm_gbs", 6780.7)
        roof_k = {"kernel": "k_stiff_patch<10> (matrix-free FP32 stiffness operator of the Hartree Poisson solve)",
                  "bound": "hbm", "achieved": sach, "peak": speak, "unit": "GB/s", "frac": sach / speak,
                  "applications": n_s, "applications_per_step": n_s / a.steps, "ms_per_application": ms_s / n_s,
                  "bytes_per_application": sbytes, "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst), of measured"}

    # the learned preconditioner's patch kernel (tcgen05 network + node sums): algorithmic network FLOPs of one
    # application (2 (n_in 64 + 64 64 + 64 n_out) per (element, orbital) row) over its CUDA-event duration inside
    # the steps, against the sustained BF16 tensor peak (the kernel runs inside a long step)
    roof_tc = None
    ms_l, n_l = prof[mk.PROF_LEARNED]
    lpasses = -(-N // 8)
    n_l //= lpasses                                # applications (a launch covers 8 orbital columns)
    if n_l:
        nin, nout = nloc + 12, nloc
        lflops = 2.0 * (nin * 64 + 64 * 64 + 64 * nout) * E * N
        lpeak = peaks.get("bf16_tflops_sustained", 1712.6)
        lach = lflops / (ms_l / n_l * 1e-3) / 1e12
        roof_tc = {"kernel": "k_learned_patch_tc (learned preconditioner: BF16 network on tcgen05 + node sums)",
                   "bound": "tensor", "achieved": lach, "peak": lpeak, "unit": "TFLOP/s", "frac": lach / lpeak,
                   "applications": n_l, "ms_per_application": ms_l / n_l, "flops_per_application": lflops,
                   "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained, of measured",
                   "note": "issue- and latency-bound on the per-tile layer chain, not on the tensor pipe"}

    cpu = None
    parity = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        try:
            o = run_oracle(a.workload, 1, 0)
            tstep = o["step_s"][0]
            # the same step by the oracle, from its own inputs (coarse eigenpairs, Lanczos shift), at the same 1e-8
            lam_o = np.asarray(o["lam"])
            parity = {"max_abs_lambda_err_Ha": float(np.abs(lam_head - lam_o).max()),
                      "sigma_gpu": sigma, "sigma_oracle": o["sigma"], "tolerance_Ha": 1e-6,
                      "compared": f"all {N} eigenvalues of the headline step against the oracle's step on the same "
                                  f"workload, both solved to 1e-8 FP64 relative residual"}
            parity["ok"] = parity["max_abs_lambda_err_Ha"] <= 1e-6
            cpu = {"value": o["n_free"] * o["N"] / tstep, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
                   "sample": f"one full oracle correction step (A1-A8, scipy.sparse CSR + Jacobi-PCG to 1e-8, dense "
                             f"LAPACK eigensolves) on the same workload, {tstep:.1f} s; static assembly excluded "
                             f"({o['setup_s']:.1f} s)"}
        except Exception as ex:  # report, never fake
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"}

    if rank == 0:
        solve = reps["solve"]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": t_max / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+bf16+f64" if head_kind == "learned" else ("f32+f64" if head_kind == "jacobi" else "f64"),
            "data": "synthetic",
            "config": dict(workload_config(wl, N, n_free, NH, E), precision=a.precision,
                           precond="learned (FCG(1))" if head_kind == "learned" else "jacobi",
                           rtol=1e-8, sigma=sigma, sigma_doublings=sigma_doublings,
                           l2="working set > L2 (no flush needed)",
                           parallelism="replicas" if world > 1 else "single GPU"),
            "e2e": {"value": float(n_free) * N * a.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "gpu_launches_per_step": launches / a.steps,
            "clocks": clk, "roofline": roof, "roofline_learned": roof_tc, "roofline_stiffness": roof_k,
            "residual_pairs_vs_fp64": pairs_vs_fp64,
            "cpu_baseline": cpu, "parity": parity,
            "compare": compare, "paper_form": paper, "joint_space": joint, "afem_estimate_mark": afem,
            "training": train_info, "batch": batch,
            "learned_vs_plain": evaluation,
            "solve_iterations": solve["iterations"], "solve_max_rel_residual": solve["max_rel_residual"],
            "poisson_iterations": reps["poisson"]["iterations"] if reps["poisson"] else None,
            "lambda": [float(x) for x in lam_head],
        }
        print(json.dumps(line))
        if parity is not None and not parity["ok"]:
            raise SystemExit(f"parity failed: |lambda - oracle| = {parity['max_abs_lambda_err_Ha']:.3e} Ha > 1e-6")
    if dist:
        dist.destroy_process_group()


def reference(a, rank, world):
    if rank != 0:
        return
    from paper_2103_02824_gb300 import synth
    wl = synth.workload(a.workload)
    o = run_oracle(a.workload, a.steps, a.warmup, timeout=3600)
    t = sum(o["step_s"])
    value = o["n_free"] * o["N"] * len(o["step_s"]) / t
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * t / len(o["step_s"]), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": dict(workload_config(wl, o["N"], o["n_free"], o["n_free_coarse"], o["n_elems"]), precision="fp64", precond="jacobi",
                       rtol=1e-8),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
                         "sample": f"{len(o['step_s'])} full oracle correction steps of the workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
