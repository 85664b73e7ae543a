"""CPU FP64 oracle for the fine-mesh correction step of the multilevel-correction AFEM for Kohn-Sham.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` / `--impl reference`
legs of `bench.py` may import or run anything in this package.  The CUDA product path never calls it and shares
no code with it: the two meet only in `paper_2103_02824_gb300.synth`, the seeded input generator.

Everything here is plain, slow and written to be checked against the paper by eye: assembled sparse matrices
(scipy.sparse), a plain Jacobi-preconditioned CG, and a dense generalised symmetric eigensolver (LAPACK via
scipy.linalg.eigh) for the augmented problem of Eq. (Eigenvalue_H_h).  Functions cite the passage they follow.

Pins (tests/test_oracle_*.py) tie it to what the paper and mathematics fix: quadrature exactness on monomials,
closed-form mesh counts, patch tests of the stiffness and mass matrices, the Galerkin identity P^T A_h P = A_H on
nested meshes, the hydrogen ground state (-0.5 Ha), the harmonic-oscillator spectrum (1.5, 2.5 Ha), closed forms
and finite-difference derivatives of the paper's LDA, the Gaussian-charge Poisson solution, Rayleigh-Ritz bounds
and the exact-eigenpair fixed point of the correction step.  Parity of the multi-molecule physics (eigenvalues
of synthetic molecules) is unpinned beyond these: the paper prints no eigenvalues.
"""
