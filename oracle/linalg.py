"""Plain linear algebra for the oracle: Jacobi-preconditioned CG, Lanczos on a pencil, and the augmented
eigenproblem of Eq. (Eigenvalue_H_h) solved densely, with the paper's selection rule (Algorithm 2, step (a))."""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

STATUS_OK = 0
STATUS_SINGULAR_AUG = 1
SINGULAR_RTOL = 1e-7   # ||u||_M / ||phi~||_M; gamma - c^T M_H^-1 c carries ~1e-16 gamma of rounding
TIE_RTOL = 1e-12


class Breakdown(RuntimeError):
    pass


def pcg(A, B, X0=None, tol=1e-13, maxit=50000):
    """Jacobi-preconditioned CG on each column of B (the boundary-value problems of Algorithm 1, step 5, are
    independent per orbital).  Stops a column when ||b - A x|| / ||b|| <= tol (recursive residual), then reports
    the true residual.  Raises Breakdown when p^T A p <= 0 (operator not positive definite)."""
    B = np.asarray(B, dtype=np.float64)
    one = B.ndim == 1
    if one:
        B = B[:, None]
    d = A.diagonal()
    X = np.zeros_like(B) if X0 is None else np.array(X0, dtype=np.float64).reshape(B.shape)
    R = B - A @ X
    Zr = R / d[:, None]
    P = Zr.copy()
    rz = np.sum(R * Zr, axis=0)
    bn = np.linalg.norm(B, axis=0)
    bn = np.where(bn > 0, bn, 1.0)
    iters = np.zeros(B.shape[1], dtype=np.int64)
    for it in range(maxit):
        active = np.linalg.norm(R, axis=0) / bn > tol
        if not active.any():
            break
        Q = A @ P
        pq = np.sum(P * Q, axis=0)
        if np.any(pq[active] <= 0):
            raise Breakdown("p^T A p <= 0")
        alpha = np.where(active, rz / np.where(active, pq, 1.0), 0.0)
        X += alpha * P
        R -= alpha * Q
        Zr = R / d[:, None]
        rz_new = np.sum(R * Zr, axis=0)
        beta = np.where(active, rz_new / np.where(active, rz, 1.0), 0.0)
        P = np.where(active, Zr + beta * P, P)
        rz = np.where(active, rz_new, rz)
        iters += active
    true_res = np.linalg.norm(B - A @ X, axis=0) / bn
    if one:
        return X[:, 0], iters, true_res
    return X, iters, true_res


def lanczos_lowest(H, M, v0, steps=60):
    """Lowest Ritz value of `steps` Lanczos steps on the pencil (H, M) in the M inner product (operator M^-1 H),
    no reorthogonalisation, start vector v0.  Used for the shift rule sigma = 1.05 max(0, -theta) + 0.5.
    M^-1 is applied by Jacobi-PCG to 1e-13 (a direct factorisation of a 3-D mass matrix fills in badly)."""
    def Msolve(r):
        return pcg(M, r, tol=1e-13)[0]
    v = v0 / np.sqrt(v0 @ (M @ v0))
    v_prev = np.zeros_like(v)
    a, b = [], []
    beta = 0.0
    for j in range(steps):
        w = Msolve(H @ v)
        alpha = v @ (H @ v)
        w = w - alpha * v - beta * v_prev
        beta = np.sqrt(w @ (M @ w))
        a.append(alpha)
        b.append(beta)
        if beta == 0.0:
            break
        v_prev, v = v, w / beta
    T = np.diag(a) + np.diag(b[:-1], 1) + np.diag(b[:-1], -1)
    return float(np.linalg.eigvalsh(T)[0])


def shift_rule(theta_min: float) -> float:
    """sigma = 1.05 max(0, -theta_min) + 0.5 Ha: makes K/2 + M_Vext + sigma M positive definite with margin."""
    return 1.05 * max(0.0, -theta_min) + 0.5


def augmented_select(AH, MH, b, c, beta, gamma):
    """Eq. (Eigenvalue_H_h) for one orbital, solved densely: all eigenpairs of
        [[A_H, b], [b^T, beta]] x = lambda [[M_H, c], [c^T, gamma]] x,
    M-normalised.  Algorithm 2 (a) keeps "the eigenfunction that has the largest component in span{phi~}".
    Reading: the component is the M-orthogonal projection on phi~, |(x, phi~)_M| = |(M_aug x)_last| for an
    M_aug-normalised x; ties within 1e-12 (relative) go to the lower eigenvalue.  If ||u||_M / ||phi~||_M < 1e-7
    with u = phi~ - Pi_H phi~ (phi~ already in V_H), the extra column is dropped and the coarse Ritz pair with the
    largest |(x, Pi_H phi~)_M| is returned with theta_2 = 0 and status STATUS_SINGULAR_AUG.
    The sign is fixed so that (x, phi~)_M >= 0.  Returns (lambda, coef [N_H+1], status, scores)."""
    n = AH.shape[0]
    t = sla.solve(MH, c, assume_a="pos")
    u2 = gamma - c @ t
    if not (u2 > (SINGULAR_RTOL ** 2) * gamma):
        lam, V = sla.eigh(AH, MH)
        proj = V.T @ c
        s = np.abs(proj)
        k = _pick(s)
        sgn = -1.0 if proj[k] < 0 else 1.0
        return lam[k], sgn * np.concatenate([V[:, k], [0.0]]), STATUS_SINGULAR_AUG, s
    A = np.zeros((n + 1, n + 1))
    M = np.zeros((n + 1, n + 1))
    A[:n, :n], A[:n, n], A[n, :n], A[n, n] = AH, b, b, beta
    M[:n, :n], M[:n, n], M[n, :n], M[n, n] = MH, c, c, gamma
    lam, X = sla.eigh(A, M)
    proj = (M @ X)[n, :]
    s = np.abs(proj)
    k = _pick(s)
    sgn = -1.0 if proj[k] < 0 else 1.0
    return lam[k], sgn * X[:, k], STATUS_OK, s


def _pick(s):
    smax = s.max()
    return int(np.nonzero(s >= smax * (1.0 - TIE_RTOL))[0][0])


def arrowhead_select(AH, MH, b, c, beta, gamma):
    """Second route to the same eigenpairs: shared M_H-orthonormal eigen-decomposition of (A_H, M_H), the extra
    direction M-orthogonalised against V_H, and the resulting arrowhead matrix solved as a standard symmetric
    problem.  Must agree with augmented_select (checked in the tests)."""
    Lam, V = sla.eigh(AH, MH)
    t = sla.solve(MH, c, assume_a="pos")
    un = np.sqrt(gamma - c @ t)
    z = V.T @ (b - AH @ t) / un
    alpha = (beta - 2.0 * t @ b + t @ (AH @ t)) / (un * un)
    n = len(Lam)
    H = np.zeros((n + 1, n + 1))
    H[:n, :n] = np.diag(Lam)
    H[:n, n] = z
    H[n, :n] = z
    H[n, n] = alpha
    mu, Y = np.linalg.eigh(H)
    p = np.concatenate([V.T @ c, [un]])   # coordinates of phi~ in the basis [V, u/|u|]
    s = np.abs(Y.T @ p)
    k = _pick(s)
    y = Y[:, k] * (-1.0 if Y[:, k] @ p < 0 else 1.0)
    coarse = V @ y[:n] - (y[n] / un) * t
    theta = y[n] / un
    return mu[k], np.concatenate([coarse, [theta]]), s


def joint_ritz(AH, MH, B, C, GA, GM, k, drop_rtol=1e-12):
    """Rayleigh-Ritz in the joint augmented space V_H + span{psi^_1, .., psi^_N} (the multilevel-correction form that
    augments the coarse space with all corrections at once, instead of one at a time): the lowest k eigenpairs of
        [[A_H, B], [B^T, G_A]] x = lambda [[M_H, C], [C^T, G_M]] x,
    B = P^T H Psi^, C = P^T M Psi^, G_A = Psi^T H Psi^, G_M = Psi^T M Psi^.  Directions of the joint basis that are
    linearly dependent (mass eigenvalues below drop_rtol times the largest; a psi^ already in V_H, or two equal
    corrections) are removed before the dense solve.  Returns (lambda [k], X [N_H + N, k]) with X M-orthonormal,
    coefficients of the coarse basis followed by those of the psi^_i."""
    A = np.block([[AH, B], [B.T, GA]])
    M = np.block([[MH, C], [C.T, GM]])
    A, M = 0.5 * (A + A.T), 0.5 * (M + M.T)
    s, U = sla.eigh(M)
    keep = s > drop_rtol * s.max()
    W = U[:, keep] / np.sqrt(s[keep])
    T = W.T @ A @ W
    lam, Y = sla.eigh(0.5 * (T + T.T))
    return lam[:k], W @ Y[:, :k]
