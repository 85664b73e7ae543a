"""Learned element-patch preconditioner inside flexible CG, plain FP64 numpy (oracle side).

TEST INFRASTRUCTURE ONLY: only `tests/`, `__graft_entry__.smoke()` and the baseline legs of `bench.py` may use
this module (see the package header).

The paper solves its boundary-value problems (Algorithm 1, step 5; Sec. 4) with standard solvers and says nothing
about learned preconditioners; the definitions below are this project's reading of the learned-preconditioner
rows of the hot path, written out plainly so that the CUDA path can be checked against them.

features   for element e and orbital column j: r_e = the residual at the element's n_loc nodes, s = ||r_e||_2,
           h_e = |det J_e|^(1/3) (the edge of a cube of the element's volume, up to a constant);
           x = [r_e / s  (zero when s = 0),  (v_k - centroid_e) / h_e for the 4 vertices]      (n_loc + 12 inputs)
network    y = W3 relu(W2 relu(W1 x + b1) + b2) + b3                                          (n_loc outputs)
assembly   c_e = y s / h_e;  z_nn(node) = (sum of c_e[slot] over the node's (element, slot) incidences)
           divided by the node's multiplicity (its number of incidences); boundary rows are zero
precond    z = r / diag(A) + z_nn
solver     flexible CG, FCG(1) (Y. Notay, SIAM J. Sci. Comput. 22 (2000)): the new direction is made
           A-orthogonal to the previous one explicitly, so a nonlinear or changing preconditioner is allowed
training   a sample is (x, u, e) with u = s / h_e and e = (x* - x_k) at the element's nodes, x* the converged
           solution and x_k an iterate of the same solve with residual r_k; the network predicts the error
           normalised the same way as its input, t = e / u, and the loss compares u y with e:
               L = sum_s ||u_s y_s - e_s||^2 / sum_s u_s^2
           (the mean squared error of the normalised prediction weighted by u^2; elements whose residual
           vanishes carry no weight, which keeps the loss finite).  Adam (Kingma & Ba 2015) updates the weights.
"""
from __future__ import annotations

import numpy as np

PARAM_ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def sizes(nloc: int, nh: int = 64):
    """Layer widths (inputs, hidden, hidden, outputs) for an element with nloc nodes."""
    return nloc + 12, nh, nh, nloc


def flatten(params) -> np.ndarray:
    return np.concatenate([np.asarray(params[k], dtype=np.float64).ravel() for k in PARAM_ORDER])


def unflatten(vec, nin: int, nh: int, nout: int):
    shapes = {"W1": (nh, nin), "b1": (nh,), "W2": (nh, nh), "b2": (nh,), "W3": (nout, nh), "b3": (nout,)}
    out, o = {}, 0
    for k in PARAM_ORDER:
        n = int(np.prod(shapes[k]))
        out[k] = np.asarray(vec[o:o + n], dtype=np.float64).reshape(shapes[k])
        o += n
    return out


# ------------------------------------------------------------------------------------------------ geometry
def geometry(mesh):
    """h_e = |det J_e|^(1/3) [E] and the vertex offsets from the centroid divided by h_e [E, 12]."""
    v = mesh.coords[mesh.tets]                         # [E, 4, 3]
    h = np.abs(mesh.det) ** (1.0 / 3.0)
    g = (v - v.mean(axis=1, keepdims=True)) / h[:, None, None]
    return h, g.reshape(len(h), 12)


def multiplicity(mesh) -> np.ndarray:
    """Number of (element, slot) incidences of every node."""
    return np.bincount(mesh.elem.ravel(), minlength=mesh.n_nodes).astype(np.float64)


def features(mesh, R):
    """Network inputs for every (element, column): X [E, N, n_loc + 12], s [E, N], h [E].  R: [n_nodes, N]."""
    h, g = geometry(mesh)
    re = np.asarray(R, dtype=np.float64)[mesh.elem]    # [E, n_loc, N]
    s = np.sqrt(np.sum(re * re, axis=1))               # [E, N]
    xin = np.where(s[:, None, :] > 0, re / np.where(s > 0, s, 1.0)[:, None, :], 0.0)
    E, _, N = re.shape
    X = np.concatenate([np.transpose(xin, (0, 2, 1)), np.broadcast_to(g[:, None, :], (E, N, 12))], axis=2)
    return X, s, h


# ------------------------------------------------------------------------------------------------ network
def relu(z):
    return np.maximum(z, 0.0)


def forward(params, X):
    """y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for the rows of X [S, nin]; returns y and the cache."""
    z1 = X @ params["W1"].T + params["b1"]
    h1 = relu(z1)
    z2 = h1 @ params["W2"].T + params["b2"]
    h2 = relu(z2)
    y = h2 @ params["W3"].T + params["b3"]
    return y, (X, z1, h1, z2, h2)


def backward(params, cache, dy):
    """Gradients of sum(dy * y) with respect to the parameters (chain rule through the three layers)."""
    X, z1, h1, z2, h2 = cache
    g = {"W3": dy.T @ h2, "b3": dy.sum(axis=0)}
    d2 = (dy @ params["W3"]) * (z2 > 0)
    g["W2"], g["b2"] = d2.T @ h1, d2.sum(axis=0)
    d1 = (d2 @ params["W2"]) * (z1 > 0)
    g["W1"], g["b1"] = d1.T @ X, d1.sum(axis=0)
    return g


def loss_and_grad(params, X, U, Eerr):
    """L = sum_s ||u_s y_s - e_s||^2 / sum_s u_s^2 and its gradient.  X [S, nin], U [S], Eerr [S, nout]."""
    y, cache = forward(params, X)
    den = float(np.sum(U * U))
    res = U[:, None] * y - Eerr
    loss = float(np.sum(res * res)) / den
    dy = 2.0 * U[:, None] * res / den
    return loss, backward(params, cache, dy)


def adam_step(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected moments); `state` holds m, v and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    out = {}
    for k in PARAM_ORDER:
        m = beta1 * state.get("m_" + k, 0.0) + (1.0 - beta1) * grads[k]
        v = beta2 * state.get("v_" + k, 0.0) + (1.0 - beta2) * grads[k] * grads[k]
        state["m_" + k], state["v_" + k] = m, v
        mhat = m / (1.0 - beta1 ** t)
        vhat = v / (1.0 - beta2 ** t)
        out[k] = params[k] - lr * mhat / (np.sqrt(vhat) + eps)
    return out


# ------------------------------------------------------------------------------------------------ preconditioner
def correction(mesh, params, R):
    """z_nn for all columns of R [n_nodes, N] (boundary rows of the result zero)."""
    X, s, h = features(mesh, R)
    E, N, nin = X.shape
    y, _ = forward(params, X.reshape(E * N, nin))
    c = y.reshape(E, N, -1) * (s / h[:, None])[:, :, None]        # [E, N, n_loc]
    Z = np.zeros((mesh.n_nodes, N))
    np.add.at(Z, mesh.elem.ravel(), np.transpose(c, (0, 2, 1)).reshape(-1, N))
    Z /= multiplicity(mesh)[:, None]
    Z[mesh.boundary] = 0.0
    return Z


def precond(mesh, params, diag, R):
    """z = r / diag(A) + z_nn on all nodes (R and the result [n_nodes, N], boundary rows zero)."""
    Z = np.where(mesh.boundary[:, None], 0.0, R / np.where(mesh.boundary, 1.0, diag)[:, None])
    if params is not None:
        Z = Z + correction(mesh, params, R)
    return Z


def fcg(A, B, M, tol=1e-8, maxit=10000):
    """FCG(1) on each column: p_0 = M(r_0); alpha = (p, r)/(p, Ap); x += alpha p; r -= alpha Ap;
    z = M(r); p = z - ((z, Ap)/(p, Ap)) p.  A [n, n] sparse on the free DOF, B [n, N], M: [n, N] -> [n, N].
    Returns X, iterations per column, true relative residuals."""
    B = np.asarray(B, dtype=np.float64)
    X = np.zeros_like(B)
    R = B.copy()
    bn = np.linalg.norm(B, axis=0)
    bn = np.where(bn > 0, bn, 1.0)
    P = M(R)
    iters = np.zeros(B.shape[1], dtype=np.int64)
    for _ in range(maxit):
        active = np.linalg.norm(R, axis=0) / bn > tol
        if not active.any():
            break
        Q = A @ P
        pq = np.sum(P * Q, axis=0)
        alpha = np.where(active, np.sum(P * R, axis=0) / np.where(active, pq, 1.0), 0.0)
        X += alpha * P
        R -= alpha * Q
        Zr = M(R)
        beta = np.where(active, -np.sum(Zr * Q, axis=0) / np.where(active, pq, 1.0), 0.0)
        P = np.where(active, Zr + beta * P, P)
        iters += active
    return X, iters, np.linalg.norm(B - A @ X, axis=0) / bn


def harvest(mesh, Rk, Xk, Xstar):
    """Training samples from one iterate of a solve: X [E*N, nin], U [E*N], Eerr [E*N, n_loc] with
    U = s / h_e and Eerr = (x* - x_k) at the element's nodes (all arrays on all nodes, [n_nodes, N])."""
    X, s, h = features(mesh, Rk)
    E, N, nin = X.shape
    err = (np.asarray(Xstar, dtype=np.float64) - np.asarray(Xk, dtype=np.float64))[mesh.elem]   # [E, n_loc, N]
    U = s / h[:, None]
    return X.reshape(E * N, nin), U.reshape(E * N), np.transpose(err, (0, 2, 1)).reshape(E * N, -1)
