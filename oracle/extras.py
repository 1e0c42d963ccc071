"""Regularised HALS (Section 3.4) and the projected-gradient stopping measure
(Section 3.3), float64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Regularised objective (elastic net, Section 3.4):
    f(W, H) = ||A - W H||_F^2 + aW ||W||_F^2 + aH ||H||_F^2 + 2 bW sum(W) + 2 bH sum(H),
W, H >= 0 (so ||.||_1 is the plain sum).  The factor 2 on the l1 weights is
the reading that makes the printed l1 rules exact: their derivation drops the
factor 2 of the quadratic term's derivative but not of the l1 term's, i.e. they
minimise (1/2)||R - W_j H_j||^2 + beta ||.||_1.  Minimising f over one component
j with the others fixed gives, for H row j (R = A^T W, S = W^T W):
    H_j <- max(0, (S_jj H_j + R_:j - bH - H^T S_:j) / (S_jj + aH)),
and for W column j (P = A H^T, V = H H^T):
    W_j <- max(0, (V_jj W_j + P_:j - bW - W V_:j) / (V_jj + aW)).
aW = aH = 0 gives the l1 rules of Section 3.4, bW = bH = 0 the l2 rules, both
zero the plain HALS rules of Section 3.1.  (The paper's H rule prints
[W^T W~]_jj in one denominator; it is read as [W^T W]_jj, the quantity of the
derivation.)

Compressed form (randomized, Section 3.2 with the Section 3.4 penalties on the
high-dimensional W = Q W~): the H rule above with R = B^T W~; the W~ column
rule W~_j <- (V_jj W~_j + T_:j - bW Q^T 1 - W~ V_:j) / (V_jj + aW) (no clamp;
bW Q^T 1 is half the gradient of 2 bW sum(Q W~_j) in the compressed
coordinates), then
W_j = max(0, Q W~_j), W~_j = Q^T W_j.

Projected gradient (Section 3.3): with G_W = df/dW, G_H = df/dH of
f = ||A - W H||_F^2, the projected entries are G where the variable is
positive and min(0, G) where it is 0; the measure is ||grad^P||_F^2 and the
stopping test ||grad^P(W, H)||^2 < eps ||grad^P(W0, H0)||^2.  The compressed
measure replaces A by Q B (A H^T -> Q T, W^T A -> W~^T B).
"""
from __future__ import annotations

import numpy as np

from . import philox
from .rhals import rqb


def _h_rows(Rt, S, H, aH, bH):
    """H rows j = 1..k in order (Gauss-Seidel), Rt = R (n x k)."""
    k = H.shape[0]
    for j in range(k):
        sjj = S[j, j]
        if sjj <= 0:
            continue
        H[j] = np.maximum(0.0, (sjj * H[j] + Rt[:, j] - bH - H.T @ S[:, j]) / (sjj + aH))


def hals_reg_sweeps(A, W, H, iters: int, aW=0.0, aH=0.0, bW=0.0, bH=0.0, track: bool = False):
    """Deterministic regularised HALS on the full A (Section 3.4 rules, H rows then
    W columns as Algorithm 1 orders them).  Returns (W, H, objective history)."""
    A = np.asarray(A, np.float64)
    W = np.array(W, np.float64, copy=True)
    H = np.array(H, np.float64, copy=True)
    hist = []
    k = W.shape[1]
    for _ in range(iters):
        _h_rows(A.T @ W, W.T @ W, H, aH, bH)
        P = A @ H.T
        V = H @ H.T
        for j in range(k):
            vjj = V[j, j]
            if vjj <= 0:
                continue
            W[:, j] = np.maximum(0.0, (vjj * W[:, j] + P[:, j] - bW - W @ V[:, j]) / (vjj + aW))
        if track:
            hist.append(reg_objective(A, W, H, aW, aH, bW, bH))
    return W, H, np.array(hist)


def rhals_reg_sweeps(Q, B, W, H, iters: int, aW=0.0, aH=0.0, bW=0.0, bH=0.0, gram_mode: int = 0, A=None,
                     order: int = 0):
    """Compressed regularised sweeps (Section 3.2 with Section 3.4 penalties).
    order 0: all H rows, then all W columns; order 2: the interleaved order
    W_1 -> H_1 -> ... -> W_k -> H_k of Section 3.2, every block from the current
    values.  Returns (W, H, W~, relative-error history if A is given)."""
    W = np.array(W, np.float64, copy=True)
    H = np.array(H, np.float64, copy=True)
    Wt = Q.T @ W
    q1 = Q.T @ np.ones(Q.shape[0])
    k = W.shape[1]
    hist = []

    def w_column(j, t, v):
        vjj = v[j]
        if vjj <= 0:
            return
        Wt[:, j] = (vjj * Wt[:, j] + t - bW * q1 - Wt @ v) / (vjj + aW)
        W[:, j] = np.maximum(0.0, Q @ Wt[:, j])
        Wt[:, j] = Q.T @ W[:, j]

    for _ in range(iters):
        if order == 2:
            for j in range(k):
                w_column(j, B @ H[j], H @ H[j])
                sv = W.T @ W[:, j] if gram_mode == 0 else Wt.T @ Wt[:, j]
                if sv[j] > 0:
                    H[j] = np.maximum(0.0, (sv[j] * H[j] + B.T @ Wt[:, j] - bH - H.T @ sv) / (sv[j] + aH))
        else:
            S = W.T @ W if gram_mode == 0 else Wt.T @ Wt
            _h_rows(B.T @ Wt, S, H, aH, bH)
            T = B @ H.T
            V = H @ H.T
            for j in range(k):
                w_column(j, T[:, j], V[:, j])
        if A is not None:
            hist.append(np.linalg.norm(A - W @ H) / np.linalg.norm(A))
    return W, H, Wt, np.array(hist)


def rhals_reg(A, k: int, p: int, q: int, iters: int, seed: int, aW=0.0, aH=0.0, bW=0.0, bH=0.0,
              gram_mode: int = 0, instance: int = 0):
    """Algorithm 1 with the regularised sweeps: same Omega, QB and initial factors
    as oracle.rhals.rhals."""
    A64 = np.asarray(A, np.float64)
    m, n = A64.shape
    l = k + p
    Q, B = rqb(A64, philox.omega(n, l, seed, 0, instance), q)
    W0, H0 = philox.init_factors(m, n, k, seed, instance)
    W, H, Wt, hist = rhals_reg_sweeps(Q, B, W0, H0, iters, aW, aH, bW, bH, gram_mode, A64)
    return dict(W=W, H=H, Wt=Wt, Q=Q, B=B, hist=hist)


def reg_objective(A, W, H, aW=0.0, aH=0.0, bW=0.0, bH=0.0):
    """The regularised objective f(W, H) of Section 3.4 (elastic net) that the
    update rules minimise exactly component by component."""
    return (np.linalg.norm(A - W @ H) ** 2 + aW * np.sum(W * W) + aH * np.sum(H * H) + 2 * bW * np.sum(W)
            + 2 * bH * np.sum(H))


def _project(G, X):
    return np.where(X > 0, G, np.minimum(0.0, G))


def projected_gradient_sq(A, W, H):
    """||grad^P f(W, H)||_F^2 for f = ||A - W H||_F^2 (Section 3.3)."""
    GW = 2.0 * (W @ (H @ H.T) - A @ H.T)
    GH = 2.0 * ((W.T @ W) @ H - W.T @ A)
    return float(np.sum(_project(GW, W) ** 2) + np.sum(_project(GH, H) ** 2))


def compressed_projected_gradient_sq(Q, B, W, Wt, H):
    """The same measure with A replaced by Q B: A H^T -> Q (B H^T), W^T A -> W~^T B."""
    GW = 2.0 * (W @ (H @ H.T) - Q @ (B @ H.T))
    GH = 2.0 * ((W.T @ W) @ H - Wt.T @ B)
    return float(np.sum(_project(GW, W) ** 2) + np.sum(_project(GH, H) ** 2))


def rqb_blocked(A, Omega, q: int, block_cols: int):
    """Randomized QB over column blocks of A (Algorithm 2, Appendix A): A is read
    one block of columns at a time, 1 + q + 1 passes in all.

        Y = sum_blocks A(:, J) Omega(J, :)
        q times: Q = qr(Y); Y = sum_blocks A(:, J) (A(:, J)^T Q)
        Q = qr(Y); B(:, J) = Q^T A(:, J)

    (The listing's power-iteration line assigns instead of accumulating; it is
    read as the sum over blocks, Y = A A^T Q.)  Returns Q (m x l), B (l x n)."""
    from .rhals import qr_q

    A = np.asarray(A, np.float64)
    m, n = A.shape
    l = Omega.shape[1]
    Y = np.zeros((m, l))
    for c0 in range(0, n, block_cols):
        J = slice(c0, min(n, c0 + block_cols))
        Y += A[:, J] @ Omega[J, :]
    for _ in range(q):
        Q = qr_q(Y)
        Y = np.zeros((m, l))
        for c0 in range(0, n, block_cols):
            J = slice(c0, min(n, c0 + block_cols))
            Y += A[:, J] @ (A[:, J].T @ Q)
    Q = qr_q(Y)
    B = np.zeros((l, n))
    for c0 in range(0, n, block_cols):
        J = slice(c0, min(n, c0 + block_cols))
        B[:, J] = Q.T @ A[:, J]
    return Q, B


def rhals_blocked(A, k: int, p: int, q: int, iters: int, seed: int, block_cols: int, gram_mode: int = 0,
                  instance: int = 0):
    """Algorithm 1's sweeps after the column-blocked QB of Algorithm 2 (same Omega
    and initial factors as oracle.rhals.rhals)."""
    from .rhals import rhals_sweeps

    A64 = np.asarray(A, np.float64)
    m, n = A64.shape
    Q, B = rqb_blocked(A64, philox.omega(n, k + p, seed, 0, instance), q, block_cols)
    W0, H0 = philox.init_factors(m, n, k, seed, instance)
    W, H, Wt, hist = rhals_sweeps(Q, B, W0, H0, iters, gram_mode, A64)
    return dict(W=W, H=H, Wt=Wt, Q=Q, B=B, hist=hist)
