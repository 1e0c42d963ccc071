"""FP64 oracle of randomized and deterministic HALS (Erichson et al., arXiv:1711.02037).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Every function follows the paper's steps in the paper's order and notation,
in float64, with numpy/LAPACK primitives (matmul, Householder QR) as steps and
no blocking, fusion or reordering.  Readings of points the paper leaves open:

  * Omega is standard Gaussian (Section 2.3) unless dist=1 (uniform, the
    remark on the random test matrix after Algorithm 1).
  * Power iterations re-orthonormalise on both sides (Algorithm 1 QB part;
    subspace iteration as Section 2.3 recommends), 2q+1 QR factorisations.
  * W_tilde starts as Q^T W_init (Algorithm 1 only says "initialise").
  * The reprojection uses Q W_tilde (the rule right after the W_tilde update
    in Section 3.2); Algorithm 1 prints Q W there.
  * T = B H^T is l x k (Algorithm 1 prints k x k).
  * The Gram that scales the H update is S = W^T W (Algorithm 1, and the note
    in Section 3.2 that W^T W is used in practice); gram_mode=1 selects
    S = W_tilde^T W_tilde, the H rule as printed in Section 3.2.
  * A block whose diagonal S_jj (or V_jj) is <= 0 (an all-zero component) is
    left unchanged for that sweep; the paper does not treat this case.
  * Update order: all H rows, then all W columns (Algorithm 1), each in index
    order; order=1 is the shuffled alternative of Section 3.2: sweep t visits
    the components in the order philox.sweep_permutation(k, order_seed, t) in
    both halves; order=2 is the first of Section 3.2's two cyclic orders,
    W_1 -> H_1 -> ... -> W_k -> H_k, each block from the current values of all
    others.
"""
from __future__ import annotations

import numpy as np

from . import philox


def qr_q(Y: np.ndarray) -> np.ndarray:
    """Thin orthonormal factor [Q, ~] = qr(Y) (Householder QR, LAPACK)."""
    return np.linalg.qr(Y, mode="reduced")[0]


def rqb(A: np.ndarray, Omega: np.ndarray, q: int):
    """Randomized QB decomposition, Section 2.3 and the first part of Algorithm 1.

    Y = A Omega; q times { Q = qr(Y); Q = qr(A^T Q); Y = A Q }; Q = qr(Y); B = Q^T A.
    Returns Q (m x l) and B (l x n), both float64.
    """
    A = np.asarray(A, np.float64)
    Y = A @ Omega
    for _ in range(q):
        Q = qr_q(Y)
        Q = qr_q(A.T @ Q)
        Y = A @ Q
    Q = qr_q(Y)
    B = Q.T @ A
    return Q, B


def rel_err(A: np.ndarray, W: np.ndarray, H: np.ndarray) -> float:
    """Relative Frobenius error ||A - W H||_F / ||A||_F (the "Error" of Section 4)."""
    A = np.asarray(A, np.float64)
    return float(np.linalg.norm(A - W @ H) / np.linalg.norm(A))


def objective(A: np.ndarray, W: np.ndarray, H: np.ndarray) -> float:
    """NMF objective f(W, H) = ||A - W H||_F^2 (Section 2.2)."""
    A = np.asarray(A, np.float64)
    return float(np.linalg.norm(A - W @ H) ** 2)


def compressed_objective(B: np.ndarray, Wt: np.ndarray, H: np.ndarray) -> float:
    """Compressed objective f~(W~, H) = ||B - W~ H||_F^2 (Section 3.2)."""
    return float(np.linalg.norm(B - Wt @ H) ** 2)


def rhals_h_half(B, Wt, W, H, gram_mode: int = 0, order=None):
    """H half-sweep of randomized HALS (Section 3.2 H rule, Algorithm 1):
    R = B^T W~, S = W^T W (or W~^T W~), then row by row
    H_j <- max(0, H_j + (R_:j - H^T S_:j) / S_jj).  Updates H in place; returns (R, S)."""
    R = B.T @ Wt
    S = W.T @ W if gram_mode == 0 else Wt.T @ Wt
    k = H.shape[0]
    for j in (range(k) if order is None else order):
        if S[j, j] > 0:
            H[j, :] = np.maximum(0.0, H[j, :] + (R[:, j] - H.T @ S[:, j]) / S[j, j])
    return R, S


def rhals_w_half(B, Q, Wt, W, H, order=None):
    """W half-sweep of randomized HALS (Section 3.2 W~ rule and reprojection, Algorithm 1):
    T = B H^T, V = H H^T, then column by column
    W~_j <- W~_j + (T_:j - W~ V_:j) / V_jj;  W_j <- max(0, Q W~_j);  W~_j <- Q^T W_j.
    Updates Wt and W in place; returns (T, V)."""
    T = B @ H.T
    V = H @ H.T
    k = H.shape[0]
    for j in (range(k) if order is None else order):
        if V[j, j] > 0:
            Wt[:, j] = Wt[:, j] + (T[:, j] - Wt @ V[:, j]) / V[j, j]
            W[:, j] = np.maximum(0.0, Q @ Wt[:, j])
            Wt[:, j] = Q.T @ W[:, j]
    return T, V


def rhals_interleaved_sweep(B, Q, Wt, W, H, gram_mode: int = 0):
    """One sweep in the order W_1 -> H_1 -> ... -> W_k -> H_k (Section 3.2): column j
    of W~ / W from T_:j = B H_j^T and V_:j = H H_j^T of the current H (W~ rule and
    reprojection), then row j of H from R_:j = B^T W~_j and S_:j = W^T W_j (or
    W~^T W~_j) of the current W (H rule).  Updates Wt, W, H in place."""
    k = H.shape[0]
    for j in range(k):
        t = B @ H[j, :]
        v = H @ H[j, :]
        if v[j] > 0:
            Wt[:, j] = Wt[:, j] + (t - Wt @ v) / v[j]
            W[:, j] = np.maximum(0.0, Q @ Wt[:, j])
            Wt[:, j] = Q.T @ W[:, j]
        r = B.T @ Wt[:, j]
        sv = W.T @ W[:, j] if gram_mode == 0 else Wt.T @ Wt[:, j]
        if sv[j] > 0:
            H[j, :] = np.maximum(0.0, H[j, :] + (r - H.T @ sv) / sv[j])


def rhals_sweeps(Q, B, W, H, iters: int, gram_mode: int = 0, A=None, Wt=None, order: int = 0, order_seed: int = 0):
    """`iters` sweeps of Algorithm 1's repeat loop on the compressed problem.

    W (m x k), H (k x n) are copied.  W~ = Q^T W unless given.  If A is given the
    relative error ||A - W H|| / ||A|| after every sweep is returned as well.
    """
    W = np.array(W, np.float64, copy=True)
    H = np.array(H, np.float64, copy=True)
    Wt = Q.T @ W if Wt is None else np.array(Wt, np.float64, copy=True)
    hist = []
    k = H.shape[0]
    for t in range(iters):
        if order == 2:
            rhals_interleaved_sweep(B, Q, Wt, W, H, gram_mode)
        else:
            perm = philox.sweep_permutation(k, order_seed, t) if order == 1 else None
            rhals_h_half(B, Wt, W, H, gram_mode, perm)
            rhals_w_half(B, Q, Wt, W, H, perm)
        if A is not None:
            hist.append(rel_err(A, W, H))
    return W, H, Wt, np.array(hist)


def rhals(A, k: int, p: int, q: int, iters: int, seed: int, gram_mode: int = 0, omega_dist: int = 0,
          track: bool = False, instance: int = 0, order: int = 0, order_seed: int = 0, init: int = 0):
    """Randomized HALS NMF, Algorithm 1: l = k + p, Omega (n x l) from Philox key
    `seed`, randomized QB with q subspace iterations, W_init/H_init ~ U[0,1) from
    key seed + 1 (or, init=1, the SVD-based factors of oracle/init_svd.py), then
    `iters` sweeps.  Returns dict with W, H, Q, B, Wt, Omega, hist."""
    A64 = np.asarray(A, np.float64)
    m, n = A64.shape
    l = k + p
    Om = philox.omega(n, l, seed, omega_dist, instance)
    Q, B = rqb(A64, Om, q)
    if init == 1:  # NNDSVD of the randomized SVD (oracle/init_svd.py)
        from .init_svd import svd_init
        W0, H0 = svd_init(Q, B, k)
    else:
        W0, H0 = philox.init_factors(m, n, k, seed, instance)
    W, H, Wt, hist = rhals_sweeps(Q, B, W0, H0, iters, gram_mode, A64 if track else None, order=order,
                                  order_seed=order_seed)
    return dict(W=W, H=H, Q=Q, B=B, Wt=Wt, Omega=Om, W_init=W0, H_init=H0, hist=hist)


def hals_sweeps(A, W, H, iters: int, track: bool = False):
    """Deterministic HALS with the residual-free rules of Section 3.1, in
    Algorithm 1's order (all H rows, then all W columns):
      R = A^T W, S = W^T W, H_j <- max(0, H_j + (R_:j - H^T S_:j) / S_jj);
      P = A H^T, V = H H^T, W_:j <- max(0, W_:j + (P_:j - W V_:j) / V_jj)."""
    A = np.asarray(A, np.float64)
    W = np.array(W, np.float64, copy=True)
    H = np.array(H, np.float64, copy=True)
    k = H.shape[0]
    hist = []
    for _ in range(iters):
        R = A.T @ W
        S = W.T @ W
        for j in range(k):
            if S[j, j] > 0:
                H[j, :] = np.maximum(0.0, H[j, :] + (R[:, j] - H.T @ S[:, j]) / S[j, j])
        P = A @ H.T
        V = H @ H.T
        for j in range(k):
            if V[j, j] > 0:
                W[:, j] = np.maximum(0.0, W[:, j] + (P[:, j] - W @ V[:, j]) / V[j, j])
        if track:
            hist.append(rel_err(A, W, H))
    return W, H, np.array(hist)


def hals(A, k: int, iters: int, seed: int, track: bool = False, instance: int = 0):
    """Deterministic HALS from the same W_init/H_init as rhals(seed)."""
    A64 = np.asarray(A, np.float64)
    m, n = A64.shape
    W0, H0 = philox.init_factors(m, n, k, seed, instance)
    W, H, hist = hals_sweeps(A64, W0, H0, iters, track)
    return dict(W=W, H=H, W_init=W0, H_init=H0, hist=hist)
