"""SVD-based initial factors from the randomized QB, float64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper's remark on initialisation (after Algorithm 1) and its experiments
(Section 4) start the factors from the (randomized) singular value
decomposition, citing Boutsidis and Gallopoulos' nonnegative double SVD
(NNDSVD).  Reading: the leading k singular triplets come from the QB of
Algorithm 1 (B = U_B diag(s) V^T, U = Q U_B: the randomized SVD of
Section 2.3), and NNDSVD maps each triplet to one nonnegative component:
  * j = 1: W_1 = sqrt(s_1) |u_1|, H_1 = sqrt(s_1) |v_1| (the leading singular
    vectors of a nonnegative matrix can be taken nonnegative);
  * j > 1: of the pairs (u+, v+) and (u-, v-) of positive and negative parts
    (x+ = max(x, 0), x- = max(-x, 0)) take the one with the larger
    m = |u.||v.|; W_j = sqrt(s_j m) u./|u.|, H_j = sqrt(s_j m) v./|v.|
    (a zero part gives a zero component).
Replacing (u_j, v_j) by (-u_j, -v_j) swaps the two pairs, so the result does
not depend on the signs the SVD routine returns.
"""
from __future__ import annotations

import numpy as np


def _unit(x):
    n = np.linalg.norm(x)
    return (x / n if n > 0 else np.zeros_like(x)), n


def nndsvd(U, s, V, k: int):
    """Nonnegative factors W (m x k), H (k x n) from the triplets (U_:j, s_j, V_:j), j < k."""
    m, n = U.shape[0], V.shape[0]
    W = np.zeros((m, k))
    H = np.zeros((k, n))
    W[:, 0] = np.sqrt(s[0]) * np.abs(U[:, 0])
    H[0, :] = np.sqrt(s[0]) * np.abs(V[:, 0])
    for j in range(1, k):
        x, y = U[:, j], V[:, j]
        xp, xpn = _unit(np.maximum(x, 0.0))
        yp, ypn = _unit(np.maximum(y, 0.0))
        xn, xnn = _unit(np.maximum(-x, 0.0))
        yn, ynn = _unit(np.maximum(-y, 0.0))
        mp, mn = xpn * ypn, xnn * ynn
        if mp > mn:
            u, v, mm = xp, yp, mp
        else:
            u, v, mm = xn, yn, mn
        W[:, j] = np.sqrt(s[j] * mm) * u
        H[j, :] = np.sqrt(s[j] * mm) * v
    return W, H


def svd_init(Q, B, k: int):
    """NNDSVD of the leading k triplets of the randomized SVD A ~ Q B."""
    Ub, s, Vt = np.linalg.svd(np.asarray(B, np.float64), full_matrices=False)
    return nndsvd(np.asarray(Q, np.float64) @ Ub[:, :k], s[:k], Vt[:k].T, k)
