"""Reference gradient of <G, W_T H_T> through T compressed HALS sweeps (float64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The forward pass is Algorithm 1's repeat loop (Section 3.2 H rule, W~ rule and
reprojection), written again with torch float64 CPU operations so that torch's
reverse-mode autograd (a library primitive) supplies the reference gradient:
  * Q is held fixed (computed from A without gradient); A reaches the sweeps
    only through B = Q^T A, so dL/dA = Q dL/dB;
  * the initial factors W_init, H_init are inputs; W~ starts as Q^T W_init;
  * max(0, x) is torch.relu, whose subgradient at exactly 0 is 0;
  * a block whose diagonal S_jj (V_jj) is <= 0 is skipped, as in rhals.py.
The pins are central finite differences of the same forward pass
(tests/test_adjoint_pins.py); `masks` exposes every clamp decision so that a
finite-difference direction crossing a kink can be rejected.
"""
from __future__ import annotations

import numpy as np
import torch


def sweeps(Q, B, W0, H0, T: int, gram_mode: int = 0, record_masks: bool = False, record_args=None):
    """T compressed sweeps from (W0, H0); returns (W_T, H_T, masks).  All inputs are
    float64 torch tensors; gradients flow to B, W0, H0 (whichever require grad).
    If record_args is a list, every clamp argument is appended to it as
    (sweep t = 1..T, "H" or "W", component j, argument array)."""
    W = W0
    H = H0
    Wt = Q.T @ W
    k = H.shape[0]
    masks = []
    for t in range(T):
        # H half: R = B^T W~, S = W^T W (or W~^T W~); rows j = 1..k in order
        R = B.T @ Wt
        S = W.T @ W if gram_mode == 0 else Wt.T @ Wt
        rows = [H[j] for j in range(k)]
        for j in range(k):
            sjj = S[j, j]
            if float(sjj.detach()) > 0:
                Hcur = torch.stack(rows)
                a = rows[j] + (R[:, j] - Hcur.T @ S[:, j]) / sjj
                if record_masks:
                    masks.append((a.detach() > 0).numpy().copy())
                if record_args is not None:
                    record_args.append((t + 1, "H", j, a.detach().numpy().copy()))
                rows[j] = torch.relu(a)
        H = torch.stack(rows)
        # W half: T = B H^T, V = H H^T; columns j = 1..k in order
        Tm = B @ H.T
        V = H @ H.T
        wt_cols = [Wt[:, j] for j in range(k)]
        w_cols = [W[:, j] for j in range(k)]
        for j in range(k):
            vjj = V[j, j]
            if float(vjj.detach()) > 0:
                Wtc = torch.stack(wt_cols, dim=1)
                u = wt_cols[j] + (Tm[:, j] - Wtc @ V[:, j]) / vjj
                z = Q @ u
                if record_masks:
                    masks.append((z.detach() > 0).numpy().copy())
                if record_args is not None:
                    record_args.append((t + 1, "W", j, z.detach().numpy().copy()))
                w_cols[j] = torch.relu(z)
                wt_cols[j] = Q.T @ w_cols[j]
        W = torch.stack(w_cols, dim=1)
        Wt = torch.stack(wt_cols, dim=1)
    return W, H, masks


def loss_and_grads(A, Q, W0, H0, G, T: int, gram_mode: int = 0):
    """L = <G, W_T H_T> and its gradients with respect to A (Q fixed), W0, H0.

    A, Q, W0, H0, G: numpy arrays (any float dtype; used as float64)."""
    At = torch.tensor(np.asarray(A, np.float64), requires_grad=True)
    Qt = torch.tensor(np.asarray(Q, np.float64))
    W0t = torch.tensor(np.asarray(W0, np.float64), requires_grad=True)
    H0t = torch.tensor(np.asarray(H0, np.float64), requires_grad=True)
    Gt = torch.tensor(np.asarray(G, np.float64))
    B = Qt.T @ At
    W, H, _ = sweeps(Qt, B, W0t, H0t, T, gram_mode)
    L = (Gt * (W @ H)).sum()
    L.backward()
    return float(L.detach()), At.grad.numpy(), W0t.grad.numpy(), H0t.grad.numpy()


def loss(A, Q, W0, H0, G, T: int, gram_mode: int = 0, record_masks: bool = False):
    """Forward only: L = <G, W_T H_T> (and the clamp decisions if requested)."""
    with torch.no_grad():
        Qt = torch.tensor(np.asarray(Q, np.float64))
        B = Qt.T @ torch.tensor(np.asarray(A, np.float64))
        W, H, masks = sweeps(Qt, B, torch.tensor(np.asarray(W0, np.float64)),
                             torch.tensor(np.asarray(H0, np.float64)), T, gram_mode, record_masks)
        L = float((torch.tensor(np.asarray(G, np.float64)) * (W @ H)).sum())
    return (L, masks) if record_masks else L


def clamp_arguments(A, Q, W0, H0, T: int, gram_mode: int = 0):
    """Every clamp argument of the forward pass: [(t, "H" | "W", j, values)], with
    values the n entries of row j's argument (H) or the m entries of column j's
    Q u_j (W), in the order the sweeps evaluate them."""
    out = []
    with torch.no_grad():
        Qt = torch.tensor(np.asarray(Q, np.float64))
        B = Qt.T @ torch.tensor(np.asarray(A, np.float64))
        sweeps(Qt, B, torch.tensor(np.asarray(W0, np.float64)), torch.tensor(np.asarray(H0, np.float64)), T,
               gram_mode, record_args=out)
    return out
