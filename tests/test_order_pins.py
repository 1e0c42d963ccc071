"""Pins of the oracle's shuffled update order (Section 3.2: the components may
be visited in a random order that changes every sweep).

* the visiting order of a sweep is a permutation, reproducible, different
  from sweep to sweep, and uniform over the k! orders (chi-square over 24000
  sweeps of k = 4);
* a shuffled sweep equals the index-order sweep run on factors whose
  components are stored in the visiting order (so the order reaches both
  halves, and nothing else changes);
* k = 1 leaves nothing to shuffle: identical to the index order;
* with gram_mode 1 the H half is exact block coordinate descent on
  ||B - W~ H||_F in any order: the compressed objective never increases
  across H rows, whatever the order.
The interleaved cyclic order (W_1 -> H_1 -> ... -> W_k -> H_k, order 2):
* with k = 1 it is the index-order sweep shifted by half a sweep;
* with Q = I every block update is an exact minimisation, so ||A - W H|| never
  increases from one block update to the next;
* it differs from the index order.
"""
import numpy as np

import synth
from oracle import philox
from oracle import rhals as R


def _problem(m=120, n=90, k=6, p=4, seed=3):
    w = synth.Workload("o", m, n, k, k, p, 1, 0, 0.01, instance=seed)
    A = synth.lowrank(w).astype(np.float64)
    Q, B = R.rqb(A, philox.omega(n, k + p, seed), 1)
    W0, H0 = philox.init_factors(m, n, k, seed)
    return A, Q, B, W0, H0


def test_visiting_order_is_a_reproducible_permutation():
    for k in (1, 2, 3, 4, 5, 17, 100, 128):
        for t in (0, 1, 7, 1000):
            pi = philox.sweep_permutation(k, 11, t)
            assert sorted(pi.tolist()) == list(range(k))
            assert np.array_equal(pi, philox.sweep_permutation(k, 11, t))
    seen = {tuple(philox.sweep_permutation(10, 0, t)) for t in range(50)}
    assert len(seen) == 50
    assert not np.array_equal(philox.sweep_permutation(10, 0, 0), philox.sweep_permutation(10, 1, 0))


def test_visiting_order_is_uniform():
    from itertools import permutations
    index = {p: i for i, p in enumerate(permutations(range(4)))}
    counts = np.zeros(24)
    T = 24000
    for t in range(T):
        counts[index[tuple(philox.sweep_permutation(4, 5, t))]] += 1
    chi2 = ((counts - T / 24) ** 2 / (T / 24)).sum()
    assert chi2 < 49.7  # 23 degrees of freedom, p = 0.001


def test_shuffled_sweep_is_the_cyclic_sweep_on_reordered_components():
    _, Q, B, W0, H0 = _problem()
    for t_sweeps in (1, 3):
        Ws, Hs, Wts, _ = R.rhals_sweeps(Q, B, W0, H0, t_sweeps, order=1, order_seed=9)
        W, H, Wt = W0.copy(), H0.copy(), Q.T @ W0
        for t in range(t_sweeps):
            pi = philox.sweep_permutation(W.shape[1], 9, t)
            Wp, Hp, Wtp, _ = R.rhals_sweeps(Q, B, W[:, pi], H[pi, :], 1, Wt=Wt[:, pi])
            inv = np.argsort(pi)
            W, H, Wt = Wp[:, inv], Hp[inv, :], Wtp[:, inv]
        assert np.max(np.abs(W - Ws)) <= 1e-12 * np.max(np.abs(Ws))
        assert np.max(np.abs(H - Hs)) <= 1e-12 * np.max(np.abs(Hs))
        assert np.max(np.abs(Wt - Wts)) <= 1e-12 * np.max(np.abs(Wts))
    Wc, Hc, _, _ = R.rhals_sweeps(Q, B, W0, H0, 1)
    Ws, Hs, _, _ = R.rhals_sweeps(Q, B, W0, H0, 1, order=1, order_seed=9)
    assert np.max(np.abs(Hc - Hs)) > 1e-6  # the order is used


def test_single_component_is_order_free():
    _, Q, B, W0, H0 = _problem(k=1, p=3)
    a = R.rhals_sweeps(Q, B, W0, H0, 4)
    b = R.rhals_sweeps(Q, B, W0, H0, 4, order=1, order_seed=2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_h_half_descends_in_any_order():
    _, Q, B, W0, H0 = _problem(k=8, p=4)
    Wt = Q.T @ W0
    for seed in range(3):
        H = H0.copy()
        order = philox.sweep_permutation(8, seed, 0)
        f = [np.linalg.norm(B - Wt @ H) ** 2]
        for j in order:
            R.rhals_h_half(B, Wt, W0, H, gram_mode=1, order=[j])
            f.append(np.linalg.norm(B - Wt @ H) ** 2)
        assert all(b <= a * (1 + 1e-12) for a, b in zip(f, f[1:]))
        assert f[-1] < f[0]


# ---- the interleaved cyclic order W_1 -> H_1 -> ... -> W_k -> H_k (order 2)

def test_interleaved_single_component_is_a_half_sweep_shift():
    # with k = 1 the interleaved sweeps are W, H, W, H, ...: one W half, then
    # the index-order sweeps (H half, W half) shifted by half a sweep, then an H half
    _, Q, B, W0, H0 = _problem(k=1, p=3)
    Wi, Hi, _, _ = R.rhals_sweeps(Q, B, W0, H0, 4, order=2)
    W, H = W0.copy(), H0.copy()
    Wt = Q.T @ W
    R.rhals_w_half(B, Q, Wt, W, H)
    W, H, Wt, _ = R.rhals_sweeps(Q, B, W, H, 3, Wt=Wt)
    R.rhals_h_half(B, Wt, W, H)
    assert np.max(np.abs(W - Wi)) <= 1e-12 * np.max(np.abs(Wi))
    assert np.max(np.abs(H - Hi)) <= 1e-12 * np.max(np.abs(Hi))


def test_interleaved_is_block_coordinate_descent_with_full_basis():
    # Q = I (l = m): the compressed problem is the full one and the reprojection
    # is the exact clamp, so every single block update of the interleaved sweep
    # is an exact minimisation: ||A - W H|| never increases between updates
    m, n, k = 30, 40, 5
    w = synth.Workload("bcd", m, n, k, k, m - k, 0, 0, 0.05)
    A = synth.lowrank(w).astype(np.float64)
    Q = np.eye(m)
    W, H = philox.init_factors(m, n, k, 4)
    Wt = Q.T @ W
    f = [np.linalg.norm(A - W @ H)]
    for _ in range(3):
        for j in range(k):
            t = A @ H[j, :]
            v = H @ H[j, :]
            Wt[:, j] = Wt[:, j] + (t - Wt @ v) / v[j]
            W[:, j] = np.maximum(0.0, Q @ Wt[:, j])
            Wt[:, j] = Q.T @ W[:, j]
            f.append(np.linalg.norm(A - W @ H))
            s = W.T @ W[:, j]
            H[j, :] = np.maximum(0.0, H[j, :] + (A.T @ Wt[:, j] - H.T @ s) / s[j])
            f.append(np.linalg.norm(A - W @ H))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(f, f[1:]))
    # and the oracle's interleaved sweeps reproduce those block updates
    W2, H2, _, _ = R.rhals_sweeps(Q, A, *philox.init_factors(m, n, k, 4), 3, order=2)
    assert np.max(np.abs(W2 - W)) <= 1e-12 * np.max(np.abs(W)) and np.max(np.abs(H2 - H)) <= 1e-12 * np.max(np.abs(H))


def test_interleaved_differs_from_the_index_order():
    _, Q, B, W0, H0 = _problem()
    a = R.rhals_sweeps(Q, B, W0, H0, 1)
    b = R.rhals_sweeps(Q, B, W0, H0, 1, order=2)
    assert np.max(np.abs(a[1] - b[1])) > 1e-6
