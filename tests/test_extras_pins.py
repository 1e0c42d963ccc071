"""Pins of oracle/extras.py: regularised HALS (Section 3.4) and the projected
gradient (Section 3.3), against what the mathematics fixes.

* zero penalties reproduce the plain sweeps of oracle/rhals.py;
* every regularised H row / W column update is the exact minimiser of its
  one-dimensional problem (dense grid search on tiny inputs);
* deterministic regularised HALS never increases the regularised objective
  (block coordinate descent), and the compressed H half never increases the
  compressed one when S = W~^T W~;
* with a square orthogonal Q (l = m) the compressed regularised sweeps equal the
  deterministic ones;
* interleaved order (W_1 -> H_1 -> ... -> W_k -> H_k): zero penalties give the
  plain interleaved sweeps of oracle/rhals.py; with k = 1 it is the index
  order shifted by half a sweep (so its H rule is the grid-pinned one); with
  Q = I every sweep is block coordinate descent on the regularised objective;
* the projected gradient's gradient agrees with central differences, its
  projection rule is the definition entry by entry, it vanishes at an exact
  nonnegative factorisation, and the compressed measure equals the full one
  for a square Q.
"""
import numpy as np
import pytest

import synth
from oracle import extras as X
from oracle import philox
from oracle import rhals as R

PENS = [(0.5, 0.0, 0.0, 0.0), (0.0, 0.3, 0.0, 0.0), (0.0, 0.0, 0.2, 0.0), (0.0, 0.0, 0.0, 0.4),
        (0.3, 0.2, 0.1, 0.05)]


def small(m=40, n=30, r=4, seed=0):
    w = synth.Workload("x", m, n, r, r, 3, 1, 5, 0.01, instance=seed)
    A = synth.lowrank(w).astype(np.float64)
    W0, H0 = philox.init_factors(m, n, r, seed)
    return A, W0, H0


def test_zero_penalties_reduce_to_plain_sweeps():
    A, W0, H0 = small()
    Wr, Hr = R.hals_sweeps(A, W0, H0, 7)[:2]
    Wx, Hx, _ = X.hals_reg_sweeps(A, W0, H0, 7)
    assert np.allclose(Wx, Wr, rtol=1e-11, atol=1e-12) and np.allclose(Hx, Hr, rtol=1e-11, atol=1e-12)
    Q, B = R.rqb(A, philox.omega(A.shape[1], 7, 0), 1)
    for gm in (0, 1):
        Wr, Hr, _, _ = R.rhals_sweeps(Q, B, W0, H0, 7, gm)
        Wx, Hx, _, _ = X.rhals_reg_sweeps(Q, B, W0, H0, 7, gram_mode=gm)
        assert np.allclose(Wx, Wr, rtol=1e-11, atol=1e-12) and np.allclose(Hx, Hr, rtol=1e-11, atol=1e-12)


def grid_min(f, hi):
    xs = np.linspace(0.0, hi, 400001)
    return xs[np.argmin(f(xs))]


@pytest.mark.parametrize("pen", PENS)
def test_single_updates_are_exact_one_dimensional_minimisers(pen):
    aW, aH, bW, bH = pen
    rng = np.random.default_rng(3)
    m, n, k = 6, 5, 3
    A = rng.random((m, n))
    W = rng.random((m, k))
    H = rng.random((k, n))
    # one H half, then check row j = 0 entries (rows updated first see the initial others)
    H1 = H.copy()
    X._h_rows(A.T @ W, W.T @ W, H1, aH, bH)
    j = 0
    Rj = A - np.delete(W, j, 1) @ np.delete(H, j, 0)
    for c in range(n):
        f = lambda h: np.sum((Rj[:, c][:, None] - W[:, j][:, None] * h[None, :]) ** 2, 0) + aH * h * h + 2 * bH * h
        assert abs(H1[j, c] - grid_min(f, 20.0)) < 1e-4
    # one W column update (deterministic rule) for column 0 from (W, H1)
    P = A @ H1.T
    V = H1 @ H1.T
    wnew = np.maximum(0.0, (V[0, 0] * W[:, 0] + P[:, 0] - bW - W @ V[:, 0]) / (V[0, 0] + aW))
    Rj = A - np.delete(W, 0, 1) @ np.delete(H1, 0, 0)
    for i in range(m):
        f = lambda x: np.sum((Rj[i][None, :] - x[:, None] * H1[0][None, :]) ** 2, 1) + aW * x * x + 2 * bW * x
        assert abs(wnew[i] - grid_min(f, 20.0)) < 1e-4


@pytest.mark.parametrize("pen", PENS)
def test_deterministic_regularised_objective_non_increasing(pen):
    A, W0, H0 = small(seed=1)
    _, _, hist = X.hals_reg_sweeps(A, W0, H0, 25, *pen, track=True)
    f0 = X.reg_objective(A, W0, H0, *pen)
    h = np.concatenate([[f0], hist])
    assert np.all(np.diff(h) <= 1e-12 * h[:-1])


@pytest.mark.parametrize("pen", PENS)
def test_compressed_h_half_descends(pen):
    aW, aH, bW, bH = pen
    A, W0, H0 = small(seed=2)
    Q, B = R.rqb(A, philox.omega(A.shape[1], 7, 0), 1)
    Wt = Q.T @ W0
    H = np.array(H0, copy=True)
    f = lambda H: np.linalg.norm(B - Wt @ H) ** 2 + aH * np.sum(H * H) + 2 * bH * np.sum(H)
    before = f(H)
    X._h_rows(B.T @ Wt, Wt.T @ Wt, H, aH, bH)
    assert f(H) <= before * (1 + 1e-13)


@pytest.mark.parametrize("pen", PENS)
def test_square_q_equals_deterministic(pen):
    A, W0, H0 = small(m=30, n=40, seed=3)
    Q, B = R.rqb(A, philox.omega(A.shape[1], 30, 0), 1)  # l = m: Q square orthogonal
    Wd, Hd, _ = X.hals_reg_sweeps(A, W0, H0, 6, *pen)
    Wc, Hc, _, _ = X.rhals_reg_sweeps(Q, B, W0, H0, 6, *pen)
    assert np.allclose(Wc, Wd, rtol=1e-9, atol=1e-10) and np.allclose(Hc, Hd, rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("gram_mode", [0, 1])
def test_interleaved_zero_penalties_is_the_plain_interleaved_order(gram_mode):
    A, W0, H0 = small(m=50, n=35, r=5, seed=4)
    Q, B = R.rqb(A, philox.omega(A.shape[1], 9, 1), 1)
    Wp, Hp, Wtp, _ = R.rhals_sweeps(Q, B, W0, H0, 3, gram_mode, order=2)
    Wx, Hx, Wtx, _ = X.rhals_reg_sweeps(Q, B, W0, H0, 3, gram_mode=gram_mode, order=2)
    assert np.allclose(Wx, Wp, rtol=1e-11, atol=1e-12) and np.allclose(Hx, Hp, rtol=1e-11, atol=1e-12)
    assert np.allclose(Wtx, Wtp, rtol=1e-11, atol=1e-12)
    Wc = X.rhals_reg_sweeps(Q, B, W0, H0, 1, 0.2, 0.1, 0.05, 0.3, order=2)[1]
    assert np.max(np.abs(Wc - X.rhals_reg_sweeps(Q, B, W0, H0, 1, 0.2, 0.1, 0.05, 0.3)[1])) > 1e-6


@pytest.mark.parametrize("pen", PENS)
def test_interleaved_single_component_is_a_half_sweep_shift(pen):
    # k = 1: W, H, W, H, ... = one W update, the index-order sweeps, then one H row
    A, W0, H0 = small(m=30, n=25, r=1, seed=6)
    Q, B = R.rqb(A, philox.omega(A.shape[1], 4, 2), 1)
    aH, bH = pen[1], pen[3]
    for gm in (0, 1):
        Wi, Hi, _, _ = X.rhals_reg_sweeps(Q, B, W0, H0, 4, *pen, gram_mode=gm, order=2)
        W1 = X.rhals_reg_sweeps(Q, B, W0, H0, 1, *pen, gram_mode=gm, order=2)[0]
        Wa, Ha, Wta, _ = X.rhals_reg_sweeps(Q, B, W1, H0, 3, *pen, gram_mode=gm)
        X._h_rows(B.T @ Wta, Wa.T @ Wa if gm == 0 else Wta.T @ Wta, Ha, aH, bH)
        assert np.allclose(Wa, Wi, rtol=1e-11, atol=1e-12) and np.allclose(Ha, Hi, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("pen", PENS)
def test_interleaved_regularised_descends_with_full_basis(pen):
    # Q = I: W~ = W and the W~ rule is the exact regularised W rule, so every
    # block update minimises the regularised objective over its block
    A, W0, H0 = small(m=20, n=30, r=4, seed=8)
    Q, B = np.eye(20), A
    W, H = W0, H0
    f = [X.reg_objective(A, W, H, *pen)]
    for _ in range(8):
        W, H, _, _ = X.rhals_reg_sweeps(Q, B, W, H, 1, *pen, order=2)
        f.append(X.reg_objective(A, W, H, *pen))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(f, f[1:]))
    assert f[1] < f[0]


def test_projected_gradient_definition_and_finite_differences():
    rng = np.random.default_rng(5)
    m, n, k = 7, 6, 3
    A = rng.random((m, n))
    W = np.maximum(0.0, rng.standard_normal((m, k)))
    H = np.maximum(0.0, rng.standard_normal((k, n)))
    f = lambda W, H: np.linalg.norm(A - W @ H) ** 2
    h = 1e-6
    pg = 0.0
    for X_, which in ((W, "W"), (H, "H")):
        for idx in np.ndindex(*X_.shape):
            E = np.zeros_like(X_)
            E[idx] = h
            if which == "W":
                g = (f(W + E, H) - f(W - E, H)) / (2 * h)
            else:
                g = (f(W, H + E) - f(W, H - E)) / (2 * h)
            p = g if X_[idx] > 0 else min(0.0, g)
            pg += p * p
    assert abs(X.projected_gradient_sq(A, W, H) - pg) <= 1e-6 * pg


def test_projected_gradient_vanishes_at_exact_factorisation():
    rng = np.random.default_rng(6)
    W = rng.random((9, 3))
    H = rng.random((3, 8))
    A = W @ H
    Wz = W.copy()
    Wz[0, 0] = 0.0  # a zero entry with a nonnegative gradient is KKT-stationary too
    assert X.projected_gradient_sq(A, W, H) <= 1e-24 * np.linalg.norm(A) ** 4
    assert X.projected_gradient_sq(A, W, H) < X.projected_gradient_sq(A, W * 1.1, H)


def test_compressed_measure_equals_full_for_square_q():
    A, W0, H0 = small(m=30, n=40, seed=4)
    Q, B = R.rqb(A, philox.omega(A.shape[1], 30, 0), 1)
    assert np.isclose(X.compressed_projected_gradient_sq(Q, B, W0, Q.T @ W0, H0),
                      X.projected_gradient_sq(A, W0, H0), rtol=1e-10)


# ---- column-blocked QB (Algorithm 2)
def subspace_gap(Q1, Q2):
    """sin of the largest principal angle between range(Q1) and range(Q2)."""
    return np.linalg.norm(Q1 - Q2 @ (Q2.T @ Q1), 2)


@pytest.mark.parametrize("bc", [1, 7, 64, 500])
def test_blocked_qb_without_power_iterations_is_the_plain_qb(bc):
    w = synth.Workload("b", 300, 200, 6, 6, 4, 0, 1, 0.01)
    A = synth.lowrank(w).astype(np.float64)
    Om = philox.omega(200, 10, 0)
    Q1, B1 = R.rqb(A, Om, 0)
    Q2, B2 = X.rqb_blocked(A, Om, 0, bc)
    assert np.allclose(Q2 @ B2, Q1 @ B1, rtol=1e-10, atol=1e-10)
    assert subspace_gap(Q1, Q2) < 1e-10


@pytest.mark.parametrize("q", [1, 2])
def test_blocked_qb_ignores_block_size_and_matches_the_subspace_iteration(q):
    # block-size independence, Q^T Q = I, B = Q^T A, and an approximation error
    # within 1% of Algorithm 1's subspace iteration (both converge to the dominant
    # subspace) and above the optimal rank-l error (Eckart-Young)
    w = synth.Workload("b", 300, 200, 6, 6, 4, 0, 1, 0.05)
    A = synth.lowrank(w).astype(np.float64)
    Om = philox.omega(200, 10, 0)
    Qa, Ba = X.rqb_blocked(A, Om, q, 13)
    Qb, Bb = X.rqb_blocked(A, Om, q, 200)
    assert np.allclose(Qa @ Ba, Qb @ Bb, rtol=1e-9, atol=1e-9)
    assert np.allclose(Qa.T @ Qa, np.eye(10), atol=1e-12)
    assert np.allclose(Ba, Qa.T @ A, atol=1e-10)
    Q1, B1 = R.rqb(A, Om, q)
    e_blocked = np.linalg.norm(A - Qa @ Ba)
    e_alg1 = np.linalg.norm(A - Q1 @ B1)
    s = np.linalg.svd(A, compute_uv=False)
    e_opt = np.sqrt(np.sum(s[10:] ** 2))
    assert e_opt * (1 - 1e-12) <= e_blocked <= 1.01 * e_alg1


def test_blocked_qb_exact_on_low_rank():
    # A = W0 H0 of rank 5 in float64, l = 8: range(A) lies in range(Q)
    w = synth.Workload("b", 120, 90, 5, 5, 3, 0, 1, 0.0)
    W0, H0 = synth.factors(w)
    A = W0 @ H0
    for q in (0, 1, 2):
        Q, B = X.rqb_blocked(A, philox.omega(90, 8, 0), q, 11)
        assert np.linalg.norm(A - Q @ B) <= 1e-12 * np.linalg.norm(A)


# ---- SVD-based initialisation (NNDSVD of the randomized SVD), oracle/init_svd.py

def test_nndsvd_rank_one_nonnegative_matrix_is_exact():
    from oracle import init_svd as I
    rng = np.random.default_rng(0)
    w, h = rng.random(40), rng.random(30)
    A = np.outer(w, h)
    U, s, Vt = np.linalg.svd(A)
    W, H = I.nndsvd(U, s, Vt.T, 1)
    assert np.max(np.abs(W @ H - A)) <= 1e-12 * np.max(A)


def test_nndsvd_is_sign_invariant_and_nonnegative():
    from oracle import init_svd as I
    A = synth.lowrank(synth.Workload("s", 60, 50, 6, 6, 2, 0, 0, 0.05)).astype(np.float64)
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    U, V = U[:, :6], Vt[:6].T
    W1, H1 = I.nndsvd(U, s, V, 6)
    flip = np.array([1, -1, 1, -1, -1, 1.0])
    W2, H2 = I.nndsvd(U * flip, s, V * flip, 6)
    assert np.array_equal(W1, W2) and np.array_equal(H1, H2)
    assert W1.min() >= 0 and H1.min() >= 0
    # component j's product is a nonnegative rank-one piece no larger than s_j in norm
    for j in range(6):
        assert np.linalg.norm(np.outer(W1[:, j], H1[j])) <= s[j] * (1 + 1e-12)


def test_svd_init_from_exact_qb_equals_nndsvd_of_the_matrix():
    # with q power iterations on an exactly rank-r matrix the randomized SVD is the SVD
    from oracle import init_svd as I
    m, n, r = 80, 70, 5
    rng = np.random.default_rng(1)
    A = rng.random((m, r)) @ rng.random((r, n))
    Q, B = R.rqb(A, philox.omega(n, r + 3, 0), 2)
    W1, H1 = I.svd_init(Q, B, r)
    U, s, Vt = np.linalg.svd(A)
    W2, H2 = I.nndsvd(U, s, Vt.T, r)
    assert np.max(np.abs(W1 - W2)) <= 1e-9 * np.max(W2) and np.max(np.abs(H1 - H2)) <= 1e-9 * np.max(H2)
