"""Pins of the FP64 oracle (oracle/rhals.py) against what the paper and mathematics fix.

Each check is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand, a missing power iteration) fails:
  * every HALS block step is the exact minimiser of its 1-D (nonnegative)
    least-squares problem (Section 3.1 derivation), checked by brute force;
  * deterministic HALS never increases ||A - WH|| (exact block coordinate descent);
  * Q^T Q = I, exact recovery of the range of an exactly low-rank A, and the
    expected QB error bound of Section 2.3;
  * span(Q) equals span((A A^T)^q A Omega), the power scheme of Section 2.3;
  * with l = m (Q square and orthogonal) randomized HALS reduces to
    deterministic HALS, and its output does not depend on the basis of range(Q);
  * near machine-precision recovery of an exactly low-rank A (Section 4.4).
"""
import math

import numpy as np
import pytest

import synth
from oracle import philox
from oracle import rhals as R


def _rand(shape, seed):
    return np.random.default_rng(seed).random(shape)


def _argmin_nonneg_1d(g, hi):
    """Brute force: minimise the convex 1-D function g over [0, hi] on a dense
    grid, then refine by golden-section search around the best grid point."""
    xs = np.linspace(0.0, hi, 4001)
    vals = np.array([g(x) for x in xs])
    i = int(np.argmin(vals))
    a, b = xs[max(i - 1, 0)], xs[min(i + 1, len(xs) - 1)]
    phi = (math.sqrt(5) - 1) / 2
    for _ in range(200):
        c, d = b - phi * (b - a), a + phi * (b - a)
        if g(c) <= g(d):
            b = d
        else:
            a = c
    return 0.5 * (a + b)


def _check_rows_are_bcd_minimisers(X, W, H_old, H_new):
    """Row j of H_new minimises ||X - sum_{i != j} W_i H_i - W_j h||^2 over h >= 0,
    column by column, with rows < j already updated (Gauss-Seidel)."""
    k = H_old.shape[0]
    for j in range(k):
        Hmix = np.vstack([H_new[:j], H_old[j:]])
        for c in range(X.shape[1]):
            resid = X[:, c] - W @ Hmix[:, c] + W[:, j] * Hmix[j, c]
            g = lambda h: float(np.sum((resid - W[:, j] * h) ** 2))  # noqa: E731
            hi = 2.0 * max(abs(resid @ W[:, j]) / (W[:, j] @ W[:, j]), H_new[j, c], 1e-3)
            hstar = _argmin_nonneg_1d(g, hi)
            assert abs(H_new[j, c] - hstar) <= 1e-6 * max(1.0, hstar), (j, c, H_new[j, c], hstar)
            assert g(H_new[j, c]) <= g(hstar) * (1 + 1e-12) + 1e-14


def test_hals_h_rows_are_exact_nonnegative_minimisers():
    A = _rand((7, 5), 1) @ _rand((5, 9), 2) - 0.3  # some negative entries make clamps active
    W = _rand((7, 3), 3)
    H = _rand((3, 9), 4)
    W1, H1, _ = R.hals_sweeps(A, W, H, 1)
    assert np.any(H1 == 0.0), "test should exercise the clamp"
    _check_rows_are_bcd_minimisers(A, W, H, H1)


def test_hals_w_columns_are_exact_nonnegative_minimisers():
    A = _rand((8, 6), 5) @ _rand((6, 7), 6) - 0.3
    W = _rand((8, 3), 7)
    H = _rand((3, 7), 8)
    W1, H1, _ = R.hals_sweeps(A, W, H, 1)
    # W columns use the updated H; transpose the problem: X^T ~ H^T W^T.
    _check_rows_are_bcd_minimisers(A.T, H1.T, W.T, W1.T)


def test_rhals_h_rows_minimise_the_compressed_problem():
    # gram_mode 1 (S = W~^T W~): the H rule of Section 3.2 is the exact BCD step
    # on ||B - W~ H||^2.
    rng = np.random.default_rng(9)
    B = rng.standard_normal((5, 8))
    Wt = rng.standard_normal((5, 3))
    W = rng.random((10, 3))
    H = rng.random((3, 8))
    H1 = H.copy()
    R.rhals_h_half(B, Wt, W, H1, gram_mode=1)
    assert np.any(H1 == 0.0)
    _check_rows_are_bcd_minimisers(B, Wt, H, H1)


def test_rhals_w_columns_are_least_squares_then_reprojected():
    rng = np.random.default_rng(10)
    m, n, l, k = 12, 9, 5, 3
    Q = R.qr_q(rng.standard_normal((m, l)))
    B = rng.standard_normal((l, n))
    W = rng.random((m, k))
    Wt = Q.T @ W
    H = rng.random((k, n))
    Wt1, W1 = Wt.copy(), W.copy()
    R.rhals_w_half(B, Q, Wt1, W1, H)
    for j in range(k):
        Wt_mix = np.hstack([Wt1[:, :j], Wt[:, j:]])
        resid = B - Wt_mix @ H + np.outer(Wt_mix[:, j], H[j])
        # unconstrained least squares min_w ||resid - w H_j||_F (library lstsq)
        w = np.linalg.lstsq(H[j][:, None], resid.T, rcond=None)[0][0]
        assert np.allclose(W1[:, j], np.maximum(0.0, Q @ w), rtol=1e-12, atol=1e-12)
        assert np.allclose(Wt1[:, j], Q.T @ W1[:, j], rtol=1e-12, atol=1e-12)
    assert np.all(W1 >= 0)


def test_deterministic_hals_objective_non_increasing():
    w = synth.Workload("t", 120, 80, 6, 6, 0, 0, 0, 0.05)
    A = synth.lowrank(w)
    out = R.hals(A, 6, 150, seed=3, track=True)
    f = out["hist"] ** 2
    assert np.all(np.diff(f) <= 1e-12 * f[:-1])
    assert f[-1] < 0.1 * f[0]
    assert np.all(out["W"] >= 0) and np.all(out["H"] >= 0)


def test_qb_orthonormal_and_exact_on_low_rank():
    w = synth.Workload("t", 200, 150, 7, 7, 5, 2, 0, 0.0)
    W0, H0 = synth.factors(w)
    A = W0 @ H0  # exactly rank 7 in float64
    Om = philox.omega(150, 12, 0)
    Q, B = R.rqb(A, Om, 2)
    assert Q.shape == (200, 12) and B.shape == (12, 150)
    assert np.max(np.abs(Q.T @ Q - np.eye(12))) < 1e-13
    assert np.linalg.norm(A - Q @ B) / np.linalg.norm(A) < 1e-12


def _spectral_test_matrix(m, n, sig, seed):
    rng = np.random.default_rng(seed)
    U = R.qr_q(rng.standard_normal((m, len(sig))))
    V = R.qr_q(rng.standard_normal((n, len(sig))))
    return (U * sig) @ V.T


@pytest.mark.parametrize("q", [0, 1, 2])
def test_qb_error_within_expected_bound(q):
    # Section 2.3: E||A - QB||_2 <= [1 + sqrt(k/(p-1)) + e sqrt(k+p)/p sqrt(n-k)]^(1/(2q+1)) sigma_{k+1}
    m, n, k, p = 150, 100, 10, 5
    sig = 0.7 ** np.arange(n)
    A = _spectral_test_matrix(m, n, sig, 1)
    errs = []
    for seed in range(20):
        Om = philox.omega(n, k + p, seed)
        Q, B = R.rqb(A, Om, q)
        errs.append(np.linalg.norm(A - Q @ B, 2))
    bound = (1 + math.sqrt(k / (p - 1)) + math.e * math.sqrt(k + p) / p * math.sqrt(n - k)) ** (1 / (2 * q + 1)) * sig[k]
    assert np.mean(errs) <= bound
    # and never better than the optimum sigma_{k+p+1} (Eckart-Young)
    assert min(errs) >= sig[k + p] * (1 - 1e-9)


def test_power_scheme_spans_the_powered_sketch():
    # span(Q) of Algorithm 1 equals span((A A^T)^q A Omega) (Section 2.3 power scheme)
    m, n, l, q = 60, 40, 6, 2
    sig = np.linspace(3.0, 1.0, n)  # mild spectrum: the direct power is well conditioned
    A = _spectral_test_matrix(m, n, sig, 4)
    Om = philox.omega(n, l, 5)
    Q, _ = R.rqb(A, Om, q)
    Y = np.linalg.matrix_power(A @ A.T, q) @ A @ Om
    Qd = R.qr_q(Y)
    assert np.max(np.abs(Q @ Q.T - Qd @ Qd.T)) < 1e-10
    # a scheme without the A^T half-step would span something else
    Qbad = R.qr_q(A @ Om)
    assert np.max(np.abs(Qbad @ Qbad.T - Qd @ Qd.T)) > 1e-3


@pytest.mark.parametrize("gram_mode", [0, 1])
def test_square_q_reduces_rhals_to_deterministic_hals(gram_mode):
    m, n, k, p = 6, 10, 2, 4   # l = k + p = m: Q square orthogonal, Q Q^T = I
    A = _rand((m, 3), 11) @ _rand((3, n), 12)
    W0, H0 = philox.init_factors(m, n, k, 0)
    Q, B = R.rqb(A, philox.omega(n, k + p, 0), 2)
    Wr, Hr, _, hr = R.rhals_sweeps(Q, B, W0, H0, 40, gram_mode, A=A)
    Wd, Hd, hd = R.hals_sweeps(A, W0, H0, 40, track=True)
    assert np.allclose(Wr, Wd, rtol=1e-10, atol=1e-12)
    assert np.allclose(Hr, Hd, rtol=1e-10, atol=1e-12)
    assert np.allclose(hr, hd, rtol=1e-10)


@pytest.mark.parametrize("gram_mode", [0, 1])
def test_rhals_invariant_to_basis_of_range(gram_mode):
    w = synth.Workload("t", 90, 60, 5, 5, 5, 1, 0, 0.02)
    A = synth.lowrank(w).astype(np.float64)
    Q, B = R.rqb(A, philox.omega(60, 10, 0), 1)
    U = R.qr_q(np.random.default_rng(13).standard_normal((10, 10)))
    W0, H0 = philox.init_factors(90, 60, 5, 0)
    W1, H1, _, _ = R.rhals_sweeps(Q, B, W0, H0, 30, gram_mode)
    W2, H2, _, _ = R.rhals_sweeps(Q @ U, U.T @ B, W0, H0, 30, gram_mode)
    assert np.allclose(W1, W2, rtol=1e-10, atol=1e-12)
    assert np.allclose(H1, H2, rtol=1e-10, atol=1e-12)


def test_compressed_h_half_is_a_descent_step():
    w = synth.Workload("t", 100, 70, 5, 5, 5, 1, 0, 0.02)
    A = synth.lowrank(w).astype(np.float64)
    Q, B = R.rqb(A, philox.omega(70, 10, 0), 1)
    W, H = philox.init_factors(100, 70, 5, 0)
    Wt = Q.T @ W
    for _ in range(20):
        f0 = R.compressed_objective(B, Wt, H)
        R.rhals_h_half(B, Wt, W, H, gram_mode=1)
        f1 = R.compressed_objective(B, Wt, H)
        assert f1 <= f0 * (1 + 1e-12)
        R.rhals_w_half(B, Q, Wt, W, H)
        assert np.all(W >= 0) and np.all(H >= 0)


def test_near_exact_recovery_of_low_rank_data():
    # Section 4.4: on exactly low-rank nonnegative data rHALS reaches nearly
    # machine precision.  A = fl32(W0 H0) with 60% of H0 zero (identifiable NMF);
    # the float32 rounding floor is ~2.5e-8.
    w = synth.Workload("t", 300, 200, 4, 4, 6, 2, 2000, 0.0, h0_zero_frac=0.6)
    A = synth.lowrank(w)
    out = R.rhals(A, 4, 6, 2, 2000, seed=0, track=True)
    assert out["hist"][-1] < 1e-6
    assert out["hist"][0] > 1e-2
    assert np.all(out["W"] >= 0) and np.all(out["H"] >= 0)


def test_noisy_data_error_near_noise_level():
    w = synth.SMALL
    A = synth.lowrank(w)
    out = R.rhals(A, w.k, w.p, w.q, w.iters, w.seed, track=True)
    # the reachable error is bounded below by the best rank-k approximation
    A64 = A.astype(np.float64)
    s = np.linalg.svd(A64, compute_uv=False)
    best = math.sqrt(np.sum(s[w.k:] ** 2)) / np.linalg.norm(A64)
    assert out["hist"][-1] >= best * (1 - 1e-9)
    assert out["hist"][-1] < out["hist"][0]


def test_dead_component_is_left_unchanged():
    # S_jj = 0 (an all-zero W column) or V_jj = 0 (an all-zero H row): that block
    # is skipped for the sweep and no NaN appears.
    rng = np.random.default_rng(14)
    B = rng.standard_normal((4, 15))
    Wt = rng.standard_normal((4, 3))
    W = rng.random((20, 3))
    W[:, 1] = 0.0
    H = rng.random((3, 15))
    H1 = H.copy()
    R.rhals_h_half(B, Wt, W, H1, gram_mode=0)
    assert np.array_equal(H1[1], H[1])
    Q = R.qr_q(rng.standard_normal((20, 4)))
    H2 = rng.random((3, 15))
    H2[2] = 0.0
    Wt2, W2 = Wt.copy(), W.copy()
    R.rhals_w_half(B, Q, Wt2, W2, H2)
    assert np.array_equal(W2[:, 2], W[:, 2]) and np.array_equal(Wt2[:, 2], Wt[:, 2])
    A = rng.random((20, 15))
    W3, H3, _ = R.hals_sweeps(A, W, H, 3)
    assert np.all(np.isfinite(W3)) and np.all(np.isfinite(H3))
