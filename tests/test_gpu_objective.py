"""GPU compressed objective f~(W~, H) = ||B - W~ H||_F^2 (Section 3.2) per sweep.

The library reports f~ after each sweep and after each sweep's H half
(rnmf_stats.obj_hist / obj_half_hist).  Checks:
  * parity with the FP64 oracle's f~ along its own trajectory, sweep by sweep:
    within 1e-5 relative when both start from the same float32 Q and B (the
    sweeps and the objective alone), and within 1e-4 relative through the whole
    of Algorithm 1 on the 1000 x 500, k = 10 workload, where the GPU's float32
    range finder moves range(Q) by ~1e-6 and f~ = ||P_Q (A - W H)||^2 feels that
    amplified by ||A - W H|| / ||P_Q (A - W H)||;
  * the H half is exact block coordinate descent on f~ when S = W~^T W~
    (gram_mode 1), so f~ never rises over an H half (Section 3.2);
  * after a sweep W~ = Q^T W, so f~ <= ||A - W H||^2, with equality when Q is
    square (l = m): the compressed problem is then the full one.
"""
import math

import numpy as np
import pytest

import synth
from oracle import philox
from oracle import rhals as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1711_02037_gb300 as pkg
    c = pkg.Context(0)
    yield c
    c.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def oracle_objectives(Q, B, W0, H0, iters, gram_mode=0):
    """f~ after each H half and after each sweep along the oracle's trajectory."""
    W = np.array(W0, np.float64, copy=True)
    H = np.array(H0, np.float64, copy=True)
    Wt = Q.T @ W
    half, end = [], []
    for _ in range(iters):
        R.rhals_h_half(B, Wt, W, H, gram_mode)
        half.append(R.compressed_objective(B, Wt, H))
        R.rhals_w_half(B, Q, Wt, W, H)
        end.append(R.compressed_objective(B, Wt, H))
    return np.array(half), np.array(end)


@pytest.mark.parametrize("gram_mode", [0, 1])
def test_objective_per_sweep_from_same_qb(ctx, gram_mode):
    w = synth.SMALL
    A = synth.lowrank(w)
    Q, B = R.rqb(A, philox.omega(w.n, w.l, w.seed), w.q)
    Q32, B32 = Q.astype(np.float32), B.astype(np.float32)
    W0, H0 = philox.init_factors(w.m, w.n, w.k, w.seed)
    half, end = oracle_objectives(Q32.astype(np.float64), B32.astype(np.float64), W0, H0, w.iters, gram_mode)
    _, _, st = ctx.sweeps(dev(Q32), dev(B32.T), dev(W0), dev(H0), w.iters, gram_mode=gram_mode, track_obj=True)
    g_end, g_half = np.array(st.obj_hist), np.array(st.obj_half_hist)
    assert g_end.shape == (w.iters,) and g_half.shape == (w.iters,)
    assert np.max(np.abs(g_end - end) / end) < 1e-5
    assert np.max(np.abs(g_half - half) / half) < 1e-5


def test_objective_per_sweep_through_algorithm_1(ctx):
    w = synth.SMALL
    A = synth.lowrank(w)
    ref = R.rhals(A, w.k, w.p, w.q, 0, w.seed)
    half, end = oracle_objectives(ref["Q"], ref["B"], ref["W_init"], ref["H_init"], w.iters)
    _, _, st = ctx.rnmf(dev(A), w.k, w.p, w.q, w.iters, w.seed, track_obj=True)
    g_end, g_half = np.array(st.obj_hist), np.array(st.obj_half_hist)
    assert np.max(np.abs(g_end - end) / end) < 1e-4
    assert np.max(np.abs(g_half - half) / half) < 1e-4


def test_h_half_descends_compressed_objective(ctx):
    # gram_mode 1: the H rows are exact minimisers of f~ one at a time
    w = synth.Workload("t", 3000, 1200, 12, 12, 8, 1, 60, 0.05)
    A = synth.lowrank(w)
    _, _, st = ctx.rnmf(dev(A), w.k, w.p, w.q, w.iters, 7, gram_mode=1, track_obj=True)
    end, half = np.array(st.obj_hist), np.array(st.obj_half_hist)
    assert np.all(np.isfinite(end)) and np.all(np.isfinite(half))
    assert np.all(half[1:] <= end[:-1] * (1 + 1e-6)), np.max(half[1:] / end[:-1])
    assert end[-1] < half[0]


def test_objective_bounded_by_true_objective(ctx):
    w = synth.Workload("t", 2000, 900, 10, 10, 6, 2, 30, 0.02)
    A = synth.lowrank(w)
    _, _, st = ctx.rnmf(dev(A), w.k, w.p, w.q, w.iters, 1, track_every=1, track_obj=True)
    a2 = float(np.sum(A.astype(np.float64) ** 2))
    true = np.array(st.rel_err_hist) ** 2 * a2
    obj = np.array(st.obj_hist)
    assert np.all(obj <= true * (1 + 1e-5))
    assert np.all(obj >= 0.5 * true)  # most of the residual lies in range(Q) on this data


def test_square_q_objective_is_the_true_objective(ctx):
    m, n, k = 24, 40, 4
    w = synth.Workload("t", m, n, 4, k, m - k, 1, 0, 0.01)
    A = synth.lowrank(w)
    _, _, st = ctx.rnmf(dev(A), k, m - k, 1, 20, 0, track_every=1, track_obj=True)
    a2 = float(np.sum(A.astype(np.float64) ** 2))
    true = np.array(st.rel_err_hist) ** 2 * a2
    assert np.max(np.abs(np.array(st.obj_hist) - true) / true) < 1e-4


def test_interleaved_order_has_no_half_objective(ctx):
    import paper_1711_02037_gb300 as pkg
    w = synth.Workload("t", 800, 500, 6, 6, 6, 1, 12, 0.02)
    A = synth.lowrank(w)
    _, _, st = ctx.rnmf(dev(A), w.k, w.p, w.q, w.iters, 0, track_every=1, track_obj=True,
                        order=pkg.ORDER_INTERLEAVED)
    assert all(math.isnan(x) for x in st.obj_half_hist)
    a2 = float(np.sum(A.astype(np.float64) ** 2))
    true = np.array(st.rel_err_hist) ** 2 * a2
    assert np.all(np.array(st.obj_hist) <= true * (1 + 1e-5))
