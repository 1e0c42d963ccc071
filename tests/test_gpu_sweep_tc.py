"""The H half's products on tensor cores (sweep_products = SWEEP_SPLIT3).

R = B^T W~, T = B H^T, V = H H^T and S = W^T W (Algorithm 1's loop body,
Section 3.2 H rule) run as 3-term split BF16 products on tcgen05: every float32 operand x is
split into hi = bf16(x) and lo = bf16(x - hi), and a product a b is taken as
hi_a hi_b + hi_a lo_b + lo_a hi_b.  Each split drops at most 2^-18 |x| and the
dropped lo_a lo_b is at most 2^-18 |a b|, so each product is off by about
3 x 2^-18 = 1.1e-5 of |a b| before the float32 accumulation.  An entry of R, T
or V is therefore within about 1.2e-5 of the sum of |terms| it adds, against
float32's 6e-8 per term; the tests bound the sweeps' outputs accordingly,
against the float64 oracle from the same float32 Q and B:
  - one sweep, entry by entry: 1e-3 of the largest entry (the 1e-4 bound of the
    float32 products, widened by the products' 1.2e-5 against float32's 6e-8
    per term, and cancellation in R's and T's sums of mixed-sign terms);
  - 20 sweeps: the relative error ||A - W H|| / ||A|| of every sweep within
    1e-4 of the oracle's (float32 products: 1e-5);
  - shapes the tensor-core path does not take (m, n not multiples of 4) run the
    float32 products: bit-identical to sweep_products = SWEEP_FP32;
  - fixed-order sums: two runs are bit-identical.
"""
import numpy as np
import pytest

import synth
from oracle import philox
from oracle import rhals as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(m, n, k, p, q=1, seed=0):
    w = synth.Workload("sweep_tc", m, n, k, k, p, q, 1, 0.02, w0_exp=True, h0_zero_frac=0.3)
    A = synth.lowrank(w)
    Q, B = R.rqb(A, philox.omega(w.n, w.l, seed), w.q)
    Q32, B32 = Q.astype(np.float32), B.astype(np.float32)
    W0, H0 = philox.init_factors(w.m, w.n, w.k, seed)
    return w, A, Q32, B32, W0, H0


def _gpu_sweeps(ctx, Q32, B32, W0, H0, iters, A=None, **kw):
    W = torch.from_numpy(W0.astype(np.float32)).cuda()
    H = torch.from_numpy(H0.astype(np.float32)).cuda()
    Qd = torch.from_numpy(Q32).cuda()
    Btd = torch.from_numpy(np.ascontiguousarray(B32.T)).cuda()
    Ad = torch.from_numpy(A).cuda() if A is not None else None
    _, _, st = ctx.sweeps(Qd, Btd, W, H, iters, A=Ad, track_every=1 if A is not None else 0, **kw)
    torch.cuda.synchronize()
    return W.double().cpu().numpy(), H.double().cpu().numpy(), st


def test_one_sweep_entrywise():
    import paper_1711_02037_gb300 as pkg
    w, A, Q32, B32, W0, H0 = _setup(20000, 10000, 100, 20)
    Wo, Ho, _, _ = R.rhals_sweeps(Q32.astype(np.float64), B32.astype(np.float64), W0, H0, 1)
    ctx = pkg.Context(0)
    Wg, Hg, _ = _gpu_sweeps(ctx, Q32, B32, W0, H0, 1, sweep_products=pkg.SWEEP_SPLIT3)
    Wf, Hf, _ = _gpu_sweeps(ctx, Q32, B32, W0, H0, 1, sweep_products=pkg.SWEEP_FP32)
    ctx.close()
    assert np.all(Wg >= 0) and np.all(Hg >= 0)
    dw = np.max(np.abs(Wg - Wo)) / np.max(np.abs(Wo))
    dh = np.max(np.abs(Hg - Ho)) / np.max(np.abs(Ho))
    dwf = np.max(np.abs(Wf - Wo)) / np.max(np.abs(Wo))
    dhf = np.max(np.abs(Hf - Ho)) / np.max(np.abs(Ho))
    print(f"one sweep: tensor-core products W {dw:.2e}, H {dh:.2e}; float32 products W {dwf:.2e}, H {dhf:.2e}")
    assert dw < 1e-3 and dh < 1e-3
    # the tensor-core products really ran (float32 products land far closer)
    assert dh > 0.0


def test_twenty_sweeps_trajectory():
    import paper_1711_02037_gb300 as pkg
    w, A, Q32, B32, W0, H0 = _setup(20000, 10000, 100, 20)
    Wo, Ho, _, ho = R.rhals_sweeps(Q32.astype(np.float64), B32.astype(np.float64), W0, H0, 20,
                                   A=A.astype(np.float64))
    ctx = pkg.Context(0)
    Wg, Hg, st = _gpu_sweeps(ctx, Q32, B32, W0, H0, 20, A=A, sweep_products=pkg.SWEEP_SPLIT3)
    ctx.close()
    dhist = np.abs(np.array(st.rel_err_hist) - ho) / ho
    dw = np.max(np.abs(Wg - Wo)) / np.max(np.abs(Wo))
    dh = np.max(np.abs(Hg - Ho)) / np.max(np.abs(Ho))
    print(f"20 sweeps: per-sweep relative error max {dhist.max():.2e}; W {dw:.2e}, H {dh:.2e}")
    assert len(st.rel_err_hist) == 20
    assert dhist.max() < 1e-4


def test_untaken_shape_is_the_float32_path():
    import paper_1711_02037_gb300 as pkg
    # neither n (the H half's products) nor m (S = W^T W) a multiple of 4
    w, A, Q32, B32, W0, H0 = _setup(3001, 1002, 16, 8)
    ctx = pkg.Context(0)
    Wa, Ha, _ = _gpu_sweeps(ctx, Q32, B32, W0, H0, 3, sweep_products=pkg.SWEEP_SPLIT3)
    Wb, Hb, _ = _gpu_sweeps(ctx, Q32, B32, W0, H0, 3, sweep_products=pkg.SWEEP_FP32)
    ctx.close()
    assert np.array_equal(Wa, Wb) and np.array_equal(Ha, Hb)


def test_deterministic_and_ragged():
    import paper_1711_02037_gb300 as pkg
    # n = 4 x 1733 and m = 4 x 1251 (ragged last 64-column steps of H and W^T), k = 37,
    # l = 48 (k and l off the 16 grid)
    w, A, Q32, B32, W0, H0 = _setup(5004, 6932, 37, 11)
    Wo, Ho, _, _ = R.rhals_sweeps(Q32.astype(np.float64), B32.astype(np.float64), W0, H0, 2)
    ctx = pkg.Context(0)
    Wa, Ha, _ = _gpu_sweeps(ctx, Q32, B32, W0, H0, 2, sweep_products=pkg.SWEEP_SPLIT3)
    Wb, Hb, _ = _gpu_sweeps(ctx, Q32, B32, W0, H0, 2, sweep_products=pkg.SWEEP_SPLIT3)
    ctx.close()
    assert np.array_equal(Wa, Wb) and np.array_equal(Ha, Hb)
    dw = np.max(np.abs(Wa - Wo)) / np.max(np.abs(Wo))
    dh = np.max(np.abs(Ha - Ho)) / np.max(np.abs(Ho))
    print(f"ragged, two sweeps: W {dw:.2e}, H {dh:.2e}")
    assert dw < 1e-3 and dh < 1e-3


def test_rnmf_bf16_form_with_tensor_core_sweeps():
    import paper_1711_02037_gb300 as pkg
    w = synth.Workload("sweep_tc_rnmf", 20000, 8000, 40, 40, 20, 2, 100, 0.02, w0_exp=True, h0_zero_frac=0.3)
    A = torch.from_numpy(synth.lowrank(w)).cuda()
    ctx = pkg.Context(0)
    _, _, s32 = ctx.rnmf(A, w.k, w.p, w.q, w.iters, 0, precision=pkg.PREC_BF16, track_every=10)
    _, _, s16 = ctx.rnmf(A, w.k, w.p, w.q, w.iters, 0, precision=pkg.PREC_BF16, track_every=10,
                         sweep_products=pkg.SWEEP_SPLIT3, track_obj=True)
    ctx.close()
    d = np.abs(np.array(s16.rel_err_hist) - np.array(s32.rel_err_hist)) / np.array(s32.rel_err_hist)
    print(f"rnmf BF16 form, 100 sweeps: float32 sweep products {s32.final_rel_err:.6g}, tensor-core "
          f"{s16.final_rel_err:.6g}; largest relative difference every 10 sweeps {d.max():.2e}")
    # the same QB: the two runs differ only by the products' rounding
    assert d.max() < 1e-3
    # the compressed objective (its own float32 residual pass) decreases along the sweeps
    o = np.array(s16.obj_hist)
    assert np.all(np.isfinite(o)) and o[-1] < o[0]


@pytest.mark.parametrize("m,n,k,p", [(300, 8, 1, 3), (2004, 1000, 120, 8), (5000, 64, 8, 8), (1001, 4096, 3, 1)])
def test_edge_shapes_one_sweep(m, n, k, p):
    # k = 1 (16-column accumulators, one valid row), l = 128 (the largest), n of one
    # 64-column contraction step or less, m not a multiple of 4 (S on CUDA cores)
    import paper_1711_02037_gb300 as pkg
    w, A, Q32, B32, W0, H0 = _setup(m, n, k, p)
    Wo, Ho, _, _ = R.rhals_sweeps(Q32.astype(np.float64), B32.astype(np.float64), W0, H0, 1)
    ctx = pkg.Context(0)
    Wg, Hg, _ = _gpu_sweeps(ctx, Q32, B32, W0, H0, 1, sweep_products=pkg.SWEEP_SPLIT3)
    ctx.close()
    assert np.all(Wg >= 0) and np.all(Hg >= 0)
    dw = np.max(np.abs(Wg - Wo)) / max(np.max(np.abs(Wo)), 1e-30)
    dh = np.max(np.abs(Hg - Ho)) / max(np.max(np.abs(Ho)), 1e-30)
    print(f"edge {m}x{n} k={k} l={k + p}: W {dw:.2e}, H {dh:.2e}")
    assert dw < 1e-3 and dh < 1e-3
