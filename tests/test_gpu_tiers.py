"""Element-wise sweep parity where the W-half kernel uses every storage tier of Q.

The W half (Section 3.2 W~ rule and reprojection) keeps each block's rows of Q
on chip: 192 rows in registers, the next 512 in tensor memory, the next in
shared memory, the rest read from L2.  With one block per SM (152) those tiers
are all in use only for m above about 152 x 1071 rows, so this test runs
m = 170000 (1119 rows per block: 192 + 512 + 367 + 48), n = 1200, k = 100,
p = 20 - the benchmark's k and l - for one sweep from the same float32 Q and
B as the float64 oracle (every column of the W half reads every row of Q), and
compares W and H entry by entry.  Tolerance 1e-4 relative (max-norm), as the
one-sweep test at 100000 x 50000: every entry of W is a 120-long dot product
with cancellation and W~ = Q^T W sums m terms; the rows of each tier are held
to it separately, so a tier that mishandled its rows could not hide behind
the others.
"""
import numpy as np
import pytest

import synth
from oracle import philox
from oracle import rhals as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_three_sweeps_every_q_tier():
    import paper_1711_02037_gb300 as pkg
    w = synth.Workload("tiers", 170000, 1200, 100, 100, 20, 1, 1, 0.02, w0_exp=True, h0_zero_frac=0.3)
    A = synth.lowrank(w)
    Q, B = R.rqb(A, philox.omega(w.n, w.l, 0), w.q)
    del A
    Q32, B32 = Q.astype(np.float32), B.astype(np.float32)
    W0, H0 = philox.init_factors(w.m, w.n, w.k, 0)
    Wo, Ho, _, _ = R.rhals_sweeps(Q32.astype(np.float64), B32.astype(np.float64), W0, H0, w.iters)
    ctx = pkg.Context(0)
    W = torch.from_numpy(W0.astype(np.float32)).cuda()
    H = torch.from_numpy(H0.astype(np.float32)).cuda()
    ctx.sweeps(torch.from_numpy(Q32).cuda(), torch.from_numpy(np.ascontiguousarray(B32.T)).cuda(), W, H, w.iters)
    torch.cuda.synchronize()
    Wg, Hg = W.double().cpu().numpy(), H.double().cpu().numpy()
    ctx.close()
    assert np.all(Wg >= 0) and np.all(Hg >= 0)
    scale = np.max(np.abs(Wo))
    # row i of a block's 1119 rows: registers [0, 192), tensor memory [192, 704),
    # shared memory [704, 1071), L2 [1071, 1119)
    i = np.arange(w.m) % 1119
    for lo, hi in ((0, 192), (192, 704), (704, 1071), (1071, 1119)):
        rows = (i >= lo) & (i < hi)
        assert np.max(np.abs(Wg[rows] - Wo[rows])) / scale < 1e-4, (lo, hi)
    assert np.max(np.abs(Hg - Ho)) / np.max(np.abs(Ho)) < 1e-4


def test_twenty_sweeps_entrywise_trajectory():
    # 40000 rows: 264 rows of Q per block, in registers and tensor memory; 20 sweeps
    # of the benchmark's k = 100, l = 120 from the same float32 Q and B as the oracle.
    # The trajectory amplifies float32 rounding (about 1e-6 relative per sweep at this
    # rank), so the bound after 20 sweeps is 1e-3 of the largest entry.
    import paper_1711_02037_gb300 as pkg
    w = synth.Workload("traj", 40000, 2000, 100, 100, 20, 1, 20, 0.02, w0_exp=True, h0_zero_frac=0.3)
    A = synth.lowrank(w)
    Q, B = R.rqb(A, philox.omega(w.n, w.l, 0), w.q)
    Q32, B32 = Q.astype(np.float32), B.astype(np.float32)
    W0, H0 = philox.init_factors(w.m, w.n, w.k, 0)
    Wo, Ho, _, ho = R.rhals_sweeps(Q32.astype(np.float64), B32.astype(np.float64), W0, H0, w.iters,
                                   A=A.astype(np.float64))
    ctx = pkg.Context(0)
    W = torch.from_numpy(W0.astype(np.float32)).cuda()
    H = torch.from_numpy(H0.astype(np.float32)).cuda()
    _, _, st = ctx.sweeps(torch.from_numpy(Q32).cuda(), torch.from_numpy(np.ascontiguousarray(B32.T)).cuda(), W, H,
                          w.iters, A=torch.from_numpy(A).cuda(), track_every=1)
    torch.cuda.synchronize()
    Wg, Hg = W.double().cpu().numpy(), H.double().cpu().numpy()
    ctx.close()
    dw = np.max(np.abs(Wg - Wo)) / np.max(np.abs(Wo))
    dh = np.max(np.abs(Hg - Ho)) / np.max(np.abs(Ho))
    dhist = np.max(np.abs(np.array(st.rel_err_hist) - ho) / ho)
    print(f"20 sweeps, entry-wise: W {dw:.2e}, H {dh:.2e}; per-sweep relative error {dhist:.2e}")
    assert dw < 1e-3 and dh < 1e-3
    assert dhist < 1e-5
