"""Edge cases of the in-memory path against the float64 oracle.

* the widest sketch the library takes (l = 128) through a full solve;
* l equal to n (the widest sketch a matrix allows);
* no sweeps: the returned factors are the initial draws, bit for bit;
* padding columns of A (lda > n) holding NaN are never read: the result is
  bit-identical to the unpadded call, in the FP32 and the BF16 forms;
* empty and oversized shapes are rejected through the C ABI without writing
  the outputs.
Tolerance for the solves: final relative error within 1e-3 of the oracle's.
"""
import ctypes

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


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


@pytest.mark.parametrize("m,n,k,p,q,iters", [(3000, 2000, 100, 28, 1, 30), (300, 40, 30, 10, 2, 40)])
def test_widest_sketches_match_oracle(ctx, m, n, k, p, q, iters):
    w = synth.Workload("edge", m, n, min(k, 40), k, p, q, iters, 0.01)
    A = synth.lowrank(w)
    W, H, st = ctx.rnmf(dev(A), k, p, q, iters, seed=0, track_every=iters)
    res = R.rhals(A, k, p, q, iters, 0)
    ref = R.rel_err(A.astype(np.float64), res["W"], res["H"])
    assert abs(st.final_rel_err - ref) <= 1e-3 * ref, (st.final_rel_err, ref)
    assert np.all(host(W) >= 0) and np.all(host(H) >= 0)


def test_zero_sweeps_return_the_initial_draws(ctx):
    m, n, k = 500, 300, 7
    A = synth.lowrank(synth.Workload("z", m, n, k, k, 5, 1, 0, 0.01))
    W, H, st = ctx.rnmf(dev(A), k, 5, 1, 0, seed=3)
    W0, H0 = philox.init_factors(m, n, k, 3)
    assert np.array_equal(W.cpu().numpy(), W0.astype(np.float32))
    assert np.array_equal(H.cpu().numpy(), H0.astype(np.float32))
    assert st.sweeps_done == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_padding_columns_are_never_read(ctx, precision):
    m, n, k = 2000, 1000, 12
    A = synth.lowrank(synth.Workload("pad", m, n, k, k, 8, 2, 20, 0.01))
    padded = np.full((m, n + 8), np.nan, np.float32)
    padded[:, :n] = A
    Ap = torch.from_numpy(padded).cuda()[:, :n]
    W1, H1, _ = ctx.rnmf(dev(A), k, 8, 2, 20, seed=0, precision=precision)
    W2, H2, _ = ctx.rnmf(Ap, k, 8, 2, 20, seed=0, precision=precision)
    torch.cuda.synchronize()
    assert torch.isfinite(W2).all() and torch.isfinite(H2).all()
    assert torch.equal(W1, W2) and torch.equal(H1, H2)


def test_empty_and_oversized_shapes_rejected(ctx):
    import paper_1711_02037_gb300 as pkg
    lib = pkg.lib()
    A = torch.ones(64, 64, device="cuda")
    W = torch.full((64, 8), -3.0, device="cuda")
    H = torch.full((8, 64), -3.0, device="cuda")
    o = pkg.default_opts()
    s = pkg.Stats()
    for m, n, lda, k, p in [(0, 64, 64, 8, 2), (64, 0, 64, 8, 2), (64, 64, 32, 8, 2), (64, 64, 64, 8, 121),
                            (64, 64, 64, 8, 60)]:
        st = lib.rnmf(ctx.h, A.data_ptr(), m, n, lda, k, p, 1, 3, 0, ctypes.byref(o), W.data_ptr(), H.data_ptr(),
                      ctypes.byref(s))
        assert st == 1, (m, n, lda, k, p)
    torch.cuda.synchronize()
    assert torch.all(W == -3.0) and torch.all(H == -3.0)


# Tall Q: with one block per SM (152 on this GPU) a block owns ceil(m / 152) rows
# of Q; the W half keeps 192 of them in registers, up to 512 in tensor memory,
# then fills shared memory and reads the rest from L2.  These sizes reach every
# class: (40000: registers + a partly filled tensor-memory slot set),
# (120000, l = 20: registers + tensor memory + shared memory), (200000, l = 128:
# all four, with full-width rows).  Tolerance (max-norm relative): 2e-5 as for
# the small sweeps, and 1e-4 at m = 200000, where every entry of W is a 128-long
# dot product Q_r u with cancellation and W~ = Q^T W sums 200000 terms - a plain
# float32 evaluation of the same sweep differs from float64 by 1.7e-5 there.
@pytest.mark.parametrize("m,n,r,k,p,tol", [(40000, 300, 20, 30, 10, 2e-5), (120000, 400, 10, 10, 10, 2e-5),
                                           (200000, 1000, 40, 40, 88, 1e-4)])
def test_single_sweep_tall_q(ctx, m, n, r, k, p, tol):
    w = synth.Workload("tall", m, n, r, k, p, 1, 0, 0.01)
    A = synth.lowrank(w)
    Q, B = R.rqb(A.astype(np.float64), philox.omega(n, k + p, 0), 1)
    Q32, B32 = Q.astype(np.float32), B.astype(np.float32)
    W0, H0 = philox.init_factors(m, n, k, 0)
    Wo, Ho, _, _ = R.rhals_sweeps(Q32.astype(np.float64), B32.astype(np.float64), W0, H0, 1)
    W, H = dev(W0), dev(H0)
    ctx.sweeps(dev(Q32), dev(B32.T), W, H, 1)
    Wg, Hg = host(W), host(H)
    assert np.all(Wg >= 0) and np.all(Hg >= 0)
    assert np.max(np.abs(Wg - Wo)) / np.max(np.abs(Wo)) < tol
    assert np.max(np.abs(Hg - Ho)) / np.max(np.abs(Ho)) < tol


# The host-buffer entry copies A in (pinned memory: the GPU's own loads,
# 16-byte pieces when rows are aligned, else words; pageable memory: the copy
# engine), runs the device path and copies W, H out: its factors equal the
# device entry's bit for bit, for padded and unpadded rows.
@pytest.mark.parametrize("pinned,pad", [(True, 0), (True, 3), (False, 0), (False, 3)])
def test_host_entry_equals_device_entry(ctx, pinned, pad):
    m, n, k = 3000, 1000, 12
    A = synth.lowrank(synth.Workload("host", m, n, k, k, 8, 1, 20, 0.01))
    buf = torch.zeros((m, n + pad), dtype=torch.float32)
    if pinned:
        buf = buf.pin_memory()
    buf[:, :n] = torch.from_numpy(A)
    A_host = buf[:, :n]
    Wh, Hh, _ = ctx.rnmf_host(A_host, k, 8, 1, 20, seed=0)
    Wd, Hd, _ = ctx.rnmf(dev(A), k, 8, 1, 20, seed=0)
    assert np.array_equal(Wh, Wd.cpu().numpy()) and np.array_equal(Hh, Hd.cpu().numpy())
