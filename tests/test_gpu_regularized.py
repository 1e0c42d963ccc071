"""Regularised HALS on the GPU (Section 3.4 penalties) against oracle/extras.py.

Tolerances as for the plain sweeps: one sweep from identical float32 inputs
(index order and the interleaved order of Section 3.2) within 2e-5 (max-norm
relative, float32 rounding of k- and l-long sums); a full randomized solve on
the small synthetic workload within 3e-5 per sweep of the oracle's relative
error and 1e-3 at the end (100 float32 sweeps of a nonlinear iteration: a
plain numpy float32 evaluation of the same sweeps deviates from float64 by up
to 4.9e-6 on this input, and by a factor 2-3 more or less when Q changes by
one float32 ulp; the GPU's summation orders differ from numpy's);
deterministic regularised HALS within 1e-4 after a few sweeps.  Zero penalties
take the plain rule's code path (bit-identical to a call without penalties).
"""
import numpy as np
import pytest

import synth
from oracle import extras as X
from oracle import philox
from oracle import rhals as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PENS = [dict(alpha_W=0.5), dict(alpha_H=2.0), dict(beta_W=0.05), dict(beta_H=0.3),
        dict(alpha_W=0.3, alpha_H=0.2, beta_W=0.02, beta_H=0.1)]


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


def args(pen):
    return (pen.get("alpha_W", 0.0), pen.get("alpha_H", 0.0), pen.get("beta_W", 0.0), pen.get("beta_H", 0.0))


@pytest.mark.parametrize("order", [0, 2])
@pytest.mark.parametrize("gram_mode", [0, 1])
@pytest.mark.parametrize("pen", PENS)
def test_single_compressed_sweep(ctx, pen, gram_mode, order):
    w = synth.Workload("t", 1000, 500, 10, 10, 10, 2, 0, 0.01)
    A = synth.lowrank(w)
    Q, B = R.rqb(A, philox.omega(500, 20, 0), 2)
    Q32, B32 = Q.astype(np.float32), B.astype(np.float32)
    W0, H0 = philox.init_factors(1000, 500, 10, 0)
    Wo, Ho, _, _ = X.rhals_reg_sweeps(Q32.astype(np.float64), B32.astype(np.float64), W0, H0, 1, *args(pen),
                                      gram_mode=gram_mode, order=order)
    W, H = dev(W0), dev(H0)
    ctx.sweeps(dev(Q32), dev(B32.T), W, H, 1, gram_mode=gram_mode, order=order, **pen)
    Wg, Hg = host(W), host(H)
    assert np.all(Wg >= 0) and np.all(Hg >= 0)
    assert np.max(np.abs(Hg - Ho)) / np.max(np.abs(Ho)) < 2e-5
    assert np.max(np.abs(Wg - Wo)) / np.max(np.abs(Wo)) < 2e-5


@pytest.mark.parametrize("pen", PENS)
def test_randomized_solve(ctx, pen):
    w = synth.SMALL
    A = synth.lowrank(w)
    W, H, st = ctx.rnmf(dev(A), w.k, w.p, w.q, w.iters, w.seed, track_every=1, **pen)
    ref = X.rhals_reg(A, w.k, w.p, w.q, w.iters, w.seed, *args(pen))
    got = np.array(st.rel_err_hist)
    rel = np.abs(got - ref["hist"]) / ref["hist"]
    assert rel.max() < 3e-5, rel.max()
    assert np.all(host(W) >= 0) and np.all(host(H) >= 0)


@pytest.mark.parametrize("pen", PENS)
def test_deterministic_sweeps(ctx, pen):
    w = synth.Workload("d", 300, 200, 6, 6, 0, 0, 4, 0.01)
    A = synth.lowrank(w)
    W, H, _ = ctx.hals(dev(A), w.k, 4, seed=0, **pen)
    W0, H0 = philox.init_factors(300, 200, 6, 0)
    Wo, Ho, _ = X.hals_reg_sweeps(A, W0, H0, 4, *args(pen))
    assert np.max(np.abs(host(H) - Ho)) / np.max(np.abs(Ho)) < 1e-4
    assert np.max(np.abs(host(W) - Wo)) / np.max(np.abs(Wo)) < 1e-4


def test_zero_penalties_are_the_plain_path(ctx):
    w = synth.SMALL
    A = dev(synth.lowrank(w))
    W1, H1, _ = ctx.rnmf(A, w.k, w.p, w.q, 20, w.seed)
    W2, H2, _ = ctx.rnmf(A, w.k, w.p, w.q, 20, w.seed, alpha_W=0.0, beta_H=0.0)
    torch.cuda.synchronize()
    assert torch.equal(W1, W2) and torch.equal(H1, H2)


def test_l1_penalty_sparsifies_h(ctx):
    w = synth.SMALL
    A = dev(synth.lowrank(w))
    _, H0, _ = ctx.rnmf(A, w.k, w.p, w.q, w.iters, w.seed)
    _, H1, _ = ctx.rnmf(A, w.k, w.p, w.q, w.iters, w.seed, beta_H=2.0)
    assert float((H1 == 0).float().mean()) > float((H0 == 0).float().mean())


def test_rejects_negative_penalty(ctx):
    import paper_1711_02037_gb300 as pkg
    A = dev(synth.lowrank(synth.SMALL))
    with pytest.raises(pkg.RnmfError):
        ctx.rnmf(A, 10, 10, 2, 1, 0, alpha_W=-1.0)
