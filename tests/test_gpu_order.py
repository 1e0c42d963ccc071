"""The shuffled and interleaved update orders (Section 3.2) on the GPU against the
float64 oracle.

* one and three sweeps from identical float32 inputs: W, H within 2e-5
  relative (max-norm) of oracle.rhals.rhals_sweeps(..., order=1) - a
  different visiting order moves them far more, so this also checks that both
  sides draw the same permutations;
* a whole solve: per-sweep relative error within 1e-5 relative of the
  oracle's shuffled run, the final error within 1e-3;
* the order seed changes the result; a tall Q (the W half's tensor-memory
  rows) gives the same agreement;
* entries that run only the cyclic order reject it;
* interleaved order (W_1 -> H_1 -> ... -> W_k -> H_k): the same bounds for one
  and three sweeps (gram_mode 0 and 1, a tall Q) and for a whole solve; shapes
  whose rows are not multiples of 16 bytes (l, m or n not multiples of 4: the
  passes' per-thread copies instead of TMA boxes, ragged last tiles); a dead
  component (a zero row of H, so V_jj = 0: its W column is left unchanged).
"""
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


def f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


@pytest.mark.parametrize("m,n,k,p,sweeps", [(1000, 500, 10, 10, 1), (1000, 500, 10, 10, 3), (120000, 400, 16, 8, 1)])
def test_shuffled_sweeps_match_oracle(ctx, m, n, k, p, sweeps):
    w = synth.Workload("ord", m, n, k, k, p, 2, 0, 0.01)
    A = synth.lowrank(w).astype(np.float64)
    Q, B = R.rqb(A, philox.omega(n, k + p, 0), 2)
    Q, B = f32(Q), f32(B)
    W0, H0 = philox.init_factors(m, n, k, 0)
    Wo, Ho, _, _ = R.rhals_sweeps(Q, B, W0, H0, sweeps, order=1, order_seed=7)
    W, H = dev(W0), dev(H0)
    ctx.sweeps(dev(Q), dev(B.T), W, H, sweeps, order=1, order_seed=7)
    Wg, Hg = host(W), host(H)
    assert np.max(np.abs(Wg - Wo)) / np.max(np.abs(Wo)) < 2e-5
    assert np.max(np.abs(Hg - Ho)) / np.max(np.abs(Ho)) < 2e-5
    Wc, Hc, _, _ = R.rhals_sweeps(Q, B, W0, H0, sweeps)
    assert np.max(np.abs(Hc - Ho)) / np.max(np.abs(Ho)) > 1e-4  # the order matters at this size


def test_shuffled_solve_matches_oracle(ctx):
    w = synth.SMALL
    A = synth.lowrank(w)
    _, _, st = ctx.rnmf(dev(A), w.k, w.p, w.q, w.iters, w.seed, track_every=1, order=1, order_seed=3)
    ref = R.rhals(A, w.k, w.p, w.q, w.iters, w.seed, track=True, order=1, order_seed=3)
    got = np.array(st.rel_err_hist)
    rel = np.abs(got - ref["hist"]) / ref["hist"]
    assert rel.max() < 1e-5, rel.max()
    assert abs(st.final_rel_err - ref["hist"][-1]) <= 1e-3 * ref["hist"][-1]


def test_order_seed_changes_the_result(ctx):
    w = synth.SMALL
    A = dev(synth.lowrank(w))
    W1, H1, _ = ctx.rnmf(A, w.k, w.p, w.q, 5, w.seed, order=1, order_seed=1)
    W2, H2, _ = ctx.rnmf(A, w.k, w.p, w.q, 5, w.seed, order=1, order_seed=2)
    W3, H3, _ = ctx.rnmf(A, w.k, w.p, w.q, 5, w.seed, order=1, order_seed=1)
    torch.cuda.synchronize()
    assert not torch.equal(H1, H2)
    assert torch.equal(W1, W3) and torch.equal(H1, H3)


def test_cyclic_only_entries_reject_shuffled(ctx):
    import paper_1711_02037_gb300 as pkg
    w = synth.SMALL
    A = dev(synth.lowrank(w))
    for order in (1, 2):
        with pytest.raises(pkg.RnmfError):
            ctx.hals(A, w.k, 2, order=order)
    with pytest.raises(pkg.RnmfError):
        ctx.rnmf(A, w.k, w.p, w.q, 2, order=3)  # no such order


@pytest.mark.parametrize("m,n,k,p,sweeps,gram_mode", [(1000, 500, 10, 10, 1, 0), (1000, 500, 10, 10, 3, 0),
                                                      (1000, 500, 10, 10, 3, 1), (120000, 400, 16, 8, 1, 0)])
def test_interleaved_sweeps_match_oracle(ctx, m, n, k, p, sweeps, gram_mode):
    w = synth.Workload("il", m, n, k, k, p, 2, 0, 0.01)
    A = synth.lowrank(w).astype(np.float64)
    Q, B = R.rqb(A, philox.omega(n, k + p, 0), 2)
    Q, B = f32(Q), f32(B)
    W0, H0 = philox.init_factors(m, n, k, 0)
    Wo, Ho, _, _ = R.rhals_sweeps(Q, B, W0, H0, sweeps, gram_mode, order=2)
    W, H = dev(W0), dev(H0)
    ctx.sweeps(dev(Q), dev(B.T), W, H, sweeps, gram_mode=gram_mode, order=2)
    Wg, Hg = host(W), host(H)
    assert np.max(np.abs(Wg - Wo)) / np.max(np.abs(Wo)) < 2e-5
    assert np.max(np.abs(Hg - Ho)) / np.max(np.abs(Ho)) < 2e-5


def test_interleaved_solve_matches_oracle(ctx):
    w = synth.SMALL
    A = synth.lowrank(w)
    _, _, st = ctx.rnmf(dev(A), w.k, w.p, w.q, w.iters, w.seed, track_every=1, order=2)
    ref = R.rhals(A, w.k, w.p, w.q, w.iters, w.seed, track=True, order=2)
    rel = np.abs(np.array(st.rel_err_hist) - ref["hist"]) / ref["hist"]
    assert rel.max() < 1e-5, rel.max()


@pytest.mark.parametrize("m,n,k,p,sweeps,gram_mode", [(1001, 503, 7, 6, 1, 0), (1001, 503, 7, 6, 3, 1),
                                                      (777, 1234, 9, 3, 2, 0)])
def test_interleaved_unaligned_shapes(ctx, m, n, k, p, sweeps, gram_mode):
    w = synth.Workload("ilu", m, n, k, k, p, 2, 0, 0.01)
    A = synth.lowrank(w).astype(np.float64)
    Q, B = R.rqb(A, philox.omega(n, k + p, 1), 2)
    Q, B = f32(Q), f32(B)
    W0, H0 = philox.init_factors(m, n, k, 1)
    Wo, Ho, _, _ = R.rhals_sweeps(Q, B, W0, H0, sweeps, gram_mode, order=2)
    W, H = dev(W0), dev(H0)
    ctx.sweeps(dev(Q), dev(B.T), W, H, sweeps, gram_mode=gram_mode, order=2)
    Wg, Hg = host(W), host(H)
    assert np.max(np.abs(Wg - Wo)) / np.max(np.abs(Wo)) < 2e-5
    assert np.max(np.abs(Hg - Ho)) / np.max(np.abs(Ho)) < 2e-5


def test_interleaved_dead_component(ctx):
    m, n, k, p = 1000, 500, 6, 6
    w = synth.Workload("ild", m, n, k, k, p, 2, 0, 0.01)
    A = synth.lowrank(w).astype(np.float64)
    Q, B = R.rqb(A, philox.omega(n, k + p, 2), 2)
    Q, B = f32(Q), f32(B)
    W0, H0 = philox.init_factors(m, n, k, 2)
    H0 = H0.copy()
    H0[2] = 0.0  # V_22 = 0 in the first sweep: W_2 and W~_2 stay as they are
    Wo, Ho, _, _ = R.rhals_sweeps(Q, B, W0, H0, 1, order=2)
    assert np.array_equal(Wo[:, 2], W0[:, 2])
    W, H = dev(W0), dev(H0)
    ctx.sweeps(dev(Q), dev(B.T), W, H, 1, order=2)
    Wg, Hg = host(W), host(H)
    assert np.array_equal(Wg[:, 2], f32(W0[:, 2]))
    assert np.max(np.abs(Wg - Wo)) / np.max(np.abs(Wo)) < 2e-5
    assert np.max(np.abs(Hg - Ho)) / np.max(np.abs(Ho)) < 2e-5

