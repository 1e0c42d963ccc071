"""SVD-based initial factors (NNDSVD of the randomized SVD) against the float64 oracle.

* zero sweeps: the GPU's factors equal oracle.init_svd.svd_init applied to the
  GPU's own Q and B (so only the eigensolver and the float32 products differ)
  within 2e-5 relative (max-norm), and are nonnegative;
* the factors do not depend on the QB basis: against the oracle's own
  Householder QB within 1e-3 (float32 QB against float64);
* a whole solve from them: per-sweep relative error within 1e-5 relative of the
  oracle's run from its SVD-based factors;
* entries that start only from uniform factors reject the option.
"""
import numpy as np
import pytest

import synth
from oracle import init_svd as I
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


@pytest.mark.parametrize("m,n,k,p", [(1000, 500, 10, 10), (3000, 1200, 31, 9), (600, 400, 1, 5)])
def test_initial_factors_match_oracle(ctx, m, n, k, p):
    w = synth.Workload("svd", m, n, k, k, p, 2, 0, 0.01)
    A = synth.lowrank(w)
    W, H, _ = ctx.rnmf(dev(A), k, p, 2, 0, seed=0, init=1)
    Q, Bt = ctx.qb(dev(A), k + p, 2, seed=0)
    Wo, Ho = I.svd_init(host(Q), host(Bt).T, k)
    Wg, Hg = host(W), host(H)
    assert Wg.min() >= 0 and Hg.min() >= 0
    assert np.max(np.abs(Wg - Wo)) / np.max(np.abs(Wo)) < 2e-5
    assert np.max(np.abs(Hg - Ho)) / np.max(np.abs(Ho)) < 2e-5
    ref = R.rhals(A, k, p, 2, 0, 0, init=1)
    assert np.max(np.abs(Wg - ref["W"])) / np.max(np.abs(ref["W"])) < 1e-3
    assert np.max(np.abs(Hg - ref["H"])) / np.max(np.abs(ref["H"])) < 1e-3


def test_solve_from_svd_factors_matches_oracle(ctx):
    w = synth.SMALL
    A = synth.lowrank(w)
    _, _, st = ctx.rnmf(dev(A), w.k, w.p, w.q, w.iters, w.seed, track_every=1, init=1)
    ref = R.rhals(A, w.k, w.p, w.q, w.iters, w.seed, track=True, init=1)
    rel = np.abs(np.array(st.rel_err_hist) - ref["hist"]) / ref["hist"]
    assert rel.max() < 1e-5, rel.max()


def test_uniform_only_entries_reject_svd_init(ctx):
    import paper_1711_02037_gb300 as pkg
    w = synth.SMALL
    A = dev(synth.lowrank(w))
    with pytest.raises(pkg.RnmfError):
        ctx.hals(A, w.k, 2, init=1)
    with pytest.raises(pkg.RnmfError):
        ctx.rnmf(A, w.k, w.p, w.q, 2, init=2)  # no such initialisation
