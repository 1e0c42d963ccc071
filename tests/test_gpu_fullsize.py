"""The benchmark's own configuration at full size, against the float64 oracle.

Workload: A = W0 H0 + sigma |z| of 100000 x 50000 (20 GB of float32), k = 100,
p = 20 (l = 120), q = 2, seed 0; the solve runs in the BF16 sketch form, in the
launch configuration the benchmark times (one whalf block per SM, 658 rows of Q
per block across registers and tensor memory).  The oracle cannot run the
whole solve in seconds, so it checks what it can compute one output at a time,
and properties that hold at any size:
  * QB, both forms: Q^T Q = I to 5e-6 (float32 CholeskyQR2); 64 sampled
    columns of B = Q^T A recomputed in float64 from the GPU's Q and the host copy
    of A, every entry within 1e-4 ||A_:c|| (3-term split products, relative
    product error 2^-16) resp. 2e-6 ||A_:c|| (float32 products, compensated sums);
  * one sweep from the initial factors on the GPU's (Q, B): W and H equal to the
    oracle's sweep on the same float32 inputs within 1e-4 relative (max-norm):
    every entry of W is a 120-long dot product Q_r u with cancellation and
    W~ = Q^T W sums 100000 terms; a plain float32 evaluation of one sweep on a
    200000 x 1000, k = 100 input of the same recipe differs from float64 by
    4.9e-5;
  * the whole solve: W, H finite and nonnegative, two runs bit-identical, and
    the BF16 form reaches 1.001 x the FP32 form's error after 300 sweeps within
    3 x 300 sweeps (the benchmark's time-to-target criterion);
  * the whole solve against the float64 oracle's own 300-sweep solve on the
    same input (stored by tests/golden/make_oracle_reference.py, oracle only).
    At rank 100 the sweeps are far from converged after 300 sweeps and the
    trajectory amplifies rounding: the same FP32 QB rotated into another
    orthonormal basis of the same range (identical in exact arithmetic) ends
    0.1-0.3 % away from the unrotated run (bench.py --subspace-report).  So the
    FP32 form's final error is held to 5e-3 relative of the oracle's here (the
    1e-3 of the smaller workloads holds at 1000 x 500 and 50000 x 20000, see
    test_gpu_parity.py and test_gpu_scale.py); the tensor-core forms, whose
    range finders pick other noise directions, are bounded at 10 % and
    reported.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import philox
from oracle import rhals as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W_FULL = synth.PRECISION


@pytest.fixture(scope="module")
def full():
    import paper_1711_02037_gb300 as pkg
    w = W_FULL
    A_host = torch.empty((w.m, w.n), dtype=torch.float32, pin_memory=True)
    synth.lowrank_into(A_host.numpy(), w)
    A = A_host.cuda()
    c = pkg.Context(0)
    yield c, A_host.numpy(), A
    c.close()
    del A
    torch.cuda.empty_cache()


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


@pytest.fixture(scope="module")
def qb_bf16(full):
    c, _, A = full
    w = W_FULL
    return c.qb(A, w.l, w.q, w.seed, precision=1)


@pytest.mark.parametrize("precision,tol", [(0, 2e-6), (1, 1e-4)])
def test_fullsize_qb(full, qb_bf16, precision, tol):
    c, Ah, A = full
    w = W_FULL
    Q, Bt = qb_bf16 if precision == 1 else c.qb(A, w.l, w.q, w.seed, precision=precision)
    Qh = host(Q)
    assert np.max(np.abs(Qh.T @ Qh - np.eye(w.l))) < 5e-6
    cols = np.sort(np.random.default_rng(7).choice(w.n, 64, replace=False))
    Ac = Ah[:, cols].astype(np.float64)  # m x 64
    ref = Qh.T @ Ac                      # l x 64
    got = host(Bt)[cols].T
    scale = np.linalg.norm(Ac, axis=0)[None, :]
    assert np.max(np.abs(got - ref) / scale) < tol


def test_fullsize_one_sweep(full, qb_bf16):
    c, _, _ = full
    w = W_FULL
    Q, Bt = qb_bf16
    Qh, Bh = host(Q), host(Bt).T
    W0, H0 = philox.init_factors(w.m, w.n, w.k, w.seed)
    Wo, Ho, _, _ = R.rhals_sweeps(Qh, Bh, W0, H0, 1)
    W = torch.from_numpy(W0.astype(np.float32)).cuda()
    H = torch.from_numpy(H0.astype(np.float32)).cuda()
    c.sweeps(Q, Bt, W, H, 1)
    Wg, Hg = host(W), host(H)
    assert np.all(Wg >= 0) and np.all(Hg >= 0)
    assert np.max(np.abs(Wg - Wo)) / np.max(np.abs(Wo)) < 1e-4
    assert np.max(np.abs(Hg - Ho)) / np.max(np.abs(Ho)) < 1e-4


def test_fullsize_solve(full):
    c, _, A = full
    w = W_FULL
    every = 10
    _, _, st32 = c.rnmf(A, w.k, w.p, w.q, w.iters, w.seed, precision=0, track_every=every)
    target = 1.001 * st32.rel_err_hist[-1]
    W1, H1, st = c.rnmf(A, w.k, w.p, w.q, 3 * w.iters, w.seed, precision=1, track_every=every)
    hist = np.array(st.rel_err_hist)
    assert np.all(np.isfinite(hist)) and np.min(hist) <= target, (hist[-1], target)
    reach = (int(np.argmax(hist <= target)) + 1) * every
    W2, H2, _ = c.rnmf(A, w.k, w.p, w.q, reach, w.seed, precision=1)
    W3, H3, _ = c.rnmf(A, w.k, w.p, w.q, reach, w.seed, precision=1)
    torch.cuda.synchronize()
    assert torch.equal(W2, W3) and torch.equal(H2, H3)
    for X in (W1, H1, W2, H2):
        assert bool(torch.isfinite(X).all()) and float(X.min()) >= 0.0
    assert c.rel_err(A, W2, H2) <= target


def test_fullsize_solve_against_oracle(full):
    c, _, A = full
    w = W_FULL
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", f"oracle_{w.name}.json")))
    ore = np.array(g["rhals"]["rel_err_every_10"])
    assert (g["m"], g["n"], g["k"], g["p"], g["q"], g["iters"]) == (w.m, w.n, w.k, w.p, w.q, w.iters)
    devs = {}
    for precision in (0, 1, 2):
        _, _, st = c.rnmf(A, w.k, w.p, w.q, w.iters, w.seed, precision=precision, track_every=10)
        h = np.array(st.rel_err_hist)
        assert h.shape == ore.shape
        devs[precision] = abs(h[-1] - ore[-1]) / ore[-1]
    print(f"final relative error vs the float64 oracle after {w.iters} sweeps: FP32 form {devs[0]:.2e}, "
          f"BF16 form {devs[1]:.2e}, 3-term split form {devs[2]:.2e}")
    assert devs[0] < 5e-3
    assert devs[1] < 0.1 and devs[2] < 0.1
