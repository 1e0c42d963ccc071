"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances:
  * random draws and initial factors: bit-identical (integer Philox + fixed
    IEEE operation order on both sides);
  * QB: Q^T Q = I to 5e-6 (float32 CholeskyQR2), span(Q) equal to the
    oracle's up to the float32 subspace error, B^T = A^T Q checked in float64;
  * per-sweep relative error ||A - WH||/||A|| within 1e-5 relative of the oracle
    for the float32 form (1000 x 500, k = 10, the small synthetic workload), and
    the final relative error within 1e-3 relative;
  * single sweeps from identical float32 inputs: W, H within 2e-5 relative
    (float32 rounding of k- and l-long sums) of the oracle.
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


# ------------------------------------------------------------- random draws
@pytest.mark.parametrize("n,l,dist", [(500, 20, 0), (37, 13, 0), (20000, 70, 0), (501, 19, 1), (1, 1, 0)])
def test_omega_bit_identical(ctx, n, l, dist):
    got = ctx.omega(n, l, seed=0, dist=dist)
    torch.cuda.synchronize()
    ref = philox.omega(n, l, 0, dist).astype(np.float32)
    assert np.array_equal(got.cpu().numpy().view(np.uint32), ref.view(np.uint32))


def test_omega_seed_changes_draw(ctx):
    a = ctx.omega(100, 10, seed=0).cpu().numpy()
    b = ctx.omega(100, 10, seed=1 << 33).cpu().numpy()
    ref = philox.omega(100, 10, 1 << 33).astype(np.float32)
    assert not np.array_equal(a, b)
    assert np.array_equal(b.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("m,n,k", [(1000, 500, 10), (33, 17, 3)])
def test_init_factors_bit_identical(ctx, m, n, k):
    W, H = ctx.init_factors(m, n, k, seed=0)
    W0, H0 = philox.init_factors(m, n, k, 0)
    assert np.array_equal(W.cpu().numpy(), W0.astype(np.float32))
    assert np.array_equal(H.cpu().numpy(), H0.astype(np.float32))


# ------------------------------------------------------------------- QB
@pytest.mark.parametrize("m,n,l,q", [(1000, 500, 20, 2), (777, 1301, 37, 1), (130, 90, 7, 0)])
def test_qb_properties_and_span(ctx, m, n, l, q):
    w = synth.Workload("t", m, n, 10, l, 0, q, 0, 0.01)
    A = synth.lowrank(w)
    Q, Bt = ctx.qb(dev(A), l, q, seed=0)
    Qh, Bth = host(Q), host(Bt)
    assert np.max(np.abs(Qh.T @ Qh - np.eye(l))) < 5e-6
    # B^T = A^T Q, checked in float64 from the GPU's own Q
    ref_Bt = A.astype(np.float64).T @ Qh
    assert np.max(np.abs(Bth - ref_Bt)) / np.max(np.abs(ref_Bt)) < 2e-6
    # the leading (signal) subspace agrees with the oracle's Householder-QR basis
    Qo, Bo = R.rqb(A, philox.omega(n, l, 0), q)
    P = Qh @ (Qh.T @ Qo[:, :10])
    assert np.linalg.norm(P - Qo[:, :10]) / np.sqrt(10) < 1e-4
    # captured energy equal to the oracle's
    e_gpu = np.linalg.norm(A.astype(np.float64) - Qh @ (Qh.T @ A)) / np.linalg.norm(A)
    e_ora = np.linalg.norm(A.astype(np.float64) - Qo @ Bo) / np.linalg.norm(A)
    assert abs(e_gpu - e_ora) <= 1e-3 * e_ora + 1e-7


def test_qb_rank_deficient_sketch_uses_shift(ctx):
    # exactly low-rank A with l > rank: Y is numerically rank deficient; the
    # shifted CholeskyQR pass must still return an orthonormal basis spanning range(A)
    w = synth.Workload("t", 400, 300, 5, 15, 0, 1, 0, 0.0)
    A = synth.lowrank(w)
    Q, Bt = ctx.qb(dev(A), 15, 1, seed=0)
    Qh = host(Q)
    assert np.max(np.abs(Qh.T @ Qh - np.eye(15))) < 5e-6
    A64 = A.astype(np.float64)
    assert np.linalg.norm(A64 - Qh @ (Qh.T @ A64)) / np.linalg.norm(A64) < 1e-6


# --------------------------------------------------------------- sweeps
@pytest.mark.parametrize("gram_mode", [0, 1])
def test_single_sweep_matches_oracle(ctx, gram_mode):
    w = synth.Workload("t", 1000, 500, 10, 10, 10, 2, 0, 0.01)
    A = synth.lowrank(w)
    Q, B = R.rqb(A, philox.omega(500, 20, 0), 2)
    Q32, B32 = Q.astype(np.float32), B.astype(np.float32)
    W0, H0 = philox.init_factors(1000, 500, 10, 0)
    # oracle sweep on the same float32 inputs
    Wo, Ho, Wto, _ = R.rhals_sweeps(Q32.astype(np.float64), B32.astype(np.float64), W0, H0, 1, gram_mode)
    W, H = dev(W0), dev(H0)
    ctx.sweeps(dev(Q32), dev(B32.T), W, H, 1, gram_mode=gram_mode)
    Wg, Hg = host(W), host(H)
    assert np.all(Wg >= 0) and np.all(Hg >= 0)
    assert np.max(np.abs(Hg - Ho)) / np.max(np.abs(Ho)) < 2e-5
    assert np.max(np.abs(Wg - Wo)) / np.max(np.abs(Wo)) < 2e-5


@pytest.mark.parametrize("m,n,k,p", [(700, 333, 7, 6), (1500, 130, 33, 15), (400, 65, 1, 0)])
def test_single_sweep_ragged_shapes(ctx, m, n, k, p):
    # odd l (rows of B^T not a multiple of 16 bytes), k not a multiple of the
    # 8-row chunk, n a ragged number of 64-column tiles
    w = synth.Workload("t", m, n, k, k, p, 1, 0, 0.02)
    A = synth.lowrank(w)
    l = k + p
    Q, B = R.rqb(A, philox.omega(n, l, 0), 1)
    Q32, B32 = Q.astype(np.float32), B.astype(np.float32)
    W0, H0 = philox.init_factors(m, n, k, 0)
    Wo, Ho, _, _ = R.rhals_sweeps(Q32.astype(np.float64), B32.astype(np.float64), W0, H0, 3)
    W, H = dev(W0), dev(H0)
    ctx.sweeps(dev(Q32), dev(B32.T), W, H, 3)
    Wg, Hg = host(W), host(H)
    # three sweeps of float32 rounding (single sweeps are held to 2e-5 above)
    assert np.max(np.abs(Hg - Ho)) / np.max(np.abs(Ho)) < 1e-4
    assert np.max(np.abs(Wg - Wo)) / np.max(np.abs(Wo)) < 1e-4


def test_rnmf_small_per_sweep_parity(ctx):
    w = synth.SMALL
    A = synth.lowrank(w)
    W, H, st = ctx.rnmf(dev(A), w.k, w.p, w.q, w.iters, w.seed, track_every=1)
    ref = R.rhals(A, w.k, w.p, w.q, w.iters, w.seed, track=True)
    got = np.array(st.rel_err_hist)
    assert got.shape == ref["hist"].shape
    rel = np.abs(got - ref["hist"]) / ref["hist"]
    assert rel.max() < 1e-5, rel.max()
    assert abs(st.final_rel_err - ref["hist"][-1]) / ref["hist"][-1] < 1e-3
    Wg, Hg = host(W), host(H)
    assert np.all(Wg >= 0) and np.all(Hg >= 0)
    # the relative error reported by the library equals the one of the returned factors
    e = np.linalg.norm(A.astype(np.float64) - Wg @ Hg) / np.linalg.norm(A.astype(np.float64))
    assert abs(e - st.final_rel_err) / e < 1e-6


def test_rnmf_gram_mode_and_uniform_omega(ctx):
    w = synth.Workload("t", 600, 400, 8, 8, 8, 1, 30, 0.02)
    A = synth.lowrank(w)
    for gm, od in [(1, 0), (0, 1)]:
        _, _, st = ctx.rnmf(dev(A), w.k, w.p, w.q, w.iters, 3, gram_mode=gm, omega_dist=od, track_every=1)
        ref = R.rhals(A, w.k, w.p, w.q, w.iters, 3, gram_mode=gm, omega_dist=od, track=True)
        rel = np.abs(np.array(st.rel_err_hist) - ref["hist"]) / ref["hist"]
        assert rel.max() < 1e-5, (gm, od, rel.max())


def test_deterministic_hals_parity(ctx):
    w = synth.Workload("t", 700, 450, 8, 8, 0, 0, 60, 0.02)
    A = synth.lowrank(w)
    W, H, st = ctx.hals(dev(A), w.k, w.iters, seed=5, track_every=1)
    ref = R.hals(A, w.k, w.iters, 5, track=True)
    rel = np.abs(np.array(st.rel_err_hist) - ref["hist"]) / ref["hist"]
    assert rel.max() < 1e-5, rel.max()
    # monotone (exact BCD), up to float32 rounding of the error itself
    h = np.array(st.rel_err_hist)
    assert np.all(np.diff(h) <= 1e-6 * h[:-1])


def test_square_q_rnmf_equals_hals(ctx):
    # l = k + p = m <= n: Q is square and orthogonal, rHALS reduces to HALS
    m, n, k = 24, 40, 4
    w = synth.Workload("t", m, n, 4, k, m - k, 1, 0, 0.01)
    A = synth.lowrank(w)
    _, _, st_r = ctx.rnmf(dev(A), k, m - k, 1, 25, 0, track_every=1)
    _, _, st_h = ctx.hals(dev(A), k, 25, 0, track_every=1)
    a, b = np.array(st_r.rel_err_hist), np.array(st_h.rel_err_hist)
    assert np.max(np.abs(a - b) / b) < 1e-4


def test_rel_err_matches_float64(ctx):
    w = synth.Workload("t", 333, 257, 6, 6, 0, 0, 0, 0.05)
    A = synth.lowrank(w)
    rng = np.random.default_rng(0)
    W, H = rng.random((333, 6)), rng.random((6, 257))
    got = ctx.rel_err(dev(A), dev(W), dev(H))
    W32, H32 = W.astype(np.float32).astype(np.float64), H.astype(np.float32).astype(np.float64)
    ref = R.rel_err(A, W32, H32)
    assert abs(got - ref) / ref < 1e-6


def test_k_equal_one_and_padded_lda(ctx):
    w = synth.Workload("t", 257, 129, 1, 1, 3, 1, 15, 0.01)
    A = synth.lowrank(w)
    Apad = np.zeros((257, 160), np.float32)
    Apad[:, :129] = A
    dA = dev(Apad)[:, :129]
    _, _, st = ctx.rnmf(dA, 1, 3, 1, 15, 0, track_every=1)
    ref = R.rhals(A, 1, 3, 1, 15, 0, track=True)
    rel = np.abs(np.array(st.rel_err_hist) - ref["hist"]) / ref["hist"]
    assert rel.max() < 1e-5


def test_dead_component_stays_finite(ctx):
    # H_init row forced to zero: V_jj = 0 on the first sweep, the column update is skipped
    w = synth.Workload("t", 200, 150, 4, 4, 4, 1, 0, 0.01)
    A = synth.lowrank(w)
    Q, B = R.rqb(A, philox.omega(150, 8, 0), 1)
    W0, H0 = philox.init_factors(200, 150, 4, 0)
    H0[2] = 0.0
    Wo, Ho, _, _ = R.rhals_sweeps(Q.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64),
                                  W0, H0, 3)
    W, H = dev(W0), dev(H0)
    ctx.sweeps(dev(Q), dev(B.T), W, H, 3)
    Wg, Hg = host(W), host(H)
    assert np.all(np.isfinite(Wg)) and np.all(np.isfinite(Hg))
    assert np.max(np.abs(Hg - Ho)) / np.max(np.abs(Ho)) < 1e-4


def test_invalid_arguments_are_rejected(ctx):
    import paper_1711_02037_gb300 as pkg
    A = dev(np.ones((50, 40), np.float32))
    W = torch.full((50, 5), -7.0, device="cuda")
    H = torch.full((5, 40), -7.0, device="cuda")
    for args in [(5, 100, 1, 3), (0, 2, 1, 3), (5, -1, 1, 3), (5, 2, -1, 3), (5, 2, 1, -1), (120, 10, 1, 1)]:
        with pytest.raises(pkg.RnmfError) as e:
            ctx.rnmf(A, *args, W=W, H=H)
        assert e.value.status == 1
    assert torch.all(W == -7.0) and torch.all(H == -7.0)
