"""GPU adjoint of T compressed sweeps against the float64 reference gradient.

Loss L = <G, W_T H_T> (formed by the caller), Q held fixed, so gradients reach A
through B = Q^T A.  Both sides start from the same float32 inputs: A, Q (the
oracle's float64 QB rounded to float32), W_init, H_init, G.  The oracle then
runs in float64 on those values.

Tolerance: the loss within 1e-5 relative; each gradient (dA, dW_init, dH_init)
within 1e-4 of the reference in relative Frobenius norm, and every entry within
2e-4 of the gradient's largest entry, when every clamp decision of the float32
forward pass equals the oracle's.  The GPU trajectory
differs from the float64 one by rounding (~1e-6 relative per sweep), so a clamp
argument within rounding of 0 can fall on the other side; the two gradients are
then those of adjacent linear pieces.  In that case the test requires the
flipped decisions to be rare (<= 1e-5 of all decisions) and each within 1e-3 of
its row's (column's) largest argument from the kink, and bounds the gradients
by 5e-3 instead.  The GPU's decisions are read from its checkpoints
(W_t > 0, H_t > 0).
"""
import numpy as np
import pytest

import synth
from oracle import adjoint as AD
from oracle import philox
from oracle import rhals as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cx():
    import paper_1711_02037_gb300 as pkg
    c = pkg.Context(0)
    yield c
    c.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def instance(w, A=None):
    A = synth.lowrank(w) if A is None else A
    Q, _ = R.rqb(A.astype(np.float64), philox.omega(w.n, w.l, w.seed), w.q)
    W0, H0 = philox.init_factors(w.m, w.n, w.k, w.seed)
    G = synth.cotangent(w.m, w.n)
    return f32(A), f32(Q), f32(W0), f32(H0), f32(G)


def gpu_grads(cx, inst, T, gm):
    import paper_1711_02037_gb300 as pkg
    A, Q, W0, H0, G = (dev(x) for x in inst)
    A.requires_grad_(True)
    W0.requires_grad_(True)
    H0.requires_grad_(True)
    W, H = pkg.rhals_sweeps(cx, A, Q, W0, H0, T, gm)
    L = (G.double() * (W.double() @ H.double())).sum()
    L.backward()
    torch.cuda.synchronize()
    return (float(L.detach()), A.grad.double().cpu().numpy(), W0.grad.double().cpu().numpy(),
            H0.grad.double().cpu().numpy(), W.detach().double().cpu().numpy(), H.detach().double().cpu().numpy())


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def clamp_flips(cx, inst, T, gm):
    """Clamp decisions of the GPU forward pass that differ from the oracle's:
    [(t, "H" | "W", j, index, argument / largest |argument| of that row or column)]
    and the number of decisions compared."""
    A, Q, W0, H0, G = inst
    args = AD.clamp_arguments(A, Q, W0, H0, T, gm)
    Ad, Qd = dev(A), dev(Q)
    Bt = cx.sketch(Ad, Qd, transpose=True)
    _, _, ck = cx.sweeps_fwd(Qd, Bt, dev(W0), dev(H0), T, gm)
    torch.cuda.synchronize()
    ckh = ck.cpu().numpy()
    m, l = Q.shape
    k, n = W0.shape[1], A.shape[1]
    size = k * m + l * k + k * n
    flips, count = [], 0
    for t, kind, j, a in args:
        base = t * size
        if kind == "W":
            got = ckh[base + j * m: base + (j + 1) * m]
        else:
            off = base + k * m + l * k
            got = ckh[off + j * n: off + (j + 1) * n]
        count += a.size
        scale = np.abs(a).max()
        flips += [(t, kind, j, int(i), float(a[i] / scale)) for i in np.nonzero((got > 0) != (a > 0))[0]]
    return flips, count


def check(cx, inst, T, gm):
    Lg, gA, gW, gH, Wg, Hg = gpu_grads(cx, inst, T, gm)
    L, rA, rW, rH = AD.loss_and_grads(*inst, T, gm)
    A, Q, W0, H0, G = inst
    Wr, Hr, _ = AD.sweeps(torch.tensor(Q), torch.tensor(Q.T @ A), torch.tensor(W0), torch.tensor(H0), T, gm)
    assert rel(Wg, Wr.numpy()) < 2e-5 and rel(Hg, Hr.numpy()) < 2e-5
    assert abs(Lg - L) <= 1e-5 * abs(L), (Lg, L)
    flips, count = clamp_flips(cx, inst, T, gm)
    tol = 1e-4
    if flips:
        assert len(flips) <= 1e-5 * count, flips[:20]
        assert all(abs(f[-1]) <= 1e-3 for f in flips), flips
        tol = 5e-3
    for name, g, r in (("dA", gA, rA), ("dW0", gW, rW), ("dH0", gH, rH)):
        assert rel(g, r) < tol, (name, rel(g, r), len(flips))
        if not flips:
            # every clamp decision agrees: entry by entry, against the gradient's largest entry
            assert np.max(np.abs(g - r)) <= 2e-4 * np.max(np.abs(r)), (name, np.max(np.abs(g - r)) / np.max(np.abs(r)))
    return gA, Q, flips


@pytest.mark.parametrize("gm", [0, 1])
def test_fd_instance(cx, gm):
    check(cx, instance(synth.ADJOINT_FD), synth.ADJOINT_FD.iters, gm)


@pytest.mark.parametrize("T", [10, 50])
def test_differentiation_workload(cx, T):
    # 4096 x 2048, k = 16, l = 26, q = 1; T = 50 is the workload, T = 10 a prefix of it
    w = synth.ADJOINT
    gA, Q, flips = check(cx, instance(w), T, 0)
    if T == 10:
        assert not flips
    # dL/dA = Q dL/dB lies in range(Q)
    assert np.linalg.norm(gA - Q @ (Q.T @ gA)) <= 1e-5 * np.linalg.norm(gA)


@pytest.mark.parametrize("m,n,k,l,T", [(300, 200, 7, 13, 3), (129, 517, 5, 5, 2), (1000, 65, 9, 20, 4)])
def test_ragged_shapes(cx, m, n, k, l, T):
    w = synth.Workload("adjoint_ragged", m, n, k, k, l - k, 1, T, 0.01)
    check(cx, instance(w), T, 0)


def test_zero_sweeps_is_identity(cx):
    # T = 0: W_T = W_init, H_T = H_init, so dW_init = G H^T, dH_init = W^T G and dA = 0
    inst = instance(synth.ADJOINT_FD)
    Lg, gA, gW, gH, _, _ = gpu_grads(cx, inst, 0, 0)
    A, Q, W0, H0, G = inst
    assert np.abs(gA).max() == 0.0
    assert rel(gW, G @ H0.T) < 1e-6 and rel(gH, W0.T @ G) < 1e-6


def test_abi_matches_autograd(cx):
    # the three C-ABI calls directly, against the autograd wrapper
    inst = instance(synth.ADJOINT_FD)
    T = synth.ADJOINT_FD.iters
    _, gA, gW, gH, _, _ = gpu_grads(cx, inst, T, 0)
    A, Q, W0, H0, G = (dev(x) for x in inst)
    Bt = cx.sketch(A, Q, transpose=True)
    W, H, ck = cx.sweeps_fwd(Q, Bt, W0.clone(), H0.clone(), T)
    # the wrapper's cotangents: L = sum(G * (W H)) in float64, cast back to float32
    dW = (G.double() @ H.double().T).float().contiguous()
    dH = (W.double().T @ G.double()).float().contiguous()
    dBt, dW0, dH0 = cx.sweeps_bwd(Q, Bt, ck, dW, dH, T)
    dA = cx.dA(Q, dBt)
    torch.cuda.synchronize()
    assert rel(dA.double().cpu().numpy(), gA) < 1e-6
    assert rel(dW0.double().cpu().numpy(), gW) < 1e-6
    assert rel(dH0.double().cpu().numpy(), gH) < 1e-6


def test_rejects_oversized_adjoint(cx):
    import paper_1711_02037_gb300 as pkg
    Q = torch.zeros(200, 128, device="cuda")
    Bt = torch.zeros(150, 128, device="cuda")
    ck = torch.zeros(1, device="cuda")
    dW = torch.zeros(200, 100, device="cuda")
    dH = torch.zeros(100, 150, device="cuda")
    with pytest.raises(pkg.RnmfError):
        cx.sweeps_bwd(Q, Bt, ck, dW, dH, 1)
