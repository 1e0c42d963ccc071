"""Failure paths of the CUDA library, made on the host, with no GPU fault.

  * A bounded device-side wait that runs out: the W half's blocks wait for
    each other's partial sums with a cycle limit (rnmf_opts.spin_limit).  With
    a limit of one cycle the first incomplete poll gives up, the kernel records
    RNMF_ETIMEOUT in the context's status word, frees its tensor memory and
    returns; the call reports it and the same context runs the next solve to
    the oracle's trajectory.
  * A Gram matrix that is not positive definite even after the shift: A = 0
    makes Y = A Omega = 0 (the degenerate input of the QR step), so CholeskyQR
    reports RNMF_ENOTPD.
  * A scratch allocation that fails: the context's scratch cap
    (rnmf_set_scratch_limit) makes the arena, the host staging and the batch
    workspace refuse to grow, so the calls return RNMF_ENOMEM before any work
    and leave their outputs untouched.
"""
import numpy as np
import pytest

import synth
from oracle import rhals as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OK, EINVAL, ENOMEM, ECUDA, ENOTPD, ETIMEOUT = 0, 1, 2, 3, 4, 5


@pytest.fixture()
def ctx():
    import paper_1711_02037_gb300 as pkg
    c = pkg.Context(0)
    yield c
    c.close()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


@pytest.mark.parametrize("m,n,k,p", [(1000, 500, 10, 10), (40000, 1500, 8, 8)])
def test_wait_limit_runs_out_then_context_recovers(ctx, m, n, k, p):
    # 40000 rows over the SMs put rows of Q in tensor memory: the early return
    # must free it, or the next launch could not allocate it
    import paper_1711_02037_gb300 as pkg
    w = synth.Workload("t", m, n, k, k, p, 1, 5, 0.01)
    A = dev(synth.lowrank(w))
    with pytest.raises(pkg.RnmfError) as e:
        ctx.rnmf(A, w.k, w.p, w.q, w.iters, 0, spin_limit=1)
    assert e.value.status == ETIMEOUT
    # the same context, default limit: the solve completes and is correct
    A_np = synth.lowrank(w)
    _, _, st = ctx.rnmf(A, w.k, w.p, w.q, w.iters, 0, track_every=1)
    if m * n <= 1000 * 500:
        ref = R.rhals(A_np, w.k, w.p, w.q, w.iters, 0, track=True)
        rel = np.abs(np.array(st.rel_err_hist) - ref["hist"]) / ref["hist"]
        assert rel.max() < 1e-5
    else:
        h = np.array(st.rel_err_hist)
        assert np.all(np.isfinite(h)) and h[-1] < h[0]


def test_zero_matrix_reports_not_positive_definite(ctx):
    import paper_1711_02037_gb300 as pkg
    A0 = torch.zeros(300, 200, device="cuda")
    with pytest.raises(pkg.RnmfError) as e:
        ctx.rnmf(A0, 5, 5, 1, 3, 0)
    assert e.value.status == ENOTPD
    with pytest.raises(pkg.RnmfError) as e:
        ctx.qb(A0, 10, 1)
    assert e.value.status == ENOTPD
    # the context stays usable
    w = synth.Workload("t", 300, 200, 5, 5, 5, 1, 10, 0.01)
    A = synth.lowrank(w)
    _, _, st = ctx.rnmf(dev(A), w.k, w.p, w.q, w.iters, 0, track_every=1)
    ref = R.rhals(A, w.k, w.p, w.q, w.iters, 0, track=True)
    assert np.max(np.abs(np.array(st.rel_err_hist) - ref["hist"]) / ref["hist"]) < 1e-5


def test_scratch_limit_reports_out_of_memory(ctx):
    import paper_1711_02037_gb300 as pkg
    w = synth.SMALL
    A_np = synth.lowrank(w)
    A = dev(A_np)
    W = torch.full((w.m, w.k), -7.0, device="cuda")
    H = torch.full((w.k, w.n), -7.0, device="cuda")
    ctx.set_scratch_limit(4096)
    with pytest.raises(pkg.RnmfError) as e:
        ctx.rnmf(A, w.k, w.p, w.q, w.iters, 0, W=W, H=H)
    assert e.value.status == ENOMEM
    assert torch.all(W == -7.0) and torch.all(H == -7.0)
    with pytest.raises(pkg.RnmfError) as e:
        ctx.rnmf_host(A_np, w.k, w.p, w.q, w.iters, 0)
    assert e.value.status == ENOMEM
    items = [dict(A=A, k=w.k, p=w.p, q=w.q, iters=2, W=W, H=H)]
    with pytest.raises(pkg.RnmfError) as e:
        ctx.batched(items)
    assert e.value.status == ENOMEM
    assert ctx.scratch_bytes() == 0
    # without the cap the same call runs; a cap at what it now holds still
    # lets calls of the same size run (no growth needed)
    ctx.set_scratch_limit(0)
    _, _, st = ctx.rnmf(A, w.k, w.p, w.q, w.iters, 0, W=W, H=H, track_every=w.iters)
    held = ctx.scratch_bytes()
    assert held > 4096
    ctx.set_scratch_limit(held)
    _, _, st2 = ctx.rnmf(A, w.k, w.p, w.q, w.iters, 0, track_every=w.iters)
    assert st2.final_rel_err == st.final_rel_err
    ref = R.rhals(A_np, w.k, w.p, w.q, w.iters, 0, track=True)
    assert abs(st.final_rel_err - ref["hist"][-1]) / ref["hist"][-1] < 1e-3
