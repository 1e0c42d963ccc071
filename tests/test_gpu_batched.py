"""Batched ragged problems (rnmf_batched) against the float64 oracle.

Each problem of a batch is what rnmf() computes for it with its own Philox
instance word, so the oracle is oracle.rhals(..., instance=i) problem by
problem.  Tolerances:
  * initial factors (iters = 0): bit-identical to the oracle's draws;
  * final relative error ||A - WH||_F / ||A||_F within 1e-3 relative of the
    oracle's (the float32 form's bound for a whole run);
  * every cluster size and thread count the autotuner can choose gives the
    same bound; a replay of the captured graph gives identical factors.
"""
import numpy as np
import pytest

import synth
from oracle import philox
from oracle import rhals as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# ragged shapes: (m, n, r = k), p = 10 unless stated; l = k + p from 12 to 42
SHAPES = [(300, 200, 5), (257, 129, 4), (600, 150, 12), (128, 500, 8), (1000, 333, 20), (64, 64, 3),
          (777, 401, 32), (150, 100, 7), (512, 512, 16), (90, 80, 2), (2048, 1100, 25), (33, 47, 1)]


@pytest.fixture(scope="module")
def cx():
    import paper_1711_02037_gb300 as pkg
    c = pkg.Context(0)
    yield c
    c.close()


def workloads(shapes=SHAPES, q=2, iters=100, p=10, seed=0):
    out = []
    for i, (m, n, r) in enumerate(shapes):
        pp = min(p, min(m, n) - r)
        out.append(synth.Workload(f"b{i}", m, n, r, r, pp, q if np.isscalar(q) else q[i], iters, 0.01,
                                  seed=seed, instance=i + 1))
    return out


def items_for(ws, lda_pad=0):
    items = []
    for w in ws:
        A = np.zeros((w.m, w.n + lda_pad), np.float32)
        synth.lowrank_into(A, w)
        Ad = torch.from_numpy(A).cuda()[:, : w.n]
        items.append(dict(A=Ad, k=w.k, p=w.p, q=w.q, iters=w.iters, seed=w.seed, instance=w.instance,
                          W=torch.empty(w.m, w.k, device="cuda"), H=torch.empty(w.k, w.n, device="cuda"),
                          host=A[:, : w.n]))
    return items


def oracle_err(w, A, gram_mode=0, omega_dist=0):
    res = R.rhals(A.astype(np.float64), w.k, w.p, w.q, w.iters, w.seed, gram_mode, omega_dist,
                  instance=w.instance)
    return R.rel_err(A.astype(np.float64), res["W"], res["H"])


@pytest.fixture(scope="module")
def batch():
    ws = workloads()
    items = items_for(ws, lda_pad=3)
    ref = [oracle_err(w, it["host"]) for w, it in zip(ws, items)]
    return ws, items, ref


def check_against_oracle(cx, items, ref):
    errs = cx.batched_rel_err(items)
    for i, (g, o) in enumerate(zip(errs, ref)):
        assert abs(g - o) <= 1e-3 * o, (i, g, o)
    for it in items:
        assert float(it["W"].min()) >= 0.0 and float(it["H"].min()) >= 0.0


def test_initial_factors_bit_identical(cx):
    ws = workloads(iters=0)
    items = items_for(ws)
    status, _ = cx.batched(items)
    torch.cuda.synchronize()
    assert status == [0] * len(ws)
    for w, it in zip(ws, items):
        W0, H0 = philox.init_factors(w.m, w.n, w.k, w.seed, w.instance)
        assert np.array_equal(it["W"].cpu().numpy(), W0.astype(np.float32))
        assert np.array_equal(it["H"].cpu().numpy(), H0.astype(np.float32))


def test_batch_matches_oracle(cx, batch):
    ws, items, ref = batch
    cx.batched_config(0, 0)
    status, stats = cx.batched(items)
    assert status == [0] * len(ws)
    assert stats["tuned"] == 1 and stats["graph_kernels"] > 0
    assert sum(stats["cluster_count"]) == len(ws)
    check_against_oracle(cx, items, ref)


def test_replay_is_identical(cx, batch):
    ws, items, ref = batch
    cx.batched(items)
    W1 = [it["W"].clone() for it in items]
    H1 = [it["H"].clone() for it in items]
    for it in items:
        it["W"].zero_()
        it["H"].zero_()
    _, stats = cx.batched(items)
    assert stats["tuned"] == 0
    for it, a, b in zip(items, W1, H1):
        assert torch.equal(it["W"], a) and torch.equal(it["H"], b)


@pytest.mark.parametrize("max_cluster,threads", [(1, 256), (1, 512), (2, 256), (4, 512), (8, 256)])
def test_every_configuration(cx, batch, max_cluster, threads):
    ws, items, ref = batch
    cx.batched_config(max_cluster, threads)
    try:
        status, stats = cx.batched(items)
        assert status == [0] * len(ws)
        if max_cluster > 1:
            assert stats["cluster_count"][{2: 1, 4: 2, 8: 3}[max_cluster]] >= 1
        check_against_oracle(cx, items, ref)
    finally:
        cx.batched_config(0, 0)


def test_mixed_power_iterations_and_options(cx):
    shapes = SHAPES[:6]
    ws = workloads(shapes, q=[0, 1, 2, 3, 0, 1], iters=60)
    items = items_for(ws)
    for gm, od in ((0, 0), (1, 0), (0, 1)):
        status, _ = cx.batched(items, gram_mode=gm, omega_dist=od)
        assert status == [0] * len(ws)
        errs = cx.batched_rel_err(items)
        for w, it, g in zip(ws, items, errs):
            o = oracle_err(w, it["host"], gm, od)
            assert abs(g - o) <= 1e-3 * o, (w, gm, od, g, o)


def test_instance_zero_equals_single_problem_entry(cx):
    w = synth.Workload("single", 1000, 500, 10, 10, 10, 2, 100, 0.01)
    items = items_for([w])
    cx.batched(items)
    Wd, Hd, _ = cx.rnmf(items[0]["A"].contiguous(), w.k, w.p, w.q, w.iters, seed=0)
    e_batch = cx.batched_rel_err(items)[0]
    e_single = cx.rel_err(items[0]["A"].contiguous(), Wd, Hd)
    assert abs(e_batch - e_single) <= 1e-3 * e_single


def test_rejects_invalid_problem(cx):
    import paper_1711_02037_gb300 as pkg
    ws = workloads(SHAPES[:2], iters=1)
    items = items_for(ws)
    items[1]["k"] = 40  # k > 32
    with pytest.raises(pkg.RnmfError, match="problem 1"):
        cx.batched(items)
    items[1]["k"] = 4
    items[1]["p"] = 200  # l > min(m, n)
    with pytest.raises(pkg.RnmfError, match="problem 1"):
        cx.batched(items)
