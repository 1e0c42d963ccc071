"""rnmf_rel_err_noalloc: the relative error with the library's fixed device
scratch instead of its allocating arena (collected last on purpose: it must pass
after every other test has run on the same device, as well as alone).

Both entries run the same tile kernel and the same fixed-order float64
reduction, so the two results are expected to agree to the last bit; the test
allows 1e-12 relative.
"""
import numpy as np
import pytest

import synth
from oracle import philox

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


def inputs(m, n, k, lda=None):
    w = synth.Workload("noalloc", m, n, k, k, 0, 1, 1, 0.01)
    A = synth.lowrank(w)
    W0, H0 = philox.init_factors(m, n, k, 3)
    Ad = dev(A)
    if lda is not None:
        buf = torch.zeros(m, lda, device="cuda")
        buf[:, :n] = Ad
        Ad = buf[:, :n]
    return Ad, dev(W0), dev(H0)


@pytest.mark.parametrize("m,n,k,lda", [(1000, 500, 10, None), (777, 333, 7, 340), (64, 64, 1, None),
                                       (50000, 2000, 50, None)])
def test_matches_allocating_entry_twice(cx, m, n, k, lda):
    A, W, H = inputs(m, n, k, lda)
    ref = cx.rel_err(A, W, H)
    first = cx.rel_err_noalloc(A, W, H)
    second = cx.rel_err_noalloc(A, W, H)
    assert ref > 0
    assert abs(first - ref) <= 1e-12 * ref, (first, ref)
    assert abs(second - ref) <= 1e-12 * ref, (second, ref)


def test_later_calls_leave_free_memory_unchanged(cx):
    A, W, H = inputs(1000, 500, 10)
    cx.rel_err_noalloc(A, W, H)  # first call on the device looks the array up
    torch.cuda.synchronize()
    before = torch.cuda.mem_get_info()[0]
    vals = [cx.rel_err_noalloc(A, W, H) for _ in range(3)]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == before
    assert vals[0] == vals[1] == vals[2]


def test_rejects_problem_beyond_fixed_scratch(cx):
    import paper_1711_02037_gb300 as pkg
    # one row: ceil(n / 64) tiles, one more than the 262144 the array holds
    n = 64 * 262144 + 1
    A = torch.ones(1, n, device="cuda")
    W = torch.ones(1, 1, device="cuda")
    H = torch.ones(1, n, device="cuda")
    with pytest.raises(pkg.RnmfError, match="262144"):
        cx.rel_err_noalloc(A, W, H)
    # the largest accepted problem of that shape still works
    A2, H2 = A[:, : n - 1].contiguous(), H[:, : n - 1].contiguous()
    assert cx.rel_err_noalloc(A2, W, H2) == 0.0


def test_rejects_while_profiling(cx):
    import paper_1711_02037_gb300 as pkg
    A, W, H = inputs(64, 64, 1)
    cx.profile(True)
    try:
        with pytest.raises(pkg.RnmfError, match="profiling"):
            cx.rel_err_noalloc(A, W, H)
    finally:
        cx.profile(False)
    assert cx.rel_err_noalloc(A, W, H) == pytest.approx(cx.rel_err(A, W, H), rel=1e-12)
