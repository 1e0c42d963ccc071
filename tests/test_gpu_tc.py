"""Tensor-core (tcgen05) forms of the QB products against float64 references.

Tolerances follow from the operand rounding: one bf16 product carries a
relative error ~2^-9 per operand; the 3-term hi/lo split leaves ~3 * 2^-18 per
product; the float32 CUDA-core form is float32 accurate.  Errors are measured
as ||out - ref||_F / ||ref||_F on shapes with ragged M, K and l tails.
"""
import numpy as np
import pytest

import synth
from oracle import rhals as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(1000, 777, 20), (300, 4100, 128), (4096, 2048, 26), (129, 65, 1), (2000, 130, 70)]
TOL = {0: 2e-6, 1: 2e-2, 2: 5e-5}


@pytest.fixture(scope="module")
def ctx():
    import paper_1711_02037_gb300 as pkg
    c = pkg.Context(0)
    yield c
    c.close()


def _A(m, n):
    w = synth.Workload("t", m, n, 8, 8, 0, 0, 0, 0.01)
    return synth.lowrank(w)


def _dev_padded(A):
    """Device copy of A with the leading dimension rounded up to a multiple of 4
    (the tensor-core forms need a 16-byte row pitch); n itself stays ragged."""
    m, n = A.shape
    lda = (n + 3) // 4 * 4
    buf = torch.zeros((m, lda), dtype=torch.float32, device="cuda")
    buf[:, :n] = torch.from_numpy(A).cuda()
    return buf[:, :n]


@pytest.mark.parametrize("form", [0, 1, 2])
@pytest.mark.parametrize("m,n,l", SHAPES)
def test_sketch_products(ctx, m, n, l, form):
    A = _A(m, n)
    rng = np.random.default_rng(m + n + l)
    A64 = A.astype(np.float64)
    dA = _dev_padded(A)
    X1 = rng.standard_normal((n, l)).astype(np.float32)
    Y = ctx.sketch(dA, torch.from_numpy(X1).cuda(), transpose=False, form=form)
    ref = A64 @ X1.astype(np.float64)
    err = np.linalg.norm(Y.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < TOL[form], ("ax", err)
    X2 = rng.standard_normal((m, l)).astype(np.float32)
    Z = ctx.sketch(dA, torch.from_numpy(X2).cuda(), transpose=True, form=form)
    ref = A64.T @ X2.astype(np.float64)
    err = np.linalg.norm(Z.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < TOL[form], ("atx", err)


def test_sketch_split3_rowwise_accuracy(ctx):
    # every output entry, not only the norm: |err_ij| <= 1e-4 * ||A_i,:|| ||X_:,j||
    m, n, l = 513, 3000, 40
    A = _A(m, n)
    X = np.random.default_rng(3).standard_normal((n, l)).astype(np.float32)
    Y = ctx.sketch(_dev_padded(A), torch.from_numpy(X).cuda(), form=2).double().cpu().numpy()
    ref = A.astype(np.float64) @ X.astype(np.float64)
    scale = np.outer(np.linalg.norm(A.astype(np.float64), axis=1), np.linalg.norm(X.astype(np.float64), axis=0))
    assert np.max(np.abs(Y - ref) / scale) < 1e-4


def test_tensor_core_forms_rejected_on_unaligned_lda(ctx):
    import paper_1711_02037_gb300 as pkg
    A = torch.zeros((64, 70), device="cuda")[:, :67]  # lda 70: not a multiple of 4
    X = torch.zeros((67, 8), device="cuda")
    with pytest.raises(pkg.RnmfError) as e:
        ctx.sketch(A, X, form=1)
    assert e.value.status == 1
    ctx.sketch(A, X, form=0)  # the float32 form has no such constraint


@pytest.mark.parametrize("precision", [1, 2])
def test_rnmf_tensor_core_forms_reach_oracle_error(ctx, precision):
    w = synth.SMALL
    A = synth.lowrank(w)
    W, H, st = ctx.rnmf(torch.from_numpy(A).cuda(), w.k, w.p, w.q, w.iters, w.seed, precision=precision,
                        track_every=10)
    ref = R.rhals(A, w.k, w.p, w.q, w.iters, w.seed, track=True)
    assert abs(st.final_rel_err - ref["hist"][-1]) / ref["hist"][-1] < 1e-3
    assert (W >= 0).all() and (H >= 0).all()


def test_rnmf_is_deterministic(ctx):
    w = synth.Workload("t", 2000, 1500, 12, 12, 8, 2, 20, 0.02)
    A = torch.from_numpy(synth.lowrank(w)).cuda()
    for prec in (0, 1):
        W1, H1, _ = ctx.rnmf(A, w.k, w.p, w.q, w.iters, 0, precision=prec)
        W1, H1 = W1.clone(), H1.clone()
        W2, H2, _ = ctx.rnmf(A, w.k, w.p, w.q, w.iters, 0, precision=prec)
        assert torch.equal(W1, W2) and torch.equal(H1, H2)


# Entry-wise forward error bounds: |out - ref| <= c (|A| |X|) entry by entry, with
# c from the operand rounding (bf16 keeps 8 significant bits: each operand within
# 2^-9 relative, a product within about 2^-8; the hi/lo split keeps 16 bits per
# operand and drops lo * lo: about 3 * 2^-17), plus the float32 accumulation.
ENTRY_C = {0: 4e-6, 1: 2.0 ** -8 * 1.01, 2: 3 * 2.0 ** -17}


@pytest.mark.parametrize("form", [0, 1, 2])
@pytest.mark.parametrize("m,n,l", [(1000, 777, 20), (300, 4100, 128), (2000, 130, 70)])
def test_sketch_products_entrywise(ctx, m, n, l, form):
    A = _A(m, n)
    rng = np.random.default_rng(3 * m + n + l)
    A64 = A.astype(np.float64)
    dA = _dev_padded(A)
    for transpose in (False, True):
        X = rng.standard_normal((m if transpose else n, l)).astype(np.float32)
        out = ctx.sketch(dA, torch.from_numpy(X).cuda(), transpose=transpose, form=form).double().cpu().numpy()
        Am = A64.T if transpose else A64
        ref = Am @ X.astype(np.float64)
        bound = np.abs(Am) @ np.abs(X.astype(np.float64))
        K = Am.shape[1]
        slack = ENTRY_C[form] + K * 2.0 ** -23 * (0.0 if form == 0 else 1.0)
        ratio = np.abs(out - ref) / (slack * bound + 1e-300)
        assert ratio.max() <= 1.0, (transpose, float(ratio.max()))


# The float32 CUDA-core products over A with many output rows run on 128 x 64
# output blocks (two per SM) with a split contraction: ragged row, column and
# contraction tails, uneven column blocks (70 columns as two blocks of 48, 128 as
# two of 64), row pitches that are (padded) and are not (n odd) 16-byte aligned.
@pytest.mark.parametrize("m,n,l", [(5003, 4501, 70), (4100, 4097, 128), (6000, 4200, 1)])
@pytest.mark.parametrize("padded", [True, False])
def test_float32_products_large_ragged(ctx, m, n, l, padded):
    A = _A(m, n)
    rng = np.random.default_rng(m + 7 * n + l)
    A64 = A.astype(np.float64)
    dA = _dev_padded(A) if padded else torch.from_numpy(A).cuda()
    for transpose in (False, True):
        X = rng.standard_normal((m if transpose else n, l)).astype(np.float32)
        out = ctx.sketch(dA, torch.from_numpy(X).cuda(), transpose=transpose, form=0).double().cpu().numpy()
        Am = A64.T if transpose else A64
        ref = Am @ X.astype(np.float64)
        bound = np.abs(Am) @ np.abs(X.astype(np.float64))
        ratio = np.abs(out - ref) / (ENTRY_C[0] * bound + 1e-300)
        assert ratio.max() <= 1.0, (transpose, float(ratio.max()))
