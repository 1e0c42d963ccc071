"""QB with A in host memory, read in column blocks (Algorithm 2), against the
float64 oracle (oracle.extras.rqb_blocked / rhals_blocked).

Tolerances: Q^T Q = I to 5e-6 (float32 CholeskyQR2); B^T = A^T Q checked in
float64 to 1e-5 relative; the approximation Q B of A within 1e-5 (relative to
||A||) of the oracle's when there are no power iterations (both are the
projection onto span(A Omega)), and its error within 1e-3 relative of the
oracle's with power iterations (the trailing directions are noise, computed
differently in float32); a full solve's final relative error within 1e-3 of
the oracle's.  Block widths: 1, multiples of 4, ragged, and wider than A.
The tensor-core forms (BF16 power passes, or every product in the 3-term
split) take the same checks with B^T = A^T Q to 1e-4 (the split keeps 16
significant bits of each operand); the range's residual within 1e-3 of the
oracle's for the split and within 1e-2 for BF16 power passes (operands rounded
to 8 significant bits, 2^-9 relative, move the trailing noise directions of
this small sketch); blocks whose width is not a multiple of 4 floats fall back
to the CUDA cores.
"""
import numpy as np
import pytest

import synth
from oracle import extras as X
from oracle import philox
from oracle import rhals as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

W = synth.Workload("streamed", 900, 500, 10, 10, 10, 2, 60, 0.01)


@pytest.fixture(scope="module")
def ctx():
    import paper_1711_02037_gb300 as pkg
    c = pkg.Context(0)
    yield c
    c.close()


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


@pytest.fixture(scope="module")
def A():
    return synth.lowrank(W)


@pytest.mark.parametrize("q", [0, 2])
@pytest.mark.parametrize("bc", [1, 36, 37, 128, 4000])
def test_qb_streamed(ctx, A, q, bc):
    A64 = A.astype(np.float64)
    Qg, Btg = ctx.qb_streamed(A, W.l, q, seed=0, block_cols=bc)
    Qg, Bg = host(Qg), host(Btg).T
    assert np.abs(Qg.T @ Qg - np.eye(W.l)).max() < 5e-6
    assert np.linalg.norm(Bg - Qg.T @ A64) <= 1e-5 * np.linalg.norm(Bg)
    Qo, Bo = X.rqb_blocked(A64, philox.omega(W.n, W.l, 0), q, bc)
    nA = np.linalg.norm(A64)
    if q == 0:
        assert np.linalg.norm(Qg @ Bg - Qo @ Bo) <= 1e-5 * nA
    eg, eo = np.linalg.norm(A64 - Qg @ Bg), np.linalg.norm(A64 - Qo @ Bo)
    assert abs(eg - eo) <= 1e-3 * eo


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("bc", [36, 37, 128, 4000])
def test_qb_streamed_tensor_cores(ctx, A, precision, bc):
    A64 = A.astype(np.float64)
    q = 2
    Qg, Btg = ctx.qb_streamed(A, W.l, q, seed=0, block_cols=bc, precision=precision)
    Qg, Bg = host(Qg), host(Btg).T
    assert np.abs(Qg.T @ Qg - np.eye(W.l)).max() < 5e-6
    assert np.linalg.norm(Bg - Qg.T @ A64) <= 1e-4 * np.linalg.norm(Bg)
    Qo, Bo = X.rqb_blocked(A64, philox.omega(W.n, W.l, 0), q, bc)
    eg, eo = np.linalg.norm(A64 - Qg @ (Qg.T @ A64)), np.linalg.norm(A64 - Qo @ Bo)
    assert abs(eg - eo) <= (1e-2 if precision == 1 else 1e-3) * eo


def test_streamed_solve_tensor_cores_matches_oracle(ctx, A):
    Wd, Hd, st = ctx.rnmf_streamed(A, W.k, W.p, W.q, W.iters, seed=0, block_cols=100, precision=2)
    Wg, Hg = host(Wd), host(Hd)
    assert np.all(Wg >= 0) and np.all(Hg >= 0)
    A64 = A.astype(np.float64)
    eg = np.linalg.norm(A64 - Wg @ Hg) / np.linalg.norm(A64)
    eo = X.rhals_blocked(A64, W.k, W.p, W.q, W.iters, 0, 100)["hist"][-1]
    assert abs(eg - eo) <= 1e-3 * eo, (eg, eo)


def test_pinned_and_pageable_host_memory_agree(ctx, A):
    pinned = torch.from_numpy(A).pin_memory()
    Q1, B1 = ctx.qb_streamed(pinned, W.l, 1, block_cols=64)
    Q2, B2 = ctx.qb_streamed(A, W.l, 1, block_cols=64)
    torch.cuda.synchronize()
    assert torch.equal(Q1, Q2) and torch.equal(B1, B2)


def test_streamed_solve_matches_oracle(ctx, A):
    Wd, Hd, st = ctx.rnmf_streamed(A, W.k, W.p, W.q, W.iters, seed=0, block_cols=100)
    Wg, Hg = host(Wd), host(Hd)
    assert np.all(Wg >= 0) and np.all(Hg >= 0)
    A64 = A.astype(np.float64)
    eg = np.linalg.norm(A64 - Wg @ Hg) / np.linalg.norm(A64)
    ref = X.rhals_blocked(A64, W.k, W.p, W.q, W.iters, 0, 100)
    eo = ref["hist"][-1]
    assert abs(eg - eo) <= 1e-3 * eo, (eg, eo)
    assert st.sweeps_done == W.iters and st.ms_qb > 0


def test_without_power_iterations_equals_in_memory_solve(ctx, A):
    Wd, Hd, _ = ctx.rnmf_streamed(A, W.k, W.p, 0, W.iters, seed=0, block_cols=64)
    Wi, Hi, _ = ctx.rnmf(torch.from_numpy(A).cuda(), W.k, W.p, 0, W.iters, seed=0)
    A64 = A.astype(np.float64)
    e1 = np.linalg.norm(A64 - host(Wd) @ host(Hd))
    e2 = np.linalg.norm(A64 - host(Wi) @ host(Hi))
    assert abs(e1 - e2) <= 1e-3 * e2


def test_rejects_unsupported_options(ctx, A):
    import paper_1711_02037_gb300 as pkg
    with pytest.raises(pkg.RnmfError):
        ctx.rnmf_streamed(A, W.k, W.p, W.q, 5, track_every=1)
    with pytest.raises(pkg.RnmfError):
        ctx.rnmf_streamed(A, W.k, W.p, W.q, 5, precision=3)
