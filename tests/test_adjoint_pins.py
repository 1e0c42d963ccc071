"""Pins of the reference gradient (oracle/adjoint.py) of L = <G, W_T H_T>.

* its forward pass equals the pinned sweep oracle (oracle/rhals.py);
* central finite differences in float64 (h = 1e-6) agree with the reverse-mode
  gradient to 1e-6 relative, on 50 random directions in (A, W_init, H_init) and
  on every entry of W_init and H_init (floored by the difference quotient's own
  rounding error), on the 64 x 32, k = 4, T = 5 instance;
  a direction is rejected when any clamp decision differs at +h or -h (the
  objective is not differentiable across a kink).
"""
import numpy as np
import pytest
import torch

import synth
from oracle import adjoint as AD
from oracle import philox
from oracle import rhals as R

W = synth.ADJOINT_FD


@pytest.fixture(scope="module")
def inst():
    A = synth.lowrank(W).astype(np.float64)
    Q, _ = R.rqb(A, philox.omega(W.n, W.l, W.seed), W.q)
    W0, H0 = philox.init_factors(W.m, W.n, W.k, W.seed)
    G = synth.cotangent(W.m, W.n).astype(np.float64)
    return A, Q, W0, H0, G


def test_forward_matches_sweep_oracle(inst):
    A, Q, W0, H0, G = inst
    for gm in (0, 1):
        B = Q.T @ A
        Wr, Hr, _, _ = R.rhals_sweeps(Q, B, W0, H0, W.iters, gm)
        Wa, Ha, _ = AD.sweeps(torch.tensor(Q), torch.tensor(B), torch.tensor(W0), torch.tensor(H0), W.iters, gm)
        assert np.allclose(Wa.numpy(), Wr, rtol=1e-12, atol=1e-13)
        assert np.allclose(Ha.numpy(), Hr, rtol=1e-12, atol=1e-13)


def _fd(inst, dA, dW, dH, h, gm):
    A, Q, W0, H0, G = inst
    Lp, mp = AD.loss(A + h * dA, Q, W0 + h * dW, H0 + h * dH, G, W.iters, gm, record_masks=True)
    Lm, mm = AD.loss(A - h * dA, Q, W0 - h * dW, H0 - h * dH, G, W.iters, gm, record_masks=True)
    same = len(mp) == len(mm) and all(np.array_equal(a, b) for a, b in zip(mp, mm))
    return (Lp - Lm) / (2 * h), same


@pytest.mark.parametrize("gm", [0, 1])
def test_random_directions(inst, gm):
    A, Q, W0, H0, G = inst
    _, gA, gW, gH = AD.loss_and_grads(A, Q, W0, H0, G, W.iters, gm)
    _, m0 = AD.loss(A, Q, W0, H0, G, W.iters, gm, record_masks=True)
    rng = np.random.default_rng(42)
    used = 0
    for _ in range(50):
        dA, dW, dH = rng.standard_normal(A.shape), rng.standard_normal(W0.shape), rng.standard_normal(H0.shape)
        fd, same = _fd(inst, dA, dW, dH, 1e-6, gm)
        if not same:
            continue
        used += 1
        ad = np.sum(gA * dA) + np.sum(gW * dW) + np.sum(gH * dH)
        assert abs(fd - ad) <= 1e-6 * max(abs(ad), abs(fd), 1e-3), (fd, ad)
    assert used >= 40


def test_every_initial_factor_entry(inst):
    # tolerance: 1e-6 relative, floored by the rounding error of a central
    # difference, ~ 4 eps |L| / h (float64 rounding of L amplified by 1/h)
    A, Q, W0, H0, G = inst
    L, gA, gW, gH = AD.loss_and_grads(A, Q, W0, H0, G, W.iters, 0)
    floor = 4 * np.finfo(np.float64).eps * abs(L) / 1e-6
    checked = 0
    for which, g in (("W", gW), ("H", gH)):
        shape = W0.shape if which == "W" else H0.shape
        for idx in np.ndindex(*shape):
            e = np.zeros(shape)
            e[idx] = 1.0
            dW = e if which == "W" else np.zeros_like(W0)
            dH = e if which == "H" else np.zeros_like(H0)
            fd, same = _fd(inst, np.zeros_like(A), dW, dH, 1e-6, 0)
            if not same:
                continue
            checked += 1
            assert abs(fd - g[idx]) <= max(1e-6 * abs(g[idx]), floor), (which, idx, fd, g[idx])
    assert checked >= 0.9 * (W0.size + H0.size)


def test_gradient_wrt_A_lies_in_range_of_Q(inst):
    # A enters only through B = Q^T A (Q fixed): dL/dA = Q dL/dB, so (I - Q Q^T) dL/dA = 0
    A, Q, W0, H0, G = inst
    _, gA, _, _ = AD.loss_and_grads(A, Q, W0, H0, G, W.iters, 0)
    assert np.linalg.norm(gA - Q @ (Q.T @ gA)) <= 1e-12 * np.linalg.norm(gA)
