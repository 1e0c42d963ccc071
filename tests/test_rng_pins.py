"""Pins of the oracle's random draws (Philox4x32-10, U[0,1), Box-Muller N(0,1)).

The oracle (oracle/philox.py) and the input generator (synth/synth.c) are two
independent implementations of the same published generator and mappings;
besides agreeing with each other bit for bit, each is checked against what
mathematics fixes: library ln/sin/cos, uniformity and normality tests, the
Box-Muller independence of a pair, and the bijectivity of Philox for a key.
The generator itself is pinned to the published known-answer vectors of
Philox4x32-10 (tests/golden/philox4x32_10_kat.txt).
"""
import math
import os

import numpy as np
import pytest
from scipy import stats

import synth
from oracle import philox


KAT_FILE = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_vectors():
    rows = []
    with open(KAT_FILE) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                w = [int(x, 16) for x in line.split()]
                assert len(w) == 10
                rows.append((w[:4], w[4:6], w[6:]))
    assert len(rows) == 3
    return rows


@pytest.mark.parametrize("row", range(3))
def test_philox_known_answer_vectors(row):
    # Salmon et al. (SC'11) publish known-answer vectors for Philox4x32-10 with
    # their reference implementation: the zero counter and key, the all-ones
    # counter and key, and counter/key words taken from the digits of pi.  A
    # wrong multiplier, a swapped output word or a misplaced key bump changes
    # every output word.
    ctr, key, want = _kat_vectors()[row]
    got_oracle = philox.philox4x32_10(*(np.array([c], dtype=np.uint32) for c in ctr), key[0], key[1])
    assert [int(x[0]) for x in got_oracle] == want
    got_synth = synth.philox4x32_10(np.array(ctr, dtype=np.uint32), np.array(key, dtype=np.uint32))
    assert [int(x) for x in got_synth] == want


def test_philox_two_implementations_agree():
    rng = np.random.default_rng(11)
    for _ in range(200):
        ctr = rng.integers(0, 2**32, 4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2**32, 2, dtype=np.uint64).astype(np.uint32)
        a = synth.philox4x32_10(ctr, key)
        b = philox.philox4x32_10(*(np.array([c]) for c in ctr), int(key[0]), int(key[1]))
        assert [int(x[0]) for x in b] == [int(x) for x in a]


def test_philox_is_a_bijection_on_a_sample():
    # Philox is a keyed bijection of the 128-bit counter space: distinct
    # counters never collide.  With 2^20 counters a 64-bit projection of a
    # random function would collide with probability ~3e-8; a broken round
    # (e.g. a dropped xor) collapses outputs and collides quickly.
    w = philox._blocks(1 << 20, 0, 1, 0)
    v = (w[0].astype(np.uint64) << np.uint64(32)) | w[1].astype(np.uint64)
    assert np.unique(v).size == v.size


def test_philox_counter_stream_and_key_matter():
    a = philox._blocks(4, 0, 1, 0)
    b = philox._blocks(4, 0, 2, 0)
    c = philox._blocks(4, 1, 1, 0)
    d = philox._blocks(4, 0, 1, 1)
    for other in (b, c, d):
        assert not np.array_equal(np.stack(a), np.stack(other))


def test_ln_matches_library_log():
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.random(20000), np.array([1.0, 0.5, 2.0 ** -53, 0.75, 1 - 2.0 ** -53])])
    x = x[x > 0]
    ours = philox.ln(x)
    ref = np.log(x)
    scale = np.maximum(np.abs(ref), 1e-300)
    assert np.max(np.abs(ours - ref) / scale) < 4e-15
    assert philox.ln(np.array([1.0]))[0] == 0.0


def test_sincos_matches_library():
    u = np.concatenate([np.random.default_rng(6).random(20000), np.array([0.0, 0.125, 0.25, 0.5, 0.75])])
    c, s = philox.sincos_2pi(u)
    assert np.max(np.abs(c - np.cos(2 * np.pi * u))) < 2e-15
    assert np.max(np.abs(s - np.sin(2 * np.pi * u))) < 2e-15
    assert c[-5] == 1.0 and s[-5] == 0.0          # u = 0
    assert c[-2] == -1.0 and s[-2] == 0.0         # u = 1/2
    assert c[-3] == 0.0 and s[-3] == 1.0          # u = 1/4 (exact quadrant boundary)


def test_ln_sincos_agree_with_synth_implementation():
    rng = np.random.default_rng(8)
    for x in rng.random(500):
        assert philox.ln(np.array([x]))[0] == synth.ln(x)
        c, s = philox.sincos_2pi(np.array([x]))
        assert (c[0], s[0]) == synth.sincos_2pi(x)


def test_uniform_f32_distribution():
    u = philox.uniform_f32(1 << 20, 3, 2)
    assert u.dtype == np.float32 and u.min() >= 0.0 and u.max() < 1.0
    # 24-bit grid
    assert np.all((u.astype(np.float64) * 2 ** 24) == np.floor(u.astype(np.float64) * 2 ** 24))
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / u.size)


def test_gaussian_f32_distribution_and_pair_independence():
    z = philox.gaussian_f32(1 << 20, 0, 1).astype(np.float64)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / z.size)
    # z0 and z1 of one Box-Muller pair are independent N(0,1): correlation ~ 0
    r = np.corrcoef(z[0::2], z[1::2])[0, 1]
    assert abs(r) < 5 / math.sqrt(z.size / 2)
    # squares of a pair sum to -2 ln u1: chi-square with 2 dof = Exp(1/2)
    assert stats.kstest(z[0::2] ** 2 + z[1::2] ** 2, "expon", args=(0, 2)).pvalue > 1e-4


def test_gaussian_oracle_equals_synth_bitwise():
    a = philox.gaussian_f32(10001, 0, 1)
    b = synth.gaussian(10001, 0, 1, 0, np.float32)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_omega_and_init_layout():
    Om = philox.omega(7, 5, 0)
    flat = philox.gaussian_f32(35, 0, philox.STREAM_OMEGA)
    assert np.array_equal(Om.reshape(-1), flat.astype(np.float64))
    W, H = philox.init_factors(6, 4, 3, 0)
    assert np.array_equal(W.reshape(-1), philox.uniform_f32(18, 1, philox.STREAM_W_INIT).astype(np.float64))
    assert np.array_equal(H.reshape(-1), philox.uniform_f32(12, 1, philox.STREAM_H_INIT).astype(np.float64))
    Ou = philox.omega(7, 5, 0, dist=1)
    assert Ou.min() >= 0 and Ou.max() < 1


@pytest.mark.parametrize("frac", [0.0, 0.3])
def test_synth_mask_fraction(frac):
    w = synth.Workload("t", 10, 20000, 3, 3, 1, 0, 0, 0.0, h0_zero_frac=frac)
    _, H0 = synth.factors(w)
    zf = np.mean(H0 == 0.0)
    assert abs(zf - frac) < 0.01
