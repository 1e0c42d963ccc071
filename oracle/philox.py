"""Oracle random draws: Philox4x32-10 and the mappings to U[0,1) and N(0,1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Philox4x32-10 is written here, in vectorised numpy, from its published
definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies by 0xD2511F53 and
0xCD9E8D57 with the Weyl key schedule 0x9E3779B9 / 0xBB67AE85.

Counter layout: (lo32(b), hi32(b), stream, instance), key (lo32(seed),
hi32(seed)), b = block index.  Streams: 1 = the test matrix Omega (Section 2.3,
Eq. for Y = A Omega), 2 = W_init, 3 = H_init (Algorithm 1, initialisation),
4 = the visiting order of a shuffled sweep (Section 3.2, the shuffled
alternative to the cyclic update orders).

Mappings (each element is a pure function of its logical row-major index e):
  * uniform float32: block e >> 2, word e & 3, u = (word >> 8) * 2^-24.
  * Gaussian float32: block e >> 1 gives a Box-Muller pair;
    u1 = (bits53(w0, w1) + 0.5) 2^-53, u2 = bits53(w2, w3) 2^-53,
    z0 = sqrt(-2 ln u1) cos(2 pi u2) -> element 2b, z1 = ... sin(...) -> 2b+1,
    evaluated in float64 with our own ln / sin / cos (below) and rounded to
    float32.  bits53(hi, lo) = (hi << 21) | (lo >> 11).
numpy's elementwise +, -, *, /, sqrt are IEEE correctly rounded and never
fused, so these values are reproducible bit for bit by any implementation that
performs the same operations in the same order.
"""
from __future__ import annotations

import numpy as np

STREAM_OMEGA, STREAM_W_INIT, STREAM_H_INIT, STREAM_ORDER = 1, 2, 3, 4

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 over uint32 arrays (broadcast); returns 4 uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint32) for x in (c0, c1, c2, c3))
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    with np.errstate(over="ignore"):
        for _ in range(10):
            p0 = _M0 * c0.astype(np.uint64)
            p1 = _M1 * c2.astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK32).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
            k0 = np.uint32(k0 + _W0)
            k1 = np.uint32(k1 + _W1)
    return c0, c1, c2, c3


def _blocks(nblocks: int, seed: int, stream: int, instance: int):
    b = np.arange(nblocks, dtype=np.uint64)
    lo = (b & _MASK32).astype(np.uint32)
    hi = (b >> np.uint64(32)).astype(np.uint32)
    n = lo.shape[0]
    return philox4x32_10(lo, hi, np.full(n, stream, np.uint32), np.full(n, instance, np.uint32),
                         seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def _bits53(hi, lo):
    return (hi.astype(np.uint64) << np.uint64(21)) | (lo.astype(np.uint64) >> np.uint64(11))


def ln(x: np.ndarray) -> np.ndarray:
    """Natural log for x in (0, 1]: x = 2^e f with f in (sqrt(1/2), sqrt(2)],
    ln f = 2 atanh(s), s = (f-1)/(f+1), atanh series through s^23."""
    x = np.asarray(x, np.float64)
    bits = x.view(np.uint64)
    e = ((bits >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64) - 1023
    f = ((bits & np.uint64(0x000FFFFFFFFFFFFF)) | np.uint64(0x3FF0000000000000)).view(np.float64)
    big = f > 1.4142135623730951
    f = np.where(big, f * 0.5, f)
    e = np.where(big, e + 1, e)
    s = (f - 1.0) / (f + 1.0)
    s2 = s * s
    p = np.full_like(s, 1.0 / 23.0)
    for d in (21.0, 19.0, 17.0, 15.0, 13.0, 11.0, 9.0, 7.0, 5.0, 3.0, 1.0):
        p = p * s2 + 1.0 / d
    return e.astype(np.float64) * 0.6931471805599453 + 2.0 * s * p


def _sincos_small(a):
    """sin a, cos a for a in [0, pi/4]: Taylor polynomials through a^17 and a^18."""
    a2 = a * a
    s = np.full_like(a, -1.0 / 355687428096000.0)
    for c in (1.0 / 1307674368000.0, -1.0 / 6227020800.0, 1.0 / 39916800.0, -1.0 / 362880.0,
              1.0 / 5040.0, -1.0 / 120.0, 1.0 / 6.0):
        s = s * a2 + c
    s = s * a2
    s = a - a * s
    c_ = np.full_like(a, 1.0 / 6402373705728000.0)
    for c in (-1.0 / 20922789888000.0, 1.0 / 87178291200.0, -1.0 / 479001600.0, 1.0 / 3628800.0,
              -1.0 / 40320.0, 1.0 / 720.0, -1.0 / 24.0, 0.5):
        c_ = c_ * a2 + c
    c_ = 1.0 - a2 * c_
    return s, c_


def sincos_2pi(u: np.ndarray):
    """(cos 2 pi u, sin 2 pi u) for u in [0,1): quadrant q = floor(4u), exact
    remainder r, reflection of r > 1/2 to 1 - r, then rotation by q quarter turns."""
    u = np.asarray(u, np.float64)
    t = 4.0 * u
    q = t.astype(np.int64)
    r = t - q.astype(np.float64)
    refl = r > 0.5
    a = np.where(refl, 1.0 - r, r) * 1.5707963267948966
    s0, c0 = _sincos_small(a)
    s = np.where(refl, c0, s0)
    c = np.where(refl, s0, c0)
    q = q & 3
    cos = np.select([q == 0, q == 1, q == 2], [c, -s, -c], s)
    sin = np.select([q == 0, q == 1, q == 2], [s, c, -s], -c)
    return cos, sin


def uniform_f32(count: int, seed: int, stream: int, instance: int = 0) -> np.ndarray:
    """count U[0,1) float32 values (24-bit)."""
    nb = (count + 3) // 4
    w = np.stack(_blocks(nb, seed, stream, instance), axis=1).reshape(-1)[:count]
    return ((w >> np.uint32(8)).astype(np.float64) * 2.0 ** -24).astype(np.float32)


def gaussian_f32(count: int, seed: int, stream: int, instance: int = 0) -> np.ndarray:
    """count N(0,1) float32 values by Box-Muller on Philox pairs."""
    nb = (count + 1) // 2
    w0, w1, w2, w3 = _blocks(nb, seed, stream, instance)
    u1 = (_bits53(w0, w1).astype(np.float64) + 0.5) * 2.0 ** -53
    u2 = _bits53(w2, w3).astype(np.float64) * 2.0 ** -53
    rho = np.sqrt(-2.0 * ln(u1))
    c, s = sincos_2pi(u2)
    z = np.empty(2 * nb, np.float64)
    z[0::2] = rho * c
    z[1::2] = rho * s
    return z[:count].astype(np.float32)


def omega(n: int, l: int, seed: int, dist: int = 0, instance: int = 0) -> np.ndarray:
    """Random test matrix Omega (n x l), Section 2.3 / Algorithm 1: Gaussian
    (dist 0) or uniform on [0,1) (dist 1, the remark on the random test
    matrix in Section 3.2).  Returned as float64 holding float32 values."""
    if dist == 0:
        v = gaussian_f32(n * l, seed, STREAM_OMEGA, instance)
    else:
        v = uniform_f32(n * l, seed, STREAM_OMEGA, instance)
    return v.reshape(n, l).astype(np.float64)


def init_factors(m: int, n: int, k: int, seed: int, instance: int = 0):
    """Nonnegative initial factors (Algorithm 1, initialisation): W_init (m x k)
    and H_init (k x n) uniform on [0,1), float32 values, key seed + 1."""
    W = uniform_f32(m * k, seed + 1, STREAM_W_INIT, instance).reshape(m, k)
    H = uniform_f32(k * n, seed + 1, STREAM_H_INIT, instance).reshape(k, n)
    return W.astype(np.float64), H.astype(np.float64)


def sweep_permutation(k: int, seed: int, t: int) -> np.ndarray:
    """Visiting order of the k components in sweep t of the shuffled update
    order (Section 3.2): u_j = word (j mod 4) of Philox block t ceil(k/4) +
    floor(j/4) (key seed, stream 4), components sorted by (u_j, j) ascending."""
    nb = (k + 3) // 4
    b = np.uint64(t) * np.uint64(nb) + np.arange(nb, dtype=np.uint64)
    lo = (b & _MASK32).astype(np.uint32)
    hi = (b >> np.uint64(32)).astype(np.uint32)
    w = philox4x32_10(lo, hi, np.full(nb, STREAM_ORDER, np.uint32), np.zeros(nb, np.uint32),
                      seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    u = np.stack(w, axis=1).reshape(-1)[:k]
    return np.lexsort((np.arange(k), u))
