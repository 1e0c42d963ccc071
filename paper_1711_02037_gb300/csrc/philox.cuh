// philox.cuh - counter-based random draws on the GPU.
//
// Philox4x32-10 from its published definition (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of
//   (c0, c1, c2, c3) <- (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// with M0 = 0xD2511F53, M1 = 0xCD9E8D57 and the Weyl key increments
// 0x9E3779B9, 0xBB67AE85.  Key (lo32(seed), hi32(seed)); counter
// (lo32(b), hi32(b), stream, instance) for block b.
//
// Mappings, chosen so that every value is reproducible bit for bit by any
// IEEE-754 implementation that performs the same operations in the same order
// (hence the __d*_rn intrinsics: no contraction into FMA):
//   uniform float32: word e&3 of block e>>2, (word >> 8) * 2^-24.
//   Gaussian float32 (Box-Muller): block e>>1; u1 = (bits53(w0,w1) + 1/2) 2^-53,
//     u2 = bits53(w2,w3) 2^-53, rho = sqrt(-2 ln u1); element 2b gets
//     rho cos(2 pi u2), element 2b+1 gets rho sin(2 pi u2), rounded to float32.
//     bits53(hi, lo) = (hi << 21) | (lo >> 11).
//   ln: x = 2^e f, f folded into (sqrt(1/2), sqrt(2)], ln f = 2 atanh(s),
//     s = (f-1)/(f+1), atanh series through s^23 (Horner in s^2).
//   cos/sin(2 pi u): q = floor(4u), r = 4u - q (exact); r > 1/2 reflected to
//     1 - r; Taylor polynomials of sin/cos through degree 17/18 on [0, pi/4];
//     rotation by q quarter turns.
#pragma once
#include <stdint.h>

namespace rnmf_rng {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t lo0 = 0xD2511F53u * c[0];
        uint32_t hi0 = __umulhi(0xD2511F53u, c[0]);
        uint32_t lo1 = 0xCD9E8D57u * c[2];
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]);
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

__device__ __forceinline__ void block(uint64_t seed, uint32_t stream, uint32_t inst, uint64_t b,
                                      uint32_t w[4]) {
    w[0] = (uint32_t)b;
    w[1] = (uint32_t)(b >> 32);
    w[2] = stream;
    w[3] = inst;
    philox4x32_10(w, (uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ __forceinline__ uint64_t bits53(uint32_t hi, uint32_t lo) {
    return ((uint64_t)hi << 21) | (uint64_t)(lo >> 11);
}

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }

__device__ inline double ln_unit(double x) {
    uint64_t u = (uint64_t)__double_as_longlong(x);
    int e = (int)((u >> 52) & 0x7ffu) - 1023;
    double f = __longlong_as_double((long long)((u & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL));
    if (f > 1.4142135623730951) {
        f = dmul(f, 0.5);
        e = e + 1;
    }
    double s = __ddiv_rn(dsub(f, 1.0), dadd(f, 1.0));
    double s2 = dmul(s, s);
    double p = 1.0 / 23.0;
    p = dadd(dmul(p, s2), 1.0 / 21.0);
    p = dadd(dmul(p, s2), 1.0 / 19.0);
    p = dadd(dmul(p, s2), 1.0 / 17.0);
    p = dadd(dmul(p, s2), 1.0 / 15.0);
    p = dadd(dmul(p, s2), 1.0 / 13.0);
    p = dadd(dmul(p, s2), 1.0 / 11.0);
    p = dadd(dmul(p, s2), 1.0 / 9.0);
    p = dadd(dmul(p, s2), 1.0 / 7.0);
    p = dadd(dmul(p, s2), 1.0 / 5.0);
    p = dadd(dmul(p, s2), 1.0 / 3.0);
    p = dadd(dmul(p, s2), 1.0);
    return dadd(dmul((double)e, 0.6931471805599453), dmul(dmul(2.0, s), p));
}

__device__ inline void sincos_small(double a, double* s_out, double* c_out) {
    double a2 = dmul(a, a);
    double s = -1.0 / 355687428096000.0;
    s = dadd(dmul(s, a2), 1.0 / 1307674368000.0);
    s = dsub(dmul(s, a2), 1.0 / 6227020800.0);
    s = dadd(dmul(s, a2), 1.0 / 39916800.0);
    s = dsub(dmul(s, a2), 1.0 / 362880.0);
    s = dadd(dmul(s, a2), 1.0 / 5040.0);
    s = dsub(dmul(s, a2), 1.0 / 120.0);
    s = dadd(dmul(s, a2), 1.0 / 6.0);
    s = dmul(s, a2);
    s = dsub(a, dmul(a, s));
    double c = 1.0 / 6402373705728000.0;
    c = dsub(dmul(c, a2), 1.0 / 20922789888000.0);
    c = dadd(dmul(c, a2), 1.0 / 87178291200.0);
    c = dsub(dmul(c, a2), 1.0 / 479001600.0);
    c = dadd(dmul(c, a2), 1.0 / 3628800.0);
    c = dsub(dmul(c, a2), 1.0 / 40320.0);
    c = dadd(dmul(c, a2), 1.0 / 720.0);
    c = dsub(dmul(c, a2), 1.0 / 24.0);
    c = dadd(dmul(c, a2), 0.5);
    c = dsub(1.0, dmul(a2, c));
    *s_out = s;
    *c_out = c;
}

__device__ inline void sincos_2pi(double u, double* c_out, double* s_out) {
    double t = dmul(4.0, u);
    int q = (int)t;
    double r = dsub(t, (double)q);
    double s, c;
    if (r <= 0.5) {
        sincos_small(dmul(r, 1.5707963267948966), &s, &c);
    } else {
        double cs, cc;
        sincos_small(dmul(dsub(1.0, r), 1.5707963267948966), &cs, &cc);
        s = cc;
        c = cs;
    }
    switch (q & 3) {
        case 0: *c_out = c; *s_out = s; break;
        case 1: *c_out = -s; *s_out = c; break;
        case 2: *c_out = -c; *s_out = -s; break;
        default: *c_out = s; *s_out = -c; break;
    }
}

// Both Gaussian values of Box-Muller pair b.
__device__ __forceinline__ void gauss_pair(uint64_t seed, uint32_t stream, uint32_t inst, uint64_t b,
                                           float* z0, float* z1) {
    uint32_t w[4];
    block(seed, stream, inst, b, w);
    double u1 = dmul(dadd((double)bits53(w[0], w[1]), 0.5), 0x1p-53);
    double u2 = dmul((double)bits53(w[2], w[3]), 0x1p-53);
    double rho = __dsqrt_rn(dmul(-2.0, ln_unit(u1)));
    double c, s;
    sincos_2pi(u2, &c, &s);
    *z0 = __double2float_rn(dmul(rho, c));
    *z1 = __double2float_rn(dmul(rho, s));
}

__device__ __forceinline__ float uniform_at(uint64_t seed, uint32_t stream, uint32_t inst, uint64_t e) {
    uint32_t w[4];
    block(seed, stream, inst, e >> 2, w);
    return (float)(w[e & 3] >> 8) * 0x1p-24f;
}

}  // namespace rnmf_rng
