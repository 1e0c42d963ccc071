/*
 * synth.c - seeded synthetic inputs for randomized HALS NMF.
 *
 * This module only MAKES INPUTS: nonnegative low-rank-plus-noise matrices
 * A = W0*H0 + sigma*|z|, the cotangent G of the differentiation workload and
 * the ragged shapes of the batched workload.  It holds none of the method's
 * arithmetic (no sketch, no QR, no HALS step) and is linked by neither the
 * oracle nor the CUDA library: tests and the benchmark call it, then hand the
 * same arrays to both sides.
 *
 * The workload shapes follow the synthetic experiments of Section 4.4
 * ("Computational performance": low-rank matrices with nonnegative entries
 * plus noise).  Everything is a pure function of (key, stream, instance,
 * element index), so results do not depend on the thread count or on the
 * machine: the code is compiled with -ffp-contract=off and uses only
 * correctly rounded IEEE +, -, *, / and sqrt in double precision.
 *
 * Random bits: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), written here from that definition.
 * key = (lo32(seed), hi32(seed)); counter = (lo32(b), hi32(b), stream,
 * instance) for block index b.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SYNTH_STREAM_W0 4u
#define SYNTH_STREAM_H0 5u
#define SYNTH_STREAM_NOISE 6u
#define SYNTH_STREAM_MASK 7u
#define SYNTH_STREAM_G 8u
#define SYNTH_STREAM_SHAPES 9u

/* ---------------------------------------------------------------- Philox */
static inline void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

static inline void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
        mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;  /* Weyl key schedule */
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static inline void block_bits(uint64_t seed, uint32_t stream, uint32_t instance, uint64_t b,
                              uint32_t out[4])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)b, (uint32_t)(b >> 32), stream, instance};
    philox4x32_10(ctr, key, out);
}

/* 53 random bits from two words: (hi << 21) | (lo >> 11). */
static inline uint64_t bits53(uint32_t hi, uint32_t lo)
{
    return ((uint64_t)hi << 21) | (uint64_t)(lo >> 11);
}

/* ------------------------------------------- own ln / sin / cos (double) */
/* ln(x), x in (0, 1]: x = 2^e * f, f folded into (sqrt(1/2), sqrt(2)],
 * ln f = 2 atanh(s), s = (f - 1)/(f + 1), atanh by its odd power series
 * truncated after s^23 (|s| <= 0.1716, truncation < 1e-19). */
static double synth_ln(double x)
{
    uint64_t u;
    memcpy(&u, &x, sizeof u);
    int e = (int)((u >> 52) & 0x7ffu) - 1023;
    uint64_t mu = (u & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL;
    double f;
    memcpy(&f, &mu, sizeof f);
    if (f > 1.4142135623730951) { f = f * 0.5; e = e + 1; }
    double s = (f - 1.0) / (f + 1.0);
    double s2 = s * s;
    double p = 1.0 / 23.0;
    p = p * s2 + 1.0 / 21.0;
    p = p * s2 + 1.0 / 19.0;
    p = p * s2 + 1.0 / 17.0;
    p = p * s2 + 1.0 / 15.0;
    p = p * s2 + 1.0 / 13.0;
    p = p * s2 + 1.0 / 11.0;
    p = p * s2 + 1.0 / 9.0;
    p = p * s2 + 1.0 / 7.0;
    p = p * s2 + 1.0 / 5.0;
    p = p * s2 + 1.0 / 3.0;
    p = p * s2 + 1.0;
    return (double)e * 0.6931471805599453 + 2.0 * s * p;
}

/* sin and cos of a in [0, pi/4] by Taylor polynomials through a^17 / a^18. */
static void synth_sincos_small(double a, double *s_out, double *c_out)
{
    double a2 = a * a;
    double s = -1.0 / 355687428096000.0;          /* -1/17! */
    s = s * a2 + 1.0 / 1307674368000.0;           /* 1/15! */
    s = s * a2 - 1.0 / 6227020800.0;              /* 1/13! */
    s = s * a2 + 1.0 / 39916800.0;                /* 1/11! */
    s = s * a2 - 1.0 / 362880.0;                  /* 1/9!  */
    s = s * a2 + 1.0 / 5040.0;                    /* 1/7!  */
    s = s * a2 - 1.0 / 120.0;                     /* 1/5!  */
    s = s * a2 + 1.0 / 6.0;                       /* 1/3!  */
    s = s * a2;
    s = a - a * s;
    double c = 1.0 / 6402373705728000.0;          /* 1/18! */
    c = c * a2 - 1.0 / 20922789888000.0;          /* 1/16! */
    c = c * a2 + 1.0 / 87178291200.0;             /* 1/14! */
    c = c * a2 - 1.0 / 479001600.0;               /* 1/12! */
    c = c * a2 + 1.0 / 3628800.0;                 /* 1/10! */
    c = c * a2 - 1.0 / 40320.0;                   /* 1/8!  */
    c = c * a2 + 1.0 / 720.0;                     /* 1/6!  */
    c = c * a2 - 1.0 / 24.0;                      /* 1/4!  */
    c = c * a2 + 0.5;                             /* 1/2!  */
    c = 1.0 - a2 * c;
    *s_out = s;
    *c_out = c;
}

/* cos(2 pi u), sin(2 pi u) for u in [0, 1): quadrant from floor(4u), exact
 * remainder, reflection to [0, pi/4], then the quadrant rotation. */
static void synth_sincos_2pi(double u, double *c_out, double *s_out)
{
    double t = 4.0 * u;
    int q = (int)t;
    double r = t - (double)q;
    double s, c;
    if (r <= 0.5) {
        synth_sincos_small(r * 1.5707963267948966, &s, &c);
    } else {
        double cs, cc;
        synth_sincos_small((1.0 - r) * 1.5707963267948966, &cs, &cc);
        s = cc; c = cs;
    }
    switch (q & 3) {
    case 0: *c_out = c;  *s_out = s;  break;
    case 1: *c_out = -s; *s_out = c;  break;
    case 2: *c_out = -c; *s_out = -s; break;
    default: *c_out = s; *s_out = -c; break;
    }
}

/* Box-Muller pair from one Philox block. */
static inline void gauss_pair(const uint32_t w[4], double *z0, double *z1)
{
    double u1 = ((double)bits53(w[0], w[1]) + 0.5) * 0x1p-53;  /* (0,1) */
    double u2 = (double)bits53(w[2], w[3]) * 0x1p-53;          /* [0,1) */
    double rho = sqrt(-2.0 * synth_ln(u1));
    double c, s;
    synth_sincos_2pi(u2, &c, &s);
    *z0 = rho * c;
    *z1 = rho * s;
}

static inline double gauss_at(uint64_t seed, uint32_t stream, uint32_t inst, uint64_t e)
{
    uint32_t w[4];
    block_bits(seed, stream, inst, e >> 1, w);
    double z0, z1;
    gauss_pair(w, &z0, &z1);
    return (e & 1) ? z1 : z0;
}

/* U[0,1) double: element e uses words (0,1) or (2,3) of block e >> 1. */
static inline double unif53_at(uint64_t seed, uint32_t stream, uint32_t inst, uint64_t e)
{
    uint32_t w[4];
    block_bits(seed, stream, inst, e >> 1, w);
    uint64_t b = (e & 1) ? bits53(w[2], w[3]) : bits53(w[0], w[1]);
    return (double)b * 0x1p-53;
}

/* Exponential(1) as -ln(u), u = (bits53 + 1) 2^-53 in (0, 1]. */
static inline double exp1_at(uint64_t seed, uint32_t stream, uint32_t inst, uint64_t e)
{
    uint32_t w[4];
    block_bits(seed, stream, inst, e >> 1, w);
    uint64_t b = (e & 1) ? bits53(w[2], w[3]) : bits53(w[0], w[1]);
    double u = ((double)b + 1.0) * 0x1p-53;
    return -synth_ln(u);
}

static inline uint32_t word_at(uint64_t seed, uint32_t stream, uint32_t inst, uint64_t e)
{
    uint32_t w[4];
    block_bits(seed, stream, inst, e >> 2, w);
    return w[e & 3];
}

/* ------------------------------------------------------------ exports */
void synth_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out)
{
    philox4x32_10(ctr, key, out);
}

double synth_ln_export(double x) { return synth_ln(x); }

void synth_sincos_2pi_export(double u, double *c, double *s) { synth_sincos_2pi(u, c, s); }

/* count standard normals (double), element e from block e >> 1. */
void synth_gaussian_f64(double *out, int64_t count, uint64_t seed, uint32_t stream, uint32_t inst)
{
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < count; ++e) out[e] = gauss_at(seed, stream, inst, (uint64_t)e);
}

/* count standard normals rounded to float. */
void synth_gaussian_f32(float *out, int64_t count, uint64_t seed, uint32_t stream, uint32_t inst)
{
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < count; ++e) out[e] = (float)gauss_at(seed, stream, inst, (uint64_t)e);
}

void synth_uniform_f64(double *out, int64_t count, uint64_t seed, uint32_t stream, uint32_t inst)
{
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < count; ++e) out[e] = unif53_at(seed, stream, inst, (uint64_t)e);
}

/*
 * Generator factors of the low-rank input.
 *   W0 (m x r, row-major): U[0,1) (w0_exp = 0) or Exponential(1) (w0_exp = 1).
 *   H0 (r x n, row-major): U[0,1); each entry set to 0 with probability
 *   h0_zero_frac (mask word < ceil(h0_zero_frac * 2^32)).
 */
void synth_factors(double *W0, double *H0, int64_t m, int64_t n, int r, int w0_exp,
                   double h0_zero_frac, uint64_t seed, uint32_t inst)
{
    uint64_t thr = (uint64_t)ceil(h0_zero_frac * 4294967296.0);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m * (int64_t)r; ++e)
        W0[e] = w0_exp ? exp1_at(seed, SYNTH_STREAM_W0, inst, (uint64_t)e)
                       : unif53_at(seed, SYNTH_STREAM_W0, inst, (uint64_t)e);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < (int64_t)r * n; ++e) {
        double h = unif53_at(seed, SYNTH_STREAM_H0, inst, (uint64_t)e);
        if (thr > 0 && (uint64_t)word_at(seed, SYNTH_STREAM_MASK, inst, (uint64_t)e) < thr) h = 0.0;
        H0[e] = h;
    }
}

/*
 * A (m x n, leading dimension lda >= n, float) with
 *   A_ij = fl32( (sum_{t=0..r-1, ascending} W0_it * H0_tj) + sigma * |z_ij| ),
 * every product and partial sum rounded to double, z_ij ~ N(0,1) from the
 * noise stream at logical element index i*n + j.  Columns n..lda-1 are left
 * untouched.  W0/H0 come from synth_factors with the same arguments.
 */
void synth_lowrank_from_factors(float *A, const double *W0, const double *H0, int64_t m, int64_t n,
                                int64_t lda, int r, double sigma, uint64_t seed, uint32_t inst)
{
    const int64_t JB = 512;
    int64_t nblk = (n + JB - 1) / JB;
#pragma omp parallel
    {
        double acc[512];
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < m; ++i) {
            for (int64_t jb = 0; jb < nblk; ++jb) {
                int64_t j0 = jb * JB;
                int64_t j1 = j0 + JB < n ? j0 + JB : n;
                int64_t len = j1 - j0;
                for (int64_t j = 0; j < len; ++j) acc[j] = 0.0;
                for (int t = 0; t < r; ++t) {
                    double w = W0[i * (int64_t)r + t];
                    const double *h = H0 + (int64_t)t * n + j0;
                    for (int64_t j = 0; j < len; ++j) acc[j] = acc[j] + w * h[j];
                }
                for (int64_t j = 0; j < len; ++j) {
                    double v = acc[j];
                    if (sigma != 0.0)
                        v = v + sigma * fabs(gauss_at(seed, SYNTH_STREAM_NOISE, inst,
                                                      (uint64_t)(i * n + j0 + j)));
                    A[i * lda + j0 + j] = (float)v;
                }
            }
        }
    }
}

/* Uniform integers in [lo, hi] by the widening multiply word * range >> 32. */
void synth_uniform_int(int32_t *out, int64_t count, int32_t lo, int32_t hi, uint64_t seed,
                       uint32_t stream, uint32_t inst)
{
    uint64_t range = (uint64_t)((int64_t)hi - (int64_t)lo + 1);
    for (int64_t e = 0; e < count; ++e) {
        uint32_t w = word_at(seed, stream, inst, (uint64_t)e);
        out[e] = lo + (int32_t)(((uint64_t)w * range) >> 32);
    }
}

int synth_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
