// df.cuh - double-float arithmetic: a value is the unevaluated sum hi + lo of
// two float32 numbers (|lo| <= ulp(hi) / 2), about 48 significant bits.
//
// Float64 arithmetic runs at a small fraction of the float32 rate on this GPU,
// so the small dense factorisations keep float64-class accuracy on the float32
// pipe.  The error-free steps are Knuth's two-sum, Dekker's fast two-sum and
// the FMA product error p - a b = fma(a, b, -p); the operations are the
// standard ones of Dekker (1971) and of the double-double libraries (Hida, Li,
// Bailey 2001) restated for float32.  Every rounding step goes through an
// explicitly rounded intrinsic so that the compiler cannot contract a product
// into a later sum (which would break the error-free transformations).
#pragma once

#ifdef __CUDA_ARCH__
#define DF_ADD(a, b) __fadd_rn((a), (b))
#define DF_SUB(a, b) __fsub_rn((a), (b))
#define DF_MUL(a, b) __fmul_rn((a), (b))
#define DF_FMA(a, b, c) __fmaf_rn((a), (b), (c))
#else
#include <cmath>
#define DF_ADD(a, b) ((a) + (b))
#define DF_SUB(a, b) ((a) - (b))
#define DF_MUL(a, b) ((a) * (b))
#define DF_FMA(a, b, c) std::fmaf((a), (b), (c))
#endif

struct dfloat {
    float hi, lo;
};

__host__ __device__ __forceinline__ dfloat df_make(float hi, float lo) {
    dfloat r;
    r.hi = hi;
    r.lo = lo;
    return r;
}
// s + e = a + b exactly, |a| >= |b| (or a == 0)
__host__ __device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
    const float s = DF_ADD(a, b);
    return df_make(s, DF_SUB(b, DF_SUB(s, a)));
}
// s + e = a + b exactly
__host__ __device__ __forceinline__ dfloat df_two_sum(float a, float b) {
    const float s = DF_ADD(a, b);
    const float bb = DF_SUB(s, a);
    return df_make(s, DF_ADD(DF_SUB(a, DF_SUB(s, bb)), DF_SUB(b, bb)));
}
__host__ __device__ __forceinline__ dfloat df_neg(dfloat x) { return df_make(-x.hi, -x.lo); }
// x + y with the low parts added once (relative error a few 2^-48)
__host__ __device__ __forceinline__ dfloat df_add(dfloat x, dfloat y) {
    dfloat s = df_two_sum(x.hi, y.hi);
    s.lo = DF_ADD(s.lo, DF_ADD(x.lo, y.lo));
    return df_fast_two_sum(s.hi, s.lo);
}
__host__ __device__ __forceinline__ dfloat df_sub(dfloat x, dfloat y) { return df_add(x, df_neg(y)); }
// x y (the lo * lo term is below the result's precision)
__host__ __device__ __forceinline__ dfloat df_mul(dfloat x, dfloat y) {
    const float p = DF_MUL(x.hi, y.hi);
    float e = DF_FMA(x.hi, y.hi, -p);
    e = DF_FMA(x.hi, y.lo, e);
    e = DF_FMA(x.lo, y.hi, e);
    return df_fast_two_sum(p, e);
}
// c - a b
__host__ __device__ __forceinline__ dfloat df_fms(dfloat c, dfloat a, dfloat b) { return df_sub(c, df_mul(a, b)); }
// 1 / x: the float32 reciprocal refined by one Newton step r + r (1 - x r)
__host__ __device__ __forceinline__ dfloat df_recip(dfloat x) {
    const float r = 1.0f / x.hi;
    const dfloat e = df_sub(df_make(1.0f, 0.0f), df_mul(x, df_make(r, 0.0f)));
    return df_fast_two_sum(r, DF_MUL(r, e.hi));
}
// sqrt(x), x > 0: the float32 root refined by one Newton step s + (x - s^2) / (2 s)
__host__ __device__ __forceinline__ dfloat df_sqrt(dfloat x) {
    const float s = sqrtf(x.hi);
    const float p = DF_MUL(s, s);
    const dfloat r = df_sub(x, df_make(p, DF_FMA(s, s, -p)));
    return df_fast_two_sum(s, r.hi / DF_ADD(s, s));
}
__host__ __device__ __forceinline__ float df_to_float(dfloat x) { return DF_ADD(x.hi, x.lo); }
