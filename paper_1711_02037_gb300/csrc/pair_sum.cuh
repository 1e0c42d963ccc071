// pair_sum.cuh - sums kept off the float64 pipe.
//
// Float64 arithmetic runs at a small fraction of the float32 rate on this GPU,
// so long fixed-order sums of float32 terms are kept as an unevaluated pair
// (s, c): s the rounded running sum, c the sum of the rounding errors, each
// error exact by Knuth's two-sum.  The pair carries about twice float32's
// precision; a sum in a fixed order is bit-identical from run to run.
#pragma once

__device__ __forceinline__ void two_sum_add(float2& a, float x) {
    const float t = __fadd_rn(a.x, x);  // explicitly rounded: never contracted with a product
    const float bp = __fsub_rn(t, a.x);
    a.y += __fadd_rn(__fsub_rn(a.x, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    a.x = t;
}
__device__ __forceinline__ float2 pair_add(float2 a, float2 b) {
    two_sum_add(a, b.x);
    a.y += b.y;
    return a;
}
__device__ __forceinline__ float pair_value(float2 a) { return a.x + a.y; }
