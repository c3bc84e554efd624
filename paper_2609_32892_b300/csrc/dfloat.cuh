// Compensated single-precision sums ("double-float": an unevaluated sum
// hi + lo of two floats, about 48 significant bits).
//
// The reductions of the TO step add up FP32 block partials.  On this GPU a
// double-precision add issues at about 1/64 of the single-precision rate, so
// long FP64 chains (warp trees over dozens of values, sums over a thousand
// partials) cost far more than the arithmetic they do.  Knuth's TwoSum gives
// the exact rounding error of a float add with six float operations; carrying
// it keeps the sum accurate to well below the rounding of the FP32 partials
// themselves, and the result is widened to double once at the end.
#pragma once

namespace lbm {

struct DF {
    float hi, lo;
};

// s + e == a + b exactly (TwoSum; no assumption on |a| vs |b|)
__device__ __forceinline__ DF df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    const DF s = df_two_sum(a.hi, b.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s.hi, e);
    return {hi, __fsub_rn(e, __fsub_rn(hi, s.hi))};
}

__device__ __forceinline__ DF df_add(DF a, float b) {
    const DF s = df_two_sum(a.hi, b);
    const float e = __fadd_rn(s.lo, a.lo);
    const float hi = __fadd_rn(s.hi, e);
    return {hi, __fsub_rn(e, __fsub_rn(hi, s.hi))};
}

__device__ __forceinline__ DF df_shfl_down(DF a, int o) {
    return {__shfl_down_sync(0xffffffffu, a.hi, o), __shfl_down_sync(0xffffffffu, a.lo, o)};
}

// sum of x[i * stride], i = lane, lane + 32, ... < n over one warp; every lane
// returns the total (as a double) when all 32 lanes call it
__device__ __forceinline__ double df_warp_sum(const float* x, int n, size_t stride, int lane) {
    DF a = {0.f, 0.f};
    for (int i = lane; i < n; i += 32) a = df_add(a, x[(size_t)i * stride]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = df_add(a, df_shfl_down(a, o));
    a.hi = __shfl_sync(0xffffffffu, a.hi, 0);
    a.lo = __shfl_sync(0xffffffffu, a.lo, 0);
    return (double)a.hi + (double)a.lo;
}

}  // namespace lbm
