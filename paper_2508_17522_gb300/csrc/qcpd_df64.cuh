// Double-float ("df64") arithmetic for the FP32 pipes.
//
// This GPU issues FP64 at 1/74 of its FP32 rate (one warp-wide FP64
// instruction per 19 SM cycles whatever its number of active lanes, and
// conversions between the two formats cost the same), so the cluster
// engine's per-pass arithmetic runs on pairs of binary32 numbers: a value is
// hi + lo with |lo| <= ulp(hi) / 2, about 48 significant bits.  The
// operations are built from two error-free transformations:
//   TwoSum (Knuth): s = fl(a + b) and the exact error e = (a + b) - s from
//     six additions;
//   TwoProduct through a fused multiply-add: p = fl(a b) and the exact error
//     e = fma(a, b, -p).
// Additions and products use the "sloppy" double-float forms (relative error
// a few units of 2^-48 of |a| + |b| or |a b|).  The round-to-nearest
// intrinsics keep the compiler from contracting a product into a following
// sum, which would break the transformations.  The exponent range is
// binary32's; callers keep magnitudes between about 2^-90 and 2^90 (the
// cluster engine scales each system's right-hand side to unit norm and falls
// back to FP64 for data outside that range).
#pragma once

#include <cuda_runtime.h>

namespace qcpd {

using df = float2;  // (hi, lo)

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// |a| >= |b| (or a = 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df df_make(float hi, float lo) { return make_float2(hi, lo); }
__device__ __forceinline__ df df_zero() { return make_float2(0.f, 0.f); }
__device__ __forceinline__ df df_neg(df a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ df df_add(df a, df b) {
    float s, e;
    two_sum(a.x, b.x, s, e);
    e = __fadd_rn(e, __fadd_rn(a.y, b.y));
    float h, l;
    fast_two_sum(s, e, h, l);
    return make_float2(h, l);
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
    float h, l;
    fast_two_sum(p, e, h, l);
    return make_float2(h, l);
}

// a b + c
__device__ __forceinline__ df df_fma(df a, df b, df c) {
    const float p = __fmul_rn(a.x, b.x);
    float pe = fmaf(a.x, b.x, -p);
    pe = fmaf(a.x, b.y, fmaf(a.y, b.x, pe));
    float s, e;
    two_sum(p, c.x, s, e);
    e = __fadd_rn(e, __fadd_rn(pe, c.y));
    float h, l;
    fast_two_sum(s, e, h, l);
    return make_float2(h, l);
}

// A running sum of products kept as an unnormalised pair (S, E): S the
// binary32 sum, E the sum of every rounding error; one TwoProduct, one
// TwoSum and two additions per term, normalised once at the end.
struct DfAcc {
    float S, E;
};

__device__ __forceinline__ DfAcc dfacc_zero() { return DfAcc{0.f, 0.f}; }

__device__ __forceinline__ void dfacc_fma(DfAcc& a, df v, df x) {
    const float p = __fmul_rn(v.x, x.x);
    float pe = fmaf(v.x, x.x, -p);
    pe = fmaf(v.x, x.y, fmaf(v.y, x.x, pe));
    float s, e;
    two_sum(a.S, p, s, e);
    a.S = s;
    a.E = __fadd_rn(a.E, __fadd_rn(e, pe));
}

__device__ __forceinline__ df dfacc_result(DfAcc a) {
    float h, l;
    two_sum(a.S, a.E, h, l);
    return make_float2(h, l);
}

// Conversions (FP64 pipe: keep them out of per-entry loops).
__device__ __forceinline__ df df_from(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ double df_to(df a) { return (double)a.x + (double)a.y; }

__device__ __forceinline__ df warp_sum_df(df v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        df w;
        w.x = __shfl_xor_sync(0xffffffffu, v.x, o);
        w.y = __shfl_xor_sync(0xffffffffu, v.y, o);
        v = df_add(v, w);
    }
    return v;
}

}  // namespace qcpd
