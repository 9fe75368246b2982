// Per-pair arithmetic shared by the pair-sum kernels (device code only).
#pragma once

#include <cuda_runtime.h>

namespace gnk {

// ------------------------------------------------------------------ reciprocal
static __device__ __forceinline__ double rcp_seed_f64(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    return y;
}

// 1/x in full FP64 from the hardware seed y0 (relative error below 2^-19):
// with e = 1 - x y0 we have 1/x = y0 / (1 - e) = y0 (1 + e + e^2 + ...), so
// y0 (1 + e + e^2) leaves the relative error e^3 < 2^-57, below half an ulp
// after rounding for all but a vanishing set of inputs.
static __device__ __forceinline__ double recip_f64(double x) {
    const double y0 = rcp_seed_f64(x);
    const double e = fma(-x, y0, 1.0);
    const double t = fma(e, e, e);
    return fma(y0, t, y0);
}

static __device__ __forceinline__ float recip_f32(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ------------------------------------------------------------------ double-float (df32)
// FP64-class Cauchy sums on the FP32 pipe.  A df32 number is an unevaluated
// sum hi + lo of two floats (about 48 significant bits).  Error-free
// transformations (Knuth's TwoSum, Dekker's product via FMA) carry the
// rounding errors of every step; positions are taken relative to the source
// tile's FP64 reference node (each target forms its offset in FP64 once per
// tile), so the difference of two nearby nodes keeps its leading bits.  Per
// pair: ~22 flops for d, 16 for |d|^2, 3 for the reciprocal (one Newton step
// from rcp.approx), 8 for 1/d, 16 for the four weight products and 32 for
// the two compensated accumulations, all on the FP32 pipe.
struct df {
    float h, l;
};

// The _rn intrinsics are never contracted into FMAs by the compiler, which
// the error-free transformations below rely on.
static __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

static __device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// a - b for df32 operands (Bailey's add with a final renormalisation)
static __device__ __forceinline__ df df_sub(float ah, float al, float bh, float bl) {
    float s, e;
    two_sum(ah, -bh, s, e);
    e = __fadd_rn(e, __fsub_rn(al, bl));
    df r;
    fast_two_sum(s, e, r.h, r.l);
    return r;
}

// product of two df32 values, unnormalised (hi = fl(a.h b.h), lo = error + cross terms)
static __device__ __forceinline__ df df_mul(df a, df b) {
    df r;
    r.h = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -r.h);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    r.l = e;
    return r;
}

// acc += p (compensated: the hi sum's rounding error goes to acc.l)
static __device__ __forceinline__ void df_acc(df& acc, df p) {
    float s, e;
    two_sum(acc.h, p.h, s, e);
    acc.h = s;
    acc.l = __fadd_rn(acc.l, __fadd_rn(e, p.l));
}

static __device__ __forceinline__ df df_split(double v) {
    df r;
    r.h = (float)v;
    r.l = (float)(v - (double)r.h);
    return r;
}

// df_split without the FP64 pipe (each conversion there is a 64-cycle
// dependent step on GB300): from the bits of v, hi = v truncated to 24
// significant bits (exact as a float) and lo = the next 23 bits, so
// |v - (hi + lo)| < 2^-46 |v|.  For 2^-80 <= |v| < 2^101; zero, tiny, huge and
// non-finite values take df_split.
// (out of line, so that the compiler branches to it instead of evaluating its
// FP64 conversions beside every fast split)
static __device__ __noinline__ df df_split_slow(double v) { return df_split(v); }

static __device__ __forceinline__ df df_split_fast(double v) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(bits >> 32), lo = (unsigned)bits;
    const unsigned e = (hi >> 20) & 0x7ffu;  // biased exponent
    if (e - 943u > 180u) return df_split_slow(v);
    const unsigned sign = hi & 0x80000000u;
    df r;
    r.h = __uint_as_float(sign | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
    // the low 29 bits of the significand: their top 23 exactly through the 2^23
    // bias, scaled by 2^(e - 1069)
    const float m = __fsub_rn(__uint_as_float(0x4b000000u | ((lo & 0x1fffffffu) >> 6)), 8388608.0f);
    r.l = __uint_as_float(__float_as_uint(__fmul_rn(m, __uint_as_float((e - 942u) << 23))) | sign);
    return r;
}

// ------------------------------------------------------------------ packed double-float
// Two independent double-float values per float2 (lane x, lane y) with the
// sm_100 packed FP32 intrinsics: one instruction issues both lanes, so the
// FP32 pipe rather than instruction issue bounds the kernels.  The _rn forms
// are never contracted.  Subtraction is written as an FMA with -1, which is
// exact and rounds once like a subtraction.
struct df2 {
    float2 h, l;
};

static __device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
static __device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
static __device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
static __device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
static __device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
static __device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }

static __device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
    s = add2(a, b);
    const float2 bb = sub2(s, a);
    e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}

static __device__ __forceinline__ void two_diff2(float2 a, float2 b, float2& s, float2& e) {
    s = sub2(a, b);
    const float2 bb = sub2(s, a);
    e = sub2(sub2(a, sub2(s, bb)), add2(b, bb));
}

// a - b, b the same for both lanes (Bailey's add, renormalised)
static __device__ __forceinline__ df2 df2_sub(float2 ah, float2 al, float2 bh, float2 bl) {
    float2 s, e;
    two_diff2(ah, bh, s, e);
    e = add2(e, sub2(al, bl));
    df2 r;
    r.h = add2(s, e);
    r.l = sub2(e, sub2(r.h, s));
    return r;
}

static __device__ __forceinline__ df2 df2_mul(df2 a, df2 b) {
    df2 r;
    r.h = mul2(a.h, b.h);
    float2 e = fma2(a.h, b.h, neg2(r.h));
    e = fma2(a.h, b.l, e);
    e = fma2(a.l, b.h, e);
    r.l = e;
    return r;
}

static __device__ __forceinline__ void df2_acc(df2& acc, df2 p) {
    float2 s, e;
    two_sum2(acc.h, p.h, s, e);
    acc.h = s;
    acc.l = add2(acc.l, add2(e, p.l));
}

static __device__ __forceinline__ void df2_dec(df2& acc, df2 p) {
    float2 s, e;
    two_diff2(acc.h, p.h, s, e);
    acc.h = s;
    acc.l = sub2(acc.l, sub2(p.l, e));
}

}  // namespace gnk
