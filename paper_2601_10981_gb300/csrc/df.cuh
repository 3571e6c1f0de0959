// Double-float ("df") arithmetic on the FP32 pipe.  GB300 issues FP64 arithmetic at 1/64
// of the FP32 rate, so the FP32 mode runs its FP64-accurate reductions (POD Grams, the
// snapshot projections) on pairs of floats: x = hi + lo, about 48 significant bits.
// Conversions move bits with integer instructions and keep the FP64 pipe free.
#pragma once
#include <cuda_runtime.h>

namespace pr {

// float -> double by moving bits (exact; float denormals, |x| < 1.2e-38, read as zero).
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned long long sgn = (unsigned long long)(b >> 31) << 63;
    const unsigned long long ed = (e == 255u) ? 2047ull : (unsigned long long)(e + (1023u - 127u));
    const unsigned long long m = (unsigned long long)(b & 0x7fffffu) << 29;
    return __longlong_as_double(e == 0u ? sgn : (sgn | (ed << 52) | m));
}

// double -> (hi, lo) by moving bits: hi is x truncated to the 24 leading significant
// bits, lo the remaining 29 bits rounded to 24, so |x - hi - lo| <= 2^-48 |x|.  |x| below
// the normal float range (2^-126) reads as zero; |x| >= 2^128, inf and nan become
// (float(x), 0).
__device__ __forceinline__ float2 d2df_bits(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const unsigned sgn = hw & 0x80000000u;
    const unsigned e = (hw >> 20) & 0x7ffu;   // biased exponent: x = 1.m * 2^(e - 1023)
    if (e < 897u) return make_float2(0.0f, 0.0f);
    if (e > 1150u) return make_float2(__double2float_rn(x), 0.0f);
    // float exponent field e - 1023 + 127; mantissa bits 51..29 of the double
    const float hi = __uint_as_float(sgn | ((e - 896u) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
    // mantissa bits 28..0, weight 2^(e - 1075) for bit 0; for e < 949 that power is not a
    // normal float and the scaling takes two steps (2^(e - 1011), then 2^-64)
    const float r = __uint2float_rn(lw & 0x1fffffffu);
    const bool small = e < 949u;
    float lo = r * __uint_as_float(sgn | ((small ? e - 884u : e - 948u) << 23));
    if (small) lo *= 5.421010862427522e-20f;   // 2^-64
    return make_float2(hi, lo);
}

// (sh, sl) += (ah + al)(bh + bl): the exact product of the hi parts (FMA residual), the
// two cross terms, and an error-free TwoSum (Knuth) of sh and the product; the rounding
// errors gather in sl, which the caller folds into an FP64 sum every few dozen terms
// (the al*bl term, 2^-48 of the product, is dropped).
__device__ __forceinline__ void df_mac(float& sh, float& sl, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    const float s = __fadd_rn(sh, p);
    const float v = __fsub_rn(s, sh);
    const float w = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, v)), __fsub_rn(p, v));
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(w, e));
}

// The FP64 value of an unevaluated sum of two floats (exact when their exponents are
// less than 29 apart, else rounded once).
__device__ __forceinline__ double df_to_double(float hi, float lo) { return f2d_bits(hi) + f2d_bits(lo); }

// ---- packed pairs: two floats in one 64-bit register, for the f32x2 instructions of
// sm_100 and later (one issue slot for two lanes' worth of FP32 work).
typedef unsigned long long f2p;
__device__ __forceinline__ f2p pk2(float a, float b) {
    f2p r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 upk2(f2p v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ f2p add2(f2p a, f2p b) {
    f2p d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p sub2(f2p a, f2p b) {
    f2p d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p mul2(f2p a, f2p b) {
    f2p d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p fma2(f2p a, f2p b, f2p c) {
    f2p d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// df_mac on both lanes: (sh, sl) += (ah + al)(bh + bl), with nah = -ah supplied by the
// caller (the product's FMA residual needs -fl(ah bh) without a negation instruction).
// Twelve packed instructions for two multiply-adds.
__device__ __forceinline__ void df_mac2(f2p& sh, f2p& sl, f2p ah, f2p nah, f2p al, f2p bh, f2p bl) {
    const f2p np = mul2(nah, bh);          // -p, p = fl(ah bh)
    f2p e = fma2(ah, bh, np);              // ah bh - p, exact
    e = fma2(ah, bl, e);
    e = fma2(al, bh, e);
    const f2p s = sub2(sh, np);            // TwoSum(sh, p)
    const f2p v = sub2(s, sh);
    const f2p w = sub2(sub2(sh, sub2(s, v)), add2(np, v));
    sh = s;
    sl = add2(sl, add2(w, e));
}
// -x on both lanes (sign bits flipped: exact, no FP instruction)
__device__ __forceinline__ f2p neg2(f2p x) { return x ^ 0x8000000080000000ull; }

// (Ah, Al) += (sh, sl) on both lanes, error-free up to the final renormalisation.
__device__ __forceinline__ void df_add2(f2p& Ah, f2p& Al, f2p sh, f2p sl) {
    const f2p s = add2(Ah, sh);
    const f2p v = sub2(s, Ah);
    const f2p w = add2(sub2(Ah, sub2(s, v)), sub2(sh, v));
    const f2p t = add2(add2(Al, sl), w);
    Ah = add2(s, t);
    Al = sub2(t, sub2(Ah, s));
}

}  // namespace pr
