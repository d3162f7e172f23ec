// Packed FP32 pairs (f32x2: one instruction, two IEEE operations), and the logarithm of the
// likelihood epilogues on such pairs.  Shared by the tensor-core and the structured Pauli projections.
#pragma once

#include "log_poly.h"
#include <cuda_runtime.h>

namespace qst {

// The pair is packed into a 64-bit register inside the asm (mov.b64 {lo, hi}), so no float2
// is ever reinterpreted through memory.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mov.b64 rc, {%6, %7};\n"
        " fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n add.rn.f32x2 rd, ra, rb;\n"
        " mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n sub.rn.f32x2 rd, ra, rb;\n"
        " mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n mul.rn.f32x2 rd, ra, rb;\n"
        " mov.b64 {%0, %1}, rd;\n}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 splat2(float v) { return make_float2(v, v); }

// Compensated (Kahan) accumulation on a packed pair: sum += c v, with the rounding error of
// every add carried in comp (the sum is sum - comp).  The log-likelihood terms of one setting
// are O(c) far from the posterior, so their plain FP32 sum would lose ~2^-24 of it per add.
__device__ __forceinline__ void kahan_fma2(float2 &sum, float2 &comp, float2 c, float2 v) {
    const float2 y = fma2(c, v, make_float2(-comp.x, -comp.y));
    const float2 t = add2(sum, y);
    comp = sub2(sub2(t, sum), y);
    sum = t;
}

// s + e = a + b exactly (Knuth's two-sum; no assumption on the magnitudes)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Adds one measurement setting's log-likelihood term, (sum - comp) summed over both halves of
// the pair minus `sub`, to the running pair (hi, lo): hi takes the large part exactly (two-sum),
// lo the errors and the small terms.
__device__ __forceinline__ void add_setting(float &hi, float &lo, float2 sum, float2 comp, float sub) {
    float s, e;
    two_sum(sum.x, sum.y, s, e);
    float h, e2;
    two_sum(hi, s, h, e2);
    hi = h;
    lo += (e2 + e) - ((comp.x + comp.y) + sub);
}

// A setting's term in the Poisson likelihood beyond its deviance sum, mu (S - t) / t, from the
// exact pairs S = s_hi + s_lo (the setting's computed sum of q) and t = t_hi + t_lo (the exact
// trace, |t - 1| a few ulps): returned as h + l, h = mu (s_hi - t_hi) rounded and l the rest
// (the product's rounding error, the small parts, and the division by t to first order), so
// that the term keeps FP32 accuracy relative to mu even where S - t is of the order of t (a
// setting whose elements do not exhaust the trials).  mu is exact in FP32.
__device__ __forceinline__ void poisson_setting(float mu, float s_hi, float s_lo, float t_hi, float t_lo, float &h,
                                                float &l) {
    float dh, de;
    two_sum(s_hi, -t_hi, dh, de);             // s_hi - t_hi exactly
    const float dl = de + (s_lo - t_lo);      // with the small parts
    h = mu * dh;
    const float e = (t_hi - 1.0f) + t_lo;     // t - 1 (t_hi - 1 is exact)
    l = (__fmaf_rn(mu, dh, -h) + mu * dl) - h * e;
}

// add_setting for a subtracted term given as a pair (sub_h + sub_l): the large part goes
// through the exact two-sums with the deviance sum and the running hi
__device__ __forceinline__ void add_setting_pair(float &hi, float &lo, float2 sum, float2 comp, float sub_h, float sub_l) {
    float s, e;
    two_sum(sum.x, sum.y, s, e);
    float dd, e1;
    two_sum(s, -sub_h, dd, e1);
    float h, e2;
    two_sum(hi, dd, h, e2);
    hi = h;
    lo += ((e2 + e1) + e) - ((comp.x + comp.y) + sub_l);
}

// qst_log_poly (log_poly.h) on two arguments at once, operation for operation, so each
// result has the same bits as the scalar function; arguments must be positive normal finite
// (the caller checks that separately).
__device__ __forceinline__ float2 log_poly2(float2 x) {
    const int ix0 = __float_as_int(x.x), ix1 = __float_as_int(x.y);
    const int k0 = (ix0 - 0x3f3504f3) >> 23, k1 = (ix1 - 0x3f3504f3) >> 23;
    const float2 m = make_float2(__int_as_float(ix0 - (k0 << 23)), __int_as_float(ix1 - (k1 << 23)));
    const float2 f = add2(m, splat2(-1.0f));
    // k as a float without a conversion instruction: adding k to the bits of 1.5 2^23 gives the
    // float 1.5 2^23 + k (|k| < 2^22), and subtracting 1.5 2^23 leaves k exactly
    const float2 kf = sub2(make_float2(__int_as_float(0x4b400000 + k0), __int_as_float(0x4b400000 + k1)),
                           splat2(12582912.0f));
    float2 q = splat2(-0.08064694682313636f);
    q = fma2(q, f, splat2(0.1291790293475221f));
    q = fma2(q, f, splat2(-0.13072555472249744f));
    q = fma2(q, f, splat2(0.14173450906326862f));
    q = fma2(q, f, splat2(-0.16628919666247013f));
    q = fma2(q, f, splat2(0.20002695649848323f));
    q = fma2(q, f, splat2(-0.25000751231191953f));
    q = fma2(q, f, splat2(0.33333312940994586f));
    q = fma2(q, f, splat2(-0.49999997733204976f));
    const float2 f2 = mul2(f, f);
    const float2 r = fma2(f2, q, fma2(kf, splat2(1.42860677e-06f), f));
    return fma2(kf, splat2(0.693145751953125f), r);
}

}  // namespace qst
