// ef64.cuh -- FP64-accurate arithmetic without the FP64 pipe.
//
// GB300 issues FP64 FMAs at about 1/70 of the FP32 rate, and FP64<->FP32 conversions as
// slowly, so the FP64 hot paths keep their doubles as bit patterns and compute with
//   * exact int64 fixed-point sums (integer pipe), and
//   * double-float pairs (hi + lo, two floats) built from the error-free transforms
//     TwoSum (Knuth, TAOCP vol. 2, 1969), Fast2Sum (Dekker 1971) and FMA-based TwoProd,
//     as used for double-float arithmetic by Dekker (1971) and Bailey's double-double.
// Conversions between IEEE binary64 bit patterns and these forms use integer operations.
// Every function is __host__ __device__ so the host tests can check it against doubles.
#pragma once

#ifndef __CUDACC_RTC__
#include <stdint.h>
#include <string.h>
#include <math.h>
#endif

#ifdef __CUDA_ARCH__
#define EF_HD __host__ __device__ __forceinline__
#else
#define EF_HD inline
#endif

namespace ef {

struct df { float hi, lo; };   // value hi + lo, |lo| <= ulp(hi) (after normalisation)

EF_HD uint32_t f2u(float f) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t u; memcpy(&u, &f, 4); return u;
#endif
}
EF_HD float u2f(uint32_t u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f; memcpy(&f, &u, 4); return f;
#endif
}
EF_HD float fma_(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return fmaf(a, b, c);
#endif
}
EF_HD float add_(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    volatile float s = a + b; return s;
#endif
}
EF_HD float sub_(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    volatile float s = a - b; return s;
#endif
}
EF_HD float mul_(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    volatile float s = a * b; return s;
#endif
}

// ---- error-free transforms -------------------------------------------------------------
// TwoSum: s + e == a + b exactly, s = fl(a + b)
EF_HD df two_sum(float a, float b) {
    float s = add_(a, b);
    float bb = sub_(s, a);
    float e = add_(sub_(a, sub_(s, bb)), sub_(b, bb));
    return {s, e};
}
// Fast2Sum, valid when |a| >= |b| (or a == 0)
EF_HD df fast_two_sum(float a, float b) {
    float s = add_(a, b);
    float e = sub_(b, sub_(s, a));
    return {s, e};
}
// TwoProd: p + e == a * b exactly (barring underflow), p = fl(a * b)
EF_HD df two_prod(float a, float b) {
    float p = mul_(a, b);
    float e = fma_(a, b, -p);
    return {p, e};
}

EF_HD df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    float e = add_(s.lo, add_(a.lo, b.lo));
    return fast_two_sum(s.hi, e);
}
EF_HD df df_neg(df a) { return {-a.hi, -a.lo}; }
EF_HD df df_mul(df a, df b) {
    df p = two_prod(a.hi, b.hi);
    float e = fma_(a.hi, b.lo, fma_(a.lo, b.hi, p.lo));
    return fast_two_sum(p.hi, e);
}
// a * b for a plain float b
EF_HD df df_mulf(df a, float b) {
    df p = two_prod(a.hi, b);
    float e = fma_(a.lo, b, p.lo);
    return fast_two_sum(p.hi, e);
}

// ---- IEEE binary64 bit patterns ----------------------------------------------------------
EF_HD uint64_t d2u(double d) {
#ifdef __CUDA_ARCH__
    return (uint64_t)__double_as_longlong(d);
#else
    uint64_t u; memcpy(&u, &d, 8); return u;
#endif
}
EF_HD double u2d(uint64_t u) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double d; memcpy(&d, &u, 8); return d;
#endif
}

// Biased exponent field of a double (0 for zero/subnormal, 2047 for inf/nan).
EF_HD int exp_field(uint64_t b) { return (int)((b >> 52) & 0x7FF); }

// float with value 2^k for -126 <= k <= 127
EF_HD float pow2f(int k) { return u2f((uint32_t)(k + 127) << 23); }

// exact float of an integer 0 <= v < 2^23 without the (slow) conversion unit
EF_HD float small_u2f(uint32_t v) { return sub_(u2f(0x4B000000u | v), 8388608.0f); }

EF_HD int clz64(uint64_t v) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)v);
#else
    return __builtin_clzll((unsigned long long)v);
#endif
}

// binary64 -> double-float.  hi is x truncated to 24 significant bits, lo the next 23
// bits (|lo| < 2^-23 |hi|), so |x - (hi + lo)| < 2^-46 |x|.  The result is
// scaled by 2^-scale (scale chosen by the caller to keep the exponents in float
// range); values whose scaled magnitude is below 2^-100 become 0, above 2^127 are not
// allowed.
EF_HD df df_from_bits(uint64_t b, int scale) {
    const uint32_t hw = (uint32_t)(b >> 32), lw = (uint32_t)b;
    const int e = (int)((hw >> 20) & 0x7FF) - 1023 - scale;   // unbiased, scaled
    if (((hw >> 20) & 0x7FF) == 0 || e < -100) return {0.0f, 0.0f};
    const uint32_t sign = hw & 0x80000000u;
    // 52-bit fraction f: top 23 bits go to hi, the following 29 bits form lo
    const uint32_t f_top = ((hw & 0xFFFFFu) << 3) | (lw >> 29);              // 23 bits
    const uint32_t f_low = lw & 0x1FFFFFFFu;                                 // 29 bits
    const float hi = u2f(sign | ((uint32_t)(e + 127) << 23) | f_top);
    // lo = f_low * 2^(e - 52): its top 23 bits (bits 6..28) exactly, the last 6 dropped
    // (relative error of the pair below 2^-46)
    const float lo_int = small_u2f(f_low >> 6);
    const int k = e - 46;
    float lo = mul_(lo_int, pow2f(k < -126 ? -126 : k));
    if (k < -126) lo = mul_(lo, pow2f(k + 126 < -126 ? -126 : k + 126));
    if (sign) lo = -lo;
    return {hi, lo};
}

// double-float (scaled by 2^scale) -> binary64 bit pattern, rounded to nearest up to
// the 2^-48 accuracy of the pair.
EF_HD uint64_t bits_from_df(df v, int scale) {
    if (v.hi == 0.0f) return 0ull;
    // renormalise so |lo| <= ulp(hi)/2 and signs are consistent enough
    df n = fast_two_sum(v.hi, v.lo);
    const uint32_t hb = f2u(n.hi);
    const uint32_t sign = hb & 0x80000000u;
    int eh = (int)((hb >> 23) & 0xFF);
    // hi significand as a 64-bit integer with the binary point at bit 60
    int64_t m = (int64_t)((hb & 0x7FFFFFu) | 0x800000u) << 37;               // 24 bits at 60..37
    const uint32_t lb = f2u(n.lo);
    const int el = (int)((lb >> 23) & 0xFF);
    if (el != 0 && n.lo != 0.0f) {
        int64_t ml = (int64_t)((lb & 0x7FFFFFu) | 0x800000u);
        const int sh = 37 - (eh - el);                                        // align to hi
        if (sh >= 0) ml <<= sh; else ml = (-sh < 63) ? (ml >> -sh) : 0;
        if ((lb ^ hb) & 0x80000000u) m -= ml; else m += ml;
    }
    // m > 0 here (|lo| < |hi|/2); normalise the leading bit to 60
    const int lead = 63 - clz64((uint64_t)m);
    int e2 = eh - 127 + (lead - 60) + scale;                                  // unbiased
    // keep 53 bits: shift so the leading bit is at 52, rounding to nearest even
    const int rs = lead - 52;
    uint64_t mant;
    if (rs > 0) {
        uint64_t um = (uint64_t)m;
        uint64_t q = um >> rs, rem = um & ((1ull << rs) - 1), half = 1ull << (rs - 1);
        if (rem > half || (rem == half && (q & 1))) ++q;
        if (q >> 53) { q >>= 1; ++e2; }
        mant = q;
    } else {
        mant = (uint64_t)m << (-rs);
    }
    const int be = e2 + 1023;
    if (be <= 0) return (uint64_t)sign << 32;                                // flush to zero
    if (be >= 2047) return ((uint64_t)sign << 32) | 0x7FF0000000000000ull;
    return ((uint64_t)sign << 32) | ((uint64_t)be << 52) | (mant & 0xFFFFFFFFFFFFFull);
}

// ---- fixed point -----------------------------------------------------------------------
// A vector whose largest biased exponent field is E (all |x| < 2^(E-1022)) is mapped to
// int64 X = x * 2^(FIX_BITS - (E - 1022)), so |X| < 2^FIX_BITS = 2^53: every double of
// the vector keeps its significand down to 2^-53 of the largest one, and the 10 bits above
// leave room for sums of up to 2^9 terms of either sign.
constexpr int FIX_BITS = 53;

// binary64 bits -> fixed point (truncated toward zero).  E: the vector's largest
// exponent field (>= the exponent field of b).
EF_HD int64_t fix_from_bits(uint64_t b, int E) {
    const uint32_t hw = (uint32_t)(b >> 32), lw = (uint32_t)b;
    const int e = (int)((hw >> 20) & 0x7FF);
    // significand with the implicit bit: M < 2^53; x = M 2^(e-1075), X = M >> (E - e)
    const uint64_t M = ((((uint64_t)(hw & 0xFFFFFu)) | 0x100000ull) << 32) | (uint64_t)lw;
    int sh = E - e;
    sh = sh > 63 ? 63 : (sh < 0 ? 0 : sh);
    const uint64_t mag = e == 0 ? 0ull : (M >> sh);
    return (hw & 0x80000000u) ? -(int64_t)mag : (int64_t)mag;
}

// T * 2^k as a binary64 bit pattern, rounded to nearest even (exact int -> double)
EF_HD uint64_t bits_from_int(int64_t T, int k) {
    if (T == 0) return 0ull;
    const uint64_t sign = T < 0 ? (1ull << 63) : 0ull;
    uint64_t a = T < 0 ? (uint64_t)(-T) : (uint64_t)T;
    const int lead = 63 - clz64(a);
    int e2 = lead + k;
    uint64_t mant;
    if (lead > 52) {
        const int rs = lead - 52;
        uint64_t q = a >> rs, rem = a & ((1ull << rs) - 1), half = 1ull << (rs - 1);
        if (rem > half || (rem == half && (q & 1))) ++q;
        if (q >> 53) { q >>= 1; ++e2; }
        mant = q;
    } else {
        mant = a << (52 - lead);
    }
    const int be = e2 + 1023;
    if (be <= 0) return sign;
    if (be >= 2047) return sign | 0x7FF0000000000000ull;
    return sign | ((uint64_t)be << 52) | (mant & 0xFFFFFFFFFFFFFull);
}

// 2^k as a double, exactly (through ldexp outside the normal exponent range); v * pow2d(k)
// then equals ldexp(v, k) with one multiply per use
EF_HD double pow2d(int k) {
    if (k >= -1022 && k <= 1023) return u2d((uint64_t)(k + 1023) << 52);
    return ldexp(1.0, k);
}

// double-float (true value (hi + lo) 2^scale) -> fixed point with unit
// 2^(E - 1022 - FIX_BITS): each float is its 24-bit significand shifted into place with
// 8 guard bits (bits of lo below them dropped), the sum rounded half up, so the result
// is within 1/2 + 2^-8 units of the value.  With |value| < 2^(E - 1022) + one unit the
// result stays within 2^FIX_BITS + 1.
EF_HD int64_t fix_from_df(df v, int E, int scale) {
    constexpr int G = 8;
    const int u = E - 1022 - FIX_BITS - scale;            // unit exponent relative to v
    int64_t s = 0;
    const float f2[2] = {v.hi, v.lo};
    for (int i = 0; i < 2; ++i) {
        const uint32_t b = f2u(f2[i]);
        const int ef = (int)((b >> 23) & 0xFF);
        if (ef == 0) continue;                             // zero (or subnormal: far below the unit)
        const int64_t M = (int64_t)((b & 0x7FFFFFu) | 0x800000u);
        const int sh = ef - 150 - u + G;                   // f = M 2^(ef - 150); in units 2^(u - G)
        int64_t t = sh >= 0 ? (sh > 38 ? (M << 38) : (M << sh)) : (sh < -62 ? 0 : (M >> -sh));
        if (b & 0x80000000u) t = -t;
        s += t;
    }
    return (s + (1ll << (G - 1))) >> G;                   // arithmetic shift: floor(x + 1/2)
}

// fixed point (unit 2^(E - 1022 - FIX_BITS)) times 2^extra -> double-float, scaled by
// 2^-scale.  Exact splitting into 21-bit pieces, then two TwoSums.
EF_HD df df_from_fix(int64_t T, int E, int extra, int scale) {
    if (T == 0) return {0.0f, 0.0f};
    const bool neg = T < 0;
    uint64_t a = neg ? (uint64_t)(-T) : (uint64_t)T;                         // < 2^63
    // pieces of 21 bits: a = p2 2^42 + p1 2^21 + p0, each exactly a float
    const float p2 = small_u2f((uint32_t)(a >> 42));
    const float p1 = small_u2f((uint32_t)((a >> 21) & 0x1FFFFFu));
    const float p0 = small_u2f((uint32_t)(a & 0x1FFFFFu));
    const int u = E - 1022 - FIX_BITS + extra - scale;                      // value of 1 unit
    // scale each piece by its power of two (exact unless it leaves float range)
    auto sc = [](float v, int k) -> float {
        if (k > 127) return mul_(mul_(v, pow2f(127)), pow2f(k - 127));
        if (k < -126) return mul_(mul_(v, pow2f(-126)), pow2f(k + 126 < -126 ? -126 : k + 126));
        return mul_(v, pow2f(k));
    };
    df s = fast_two_sum(sc(p2, u + 42), sc(p1, u + 21));
    df r = df_add(s, {sc(p0, u), 0.0f});
    return neg ? df_neg(r) : r;
}

}  // namespace ef
