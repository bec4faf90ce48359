// Double-word ("double-float") arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, about 48 significant
// bits.  On GB300 an FP64 warp instruction occupies the FP64 pipe for 64
// cycles whatever the number of active lanes, while FP32 instructions issue
// every cycle or two; latency-bound serial FP64 code (the QR iteration of the
// small projected problem) runs several times faster in double-word form.
//
// The building blocks are the error-free transformations of Knuth (TwoSum),
// Dekker (Fast2Sum) and the FMA-based exact product, combined as in
// M. Joldes, J.-M. Muller, V. Popescu, "Tight and rigorous error bounds for
// basic building blocks of double-word arithmetic", ACM TOMS 44(2), 2017:
// the accurate double-word sum (relative error a small multiple of u^2), the
// FMA-based double-word product, and Newton-type corrections for the quotient
// and the square root.  u = 2^-24.  Every operation uses the _rn intrinsics
// so that the compiler neither contracts nor reassociates them.
//
// The exponent range is FP32's: callers scale their data by a power of two
// so that the magnitudes of interest stay far from under- and overflow.
#pragma once

#include <cuda_runtime.h>

namespace plhr {

struct __align__(8) dw {   // 8-byte aligned: one 64-bit load or store per value
    float hi, lo;
};

__device__ __forceinline__ dw dw_make(float a) { return {a, 0.0f}; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ dw dw_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// s + e = a + b exactly when |a| >= |b| or a == 0 (Dekker)
__device__ __forceinline__ dw dw_fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

// p + e = a * b exactly (FMA)
__device__ __forceinline__ dw dw_two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return {p, e};
}

__device__ __forceinline__ dw dw_add(dw a, dw b) {
    dw s = dw_two_sum(a.hi, b.hi);
    dw t = dw_two_sum(a.lo, b.lo);
    float c = __fadd_rn(s.lo, t.hi);
    dw v = dw_fast_two_sum(s.hi, c);
    float w = __fadd_rn(t.lo, v.lo);
    return dw_fast_two_sum(v.hi, w);
}

__device__ __forceinline__ dw dw_neg(dw a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dw dw_sub(dw a, dw b) { return dw_add(a, dw_neg(b)); }

__device__ __forceinline__ dw dw_mul(dw a, dw b) {
    dw p = dw_two_prod(a.hi, b.hi);
    float t = __fmul_rn(a.hi, b.lo);
    t = __fmaf_rn(a.lo, b.hi, t);
    float c = __fadd_rn(p.lo, t);
    return dw_fast_two_sum(p.hi, c);
}

// a * b for an FP32 b
__device__ __forceinline__ dw dw_mul_f(dw a, float b) {
    dw p = dw_two_prod(a.hi, b);
    float c = __fmaf_rn(a.lo, b, p.lo);
    return dw_fast_two_sum(p.hi, c);
}

// a / b: q1 = a_hi * rcp(b_hi) with the hardware reciprocal approximation,
// then two corrections with the exact remainder a - q b (each roughly squares
// the relative error: 2^-22 -> 2^-44 -> full double-word precision)
__device__ __forceinline__ dw dw_div(dw a, dw b) {
    const float r = __fdividef(1.0f, b.hi);
    const float q1 = __fmul_rn(a.hi, r);
    dw rem = dw_sub(a, dw_mul_f(b, q1));
    dw q = dw_fast_two_sum(q1, __fmul_rn(rem.hi, r));
    dw rem2 = dw_sub(a, dw_mul(b, q));
    return dw_add(q, dw_make(__fmul_rn(rem2.hi, r)));
}

// sqrt(a), a >= 0: s1 = a_hi * rsqrt(a_hi) (hardware approximation), then two
// Newton corrections s += (a - s^2) / (2 s)
__device__ __forceinline__ dw dw_sqrt(dw a) {
    if (a.hi <= 0.0f) return {0.0f, 0.0f};
    const float rs = rsqrtf(a.hi);
    const float s1 = __fmul_rn(a.hi, rs);
    const float half_inv = __fmul_rn(0.5f, rs);   // ~ 1 / (2 s)
    dw rem = dw_sub(a, dw_two_prod(s1, s1));
    dw s = dw_fast_two_sum(s1, __fmul_rn(rem.hi, half_inv));
    dw rem2 = dw_sub(a, dw_mul(s, s));
    return dw_add(s, dw_make(__fmul_rn(rem2.hi, half_inv)));
}

// a * 2^k for a power of two p = 2^k (exact unless a component leaves the
// FP32 range)
__device__ __forceinline__ dw dw_mul_pow2(dw a, float p) { return {__fmul_rn(a.hi, p), __fmul_rn(a.lo, p)}; }

// 2^-e for the binary exponent e of |x| (x normal: x 2^-e in [1, 2));
// zero and subnormal x give 2^100, which brings any subnormal to about 1
__device__ __forceinline__ float pow2_inverse_of(float x) {
    const int be = (__float_as_int(x) >> 23) & 0xff;   // biased exponent
    if (be == 0) return 0x1p100f;
    const int k = be > 253 ? 253 : be;                // 2^-(k - 127) stays normal
    return __int_as_float((254 - k) << 23);
}

__device__ __forceinline__ float dw_abs_hi(dw a) { return fabsf(a.hi); }
__device__ __forceinline__ bool dw_is_zero(dw a) { return a.hi == 0.0f; }

// conversions (FP64 instructions: use outside inner loops)
__device__ __forceinline__ dw dw_from_double(double d) {
    float hi = __double2float_rn(d);
    float lo = __double2float_rn(d - (double)hi);
    return {hi, lo};
}
__device__ __forceinline__ double dw_to_double(dw a) { return (double)a.hi + (double)a.lo; }
// The same as a call: the rare-input branch of the integer splits below calls
// it, so the compiler keeps that branch instead of evaluating the FP64 route
// for every element
static __device__ __noinline__ dw dw_from_double_call(double d) { return dw_from_double(d); }

// The same split without FP64 instructions (GB300 issues FP64 at 1/64 of the
// FP32 rate), by integer operations on the IEEE-754 encodings: hi is x
// rounded to 24 significant bits (to nearest, ties to even: the 29 discarded
// mantissa bits decide, and an increment of the encoding carries into the
// exponent), lo is the remainder x - hi, an integer of at most 2^28 times
// 2^(e - 52) converted to FP32 (rounded) with its sign.  The pair is the one
// the FP64 route gives, bit for bit, in the fast range.  Zero, values
// below 2^-74 or from 2^127 up, Inf and NaN take the FP64 route.
__device__ __forceinline__ dw dw_from_double_fast(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ffu) - 1023;
    if (e < -74 || e > 126) return dw_from_double_call(x);
    const unsigned sign = (unsigned)(b >> 63) << 31;
    const unsigned long long mant = b & 0xfffffffffffffull;
    const unsigned m29 = (unsigned)(mant & 0x1fffffffu);
    // round to nearest, ties to even (the FP64 route's conversion)
    const unsigned up = (m29 > 0x10000000u) | ((m29 == 0x10000000u) & (unsigned)(mant >> 29) & 1u);
    const float hi = __uint_as_float((sign | ((unsigned)(e + 127) << 23) | (unsigned)(mant >> 29)) + up);
    const float scale = __uint_as_float((unsigned)(e - 52 + 127) << 23);
    const float mag = __fmul_rn(__uint2float_rn(up ? 0x20000000u - m29 : m29), scale);
    return {hi, __uint_as_float(__float_as_uint(mag) ^ (up ? sign ^ 0x80000000u : sign))};
}

// acc += a * b (a, b double-word): exact product of the high parts, FP32
// cross terms, TwoSum on the high part of the accumulator
__device__ __forceinline__ void dw_fma_acc(float& hi, float& lo, const dw& a, const dw& b) {
    const float ph = __fmul_rn(a.hi, b.hi);
    const float pl = __fmaf_rn(a.hi, b.hi, -ph);
    const float cr = __fmaf_rn(a.hi, b.lo, __fmul_rn(a.lo, b.hi));
    const dw s = dw_two_sum(hi, ph);
    hi = s.hi;
    lo = __fadd_rn(lo, __fadd_rn(s.lo, __fadd_rn(pl, cr)));
}

// Lazily normalised double-word sum: the high part takes each term's high
// part through TwoSum (exact), every low-order term (the TwoSum error, the
// product's error and cross terms, the operands' low parts) is added to the
// low part in FP32, and the pair is normalised once at the end.  For the
// handful of terms of a stencil, a transfer or an update it carries about
// 2^-46 of the sum of |terms| (the accurate pairwise sum's error class) in
// half its instructions.
struct dwacc {
    float hi, lo;
};
__device__ __forceinline__ dwacc dwacc_of(dw a) { return {a.hi, a.lo}; }
// s += a
__device__ __forceinline__ void dwacc_add(dwacc& s, dw a) {
    const dw t = dw_two_sum(s.hi, a.hi);
    s.hi = t.hi;
    s.lo = __fadd_rn(s.lo, __fadd_rn(t.lo, a.lo));
}
// s -= a
__device__ __forceinline__ void dwacc_sub(dwacc& s, dw a) { dwacc_add(s, dw_neg(a)); }
// s += a w (w FP32)
__device__ __forceinline__ void dwacc_add_mul_f(dwacc& s, dw a, float w) {
    const float ph = __fmul_rn(a.hi, w);
    const float pl = __fmaf_rn(a.hi, w, -ph);
    const dw t = dw_two_sum(s.hi, ph);
    s.hi = t.hi;
    s.lo = __fadd_rn(s.lo, __fadd_rn(t.lo, __fmaf_rn(a.lo, w, pl)));
}
// s += a b (double-word operands)
__device__ __forceinline__ void dwacc_add_mul(dwacc& s, dw a, dw b) { dw_fma_acc(s.hi, s.lo, a, b); }
__device__ __forceinline__ dw dwacc_result(dwacc s) { return dw_two_sum(s.hi, s.lo); }

// FP64 -> FP32 rounding (to nearest, ties to even: the conversion
// instruction's result) by integer operations on the encodings, for normal
// FP32 results; other inputs take the conversion instruction
__device__ __forceinline__ float f64_to_f32_rn(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ffu) - 1023;
    if (e < -126 || e > 126) return __double2float_rn(x);
    const unsigned long long mant = b & 0xfffffffffffffull;
    const unsigned m29 = (unsigned)(mant & 0x1fffffffu);
    const unsigned up = (m29 > 0x10000000u) | ((m29 == 0x10000000u) & (unsigned)(mant >> 29) & 1u);
    return __uint_as_float(((unsigned)(b >> 63) << 31 | ((unsigned)(e + 127) << 23) | (unsigned)(mant >> 29)) + up);
}

// Truncating form of the same split: hi is x with the 29 low mantissa bits
// cleared, lo the remainder (same sign as x, |lo| < ulp(hi)); x = hi + lo to
// ~2^-48 relative.  Used where only the pair's sum matters (the double-word
// Gram, update and V-cycle), never where hi serves as the FP32 value of x.
__device__ __forceinline__ dw dw_split_trunc(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ffu) - 1023;
    if (e < -74 || e > 127) return dw_from_double_call(x);
    const unsigned sign = (unsigned)(b >> 63) << 31;
    const unsigned long long mant = b & 0xfffffffffffffull;
    const float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)(mant >> 29));
    const float scale = __uint_as_float((unsigned)(e - 52 + 127) << 23);
    const float lo = __fmul_rn(__uint2float_rn((unsigned)(mant & 0x1fffffffu)), scale);
    return {hi, __uint_as_float(__float_as_uint(lo) ^ sign)};
}

// FP32 -> FP64 widening by re-biasing the exponent of the encoding (exact for
// normal numbers and zero); subnormal, Inf and NaN inputs take the conversion
// instruction
__device__ __forceinline__ double f32_to_f64_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    if (e == 0u) return (u & 0x7fffffu) ? (double)f : __longlong_as_double((long long)sign);
    if (e == 0xffu) return (double)f;
    return __longlong_as_double((long long)(sign | ((unsigned long long)(e + 896u) << 52) |
                                            ((unsigned long long)(u & 0x7fffffu) << 29)));
}
// hi + lo with one FP64 addition (the widenings are integer operations)
__device__ __forceinline__ double dw_to_double_fast(dw a) { return f32_to_f64_bits(a.hi) + f32_to_f64_bits(a.lo); }

}  // namespace plhr
