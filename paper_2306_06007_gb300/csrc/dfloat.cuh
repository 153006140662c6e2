// Double-float arithmetic on the FP32 pipes: a value is an unevaluated pair of floats
// hi + lo (~48 significant bits; Dekker 1971, products by FMA). Shared by the double-float
// FFT (k_dffft.cu) and the double-float gathers of FP64 NUFFT sub-problems (k_nufft.cu).
// Every operation is written with explicit round-to-nearest intrinsics, so the compiler
// contracts nothing.
#pragma once

#include <cuda_runtime.h>

namespace hvox {
namespace df {

struct DF {
    float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// Double-float sum: an exact TwoSum of the high parts, the low parts added in FP32, then
// renormalised (the "sloppy" sum of Dekker 1971 / QD). Its error is bounded by ~2^-47 of
// |a| + |b|, the norm-wise bound an FFT or a windowed sum needs (an exactly-rounded sum
// would cost twice the instructions).
__device__ __forceinline__ DF dadd(DF a, DF b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    fast_two_sum(s, e, s, e);
    return {s, e};
}

// The same sum without its renormalisation, for a value that only feeds further sums or
// products: the pair (s, e) is not normalised (|e| may exceed ulp(s) / 2 after
// cancellation), but it is within the same ~2^-47 (|a| + |b|) of a + b, and an operation
// that consumes it keeps its norm-wise bound (its hi parts are combined exactly, its lo
// parts in FP32).
__device__ __forceinline__ DF dadd_lazy(DF a, DF b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    return {s, __fadd_rn(e, __fadd_rn(a.l, b.l))};
}

__device__ __forceinline__ DF dneg(DF a) { return {-a.h, -a.l}; }

// a b as an unnormalised pair (p, e): p = fl(a.h b.h), e = the rounding error of p (FMA,
// exact) + the cross terms (a.l b.l, below 2^-46 of the product, is dropped).
__device__ __forceinline__ void dmul_raw(DF a, DF b, float &p, float &e) {
    p = __fmul_rn(a.h, b.h);
    e = __fmaf_rn(a.l, b.h, __fmaf_rn(a.h, b.l, __fmaf_rn(a.h, b.h, -p)));
}

__device__ __forceinline__ DF dmul(DF a, DF b) {
    float p, e, s;
    dmul_raw(a, b, p, e);
    fast_two_sum(p, e, s, e);
    return {s, e};
}

// a b + sg c d for sg = +-1, with one renormalisation (the real or imaginary part of a
// complex product); the lazy form leaves it out, as dadd_lazy does.
__device__ __forceinline__ DF dmul2_lazy(DF a, DF b, DF c, DF d, float sg) {
    float p, e, q, f, s, t;
    dmul_raw(a, b, p, e);
    dmul_raw(c, d, q, f);
    two_sum(p, sg * q, s, t);
    return {s, __fadd_rn(t, __fmaf_rn(sg, f, e))};
}
__device__ __forceinline__ DF dmul2(DF a, DF b, DF c, DF d, float sg) {
    const DF r = dmul2_lazy(a, b, c, d, sg);
    float s, t;
    fast_two_sum(r.h, r.l, s, t);
    return {s, t};
}

// Lazy sum of several double-float terms with one renormalisation at the end: s is the
// exact running sum of the high parts (TwoSum), e collects the low parts and the TwoSum
// errors in FP32 (error ~2^-47 of the sum of magnitudes).
struct DAcc {
    float s, e;
};
__device__ __forceinline__ DAcc acc_of(DF a) { return {a.h, a.l}; }
__device__ __forceinline__ void acc_add(DAcc &a, float p, float e) {
    float s, t;
    two_sum(a.s, p, s, t);
    a.s = s;
    a.e = __fadd_rn(a.e, __fadd_rn(t, e));
}
// a += x y for double-float x, y
__device__ __forceinline__ void acc_fma(DAcc &a, DF x, DF y) {
    float p, e;
    dmul_raw(x, y, p, e);
    acc_add(a, p, e);
}
__device__ __forceinline__ DAcc acc_mul(DF x, DF y) {
    float p, e;
    dmul_raw(x, y, p, e);
    return {p, e};
}
__device__ __forceinline__ DF acc_done(DAcc a) {
    float s, e;
    fast_two_sum(a.s, a.e, s, e);
    return {s, e};
}
// The sum as an unnormalised pair, for a value that feeds a dadd (see dadd_lazy).
__device__ __forceinline__ DF acc_lazy(DAcc a) { return {a.s, a.e}; }

// FP64 <-> double-float by bit manipulation: GB300 issues FP64 instructions (conversions
// included) at 1/64 of its FP32 rate.
// split: hi = x truncated to 24 significant bits (exact), lo = the remaining 29 bits of the
// significand rounded to 24 (one integer-to-float conversion and exact power-of-two
// scales). |x| below 2^-126 flushes to 0, lo below 2^-126 too (|x| < 2^-102 keeps fewer
// bits); |x| >= 2^128 becomes infinite.
__device__ __forceinline__ DF split_bits(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi32 = (unsigned)(b >> 32), lo32 = (unsigned)b;
    const unsigned sign = hi32 & 0x80000000u;
    const int e = (int)((hi32 >> 20) & 0x7FFu) - 896;  // biased float exponent (1023 - 127)
    if (e <= 0) return {0.f, 0.f};
    if (e >= 255) return {__uint_as_float(sign | 0x7F800000u), 0.f};
    const float h = __uint_as_float(sign | ((unsigned)e << 23) | ((hi32 & 0xFFFFFu) << 3) | (lo32 >> 29));
    // lo = r 2^(E - 1075) with E the double's biased exponent = (r 2^-29) 2^(e - 150); the
    // second factor is a normal float (biased exponent e - 23) for e >= 24.
    const float scale = e >= 24 ? __uint_as_float(sign | ((unsigned)(e - 23) << 23)) : 0.f;
    return {h, __fmul_rn(__fmul_rn(__uint2float_rn(lo32 & 0x1FFFFFFFu), 0x1p-29f), scale)};
}

// A float as the double of the same value (exact; subnormal floats, below 2^-126, as 0).
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned ef = (u >> 23) & 0xFFu;
    if (ef == 0) return 0.0;
    const unsigned long long E = ef == 255 ? 2047ull : (unsigned long long)(ef + 896);
    return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) | (E << 52) |
                                            ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

// hi + lo as a double (one FP64 add).
__device__ __forceinline__ double to_double(DF a) { return f2d_bits(a.h) + f2d_bits(a.l); }

}  // namespace df
}  // namespace hvox
