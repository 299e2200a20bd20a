// dfloat.cuh -- double-float arithmetic: a value is the unevaluated sum
// hi + lo of two floats (|lo| <= ulp(hi)/2), about 48 significant bits.
//
// GB300 runs FP32 at 69 times its FP64 rate (FFMA 36.7 T/s against DFMA
// 0.6 T/s), so FP64-class transforms are cheaper as double-float on the FP32
// pipe: an addition costs 11 float operations (the error-free sum of the high
// parts, Knuth's TwoSum, plus the low parts, renormalised with the Fast2Sum of
// Dekker), a product 7 (the error-free product of the high parts through one
// fused multiply-add, plus the cross terms).  This "sloppy" addition bounds
// the error by a small multiple of 2^-46 (|a| + |b|), which is what a
// transform's norm-wise error analysis needs; it is not correctly rounded.
// Conversions from and to double use the integer pipe only.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace nm {

struct __align__(8) df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    // from an integer or a float: exact
    __host__ __device__ constexpr df(int v) : hi((float)v), lo(0.0f) {}
    __host__ __device__ constexpr df(float v) : hi(v), lo(0.0f) {}
    // from a double: hi = the double rounded to float, lo = the float nearest
    // to the remainder.  Written in plain arithmetic so that constants fold at
    // compile time; runtime values on the device go through df_from_double
    // (integer pipe) instead, see conv_in.
    __host__ __device__ constexpr df(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
};

__host__ __device__ __forceinline__ df df_quick_two_sum(float a, float b) {
    const float s = a + b;
    return df(s, b - (s - a));
}

__device__ __forceinline__ df operator+(df a, df b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float r = __fadd_rn(s, e);
    return df(r, __fsub_rn(e, __fsub_rn(r, s)));
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
__device__ __forceinline__ df operator*(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float r = __fadd_rn(p, e);
    return df(r, __fsub_rn(e, __fsub_rn(r, p)));
}
__device__ __forceinline__ df& operator+=(df& a, df b) { return a = a + b; }
__device__ __forceinline__ df& operator*=(df& a, df b) { return a = a * b; }

// Integer-pipe conversions.  A finite normal double d = m 2^e (53-bit m):
// hi takes its top 24 bits rounded to nearest (ties away from zero, an
// acceptable rounding for a split), lo the remaining bits as a float (exact
// up to its own rounding).  Subnormal floats are flushed to zero.
__device__ __forceinline__ float f_from_parts(uint32_t sign, int exp2, uint64_t mant, int bits) {
    // value = mant * 2^(exp2), mant < 2^bits; returns it rounded to float
    if (mant == 0) return __uint_as_float(sign);
    const int lz = __clzll((long long)mant) - (64 - bits);   // leading zeros within `bits`
    const int top = bits - lz;                                // position of the leading one + 1
    int sh = top - 24;
    uint64_t m24 = sh > 0 ? (mant + (1ull << (sh - 1))) >> sh : mant << (-sh);
    int e = exp2 + sh + 23;                                   // unbiased exponent of the result
    if (m24 >> 24) { m24 >>= 1; ++e; }                       // rounding carried into a new bit
    if (e < -126) return __uint_as_float(sign);               // below the float normal range
    if (e > 127) return __uint_as_float(sign | 0x7f800000u);
    return __uint_as_float(sign | ((uint32_t)(e + 127) << 23) | ((uint32_t)m24 & 0x7fffffu));
}
__device__ __forceinline__ df df_from_double(double d) {
    const uint64_t u = (uint64_t)__double_as_longlong(d);
    const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
    const int ex = (int)((u >> 52) & 0x7ff);
    if (ex == 0) return df(0.0f, 0.0f);
    if (ex == 0x7ff) return df(__uint_as_float(sign | 0x7f800000u), 0.0f);
    const uint64_t m = (u & 0xfffffffffffffull) | (1ull << 52);   // 53 bits
    const int e = ex - 1075;                                        // d = m 2^e
    const float hi = f_from_parts(sign, e, m, 53);
    // remainder d - hi, exactly, as an integer multiple of 2^e
    const uint64_t hu = (uint64_t)__float_as_uint(hi);
    const int hex = (int)((hu >> 23) & 0xff);
    if (hex == 0) return df(hi, 0.0f);
    const int64_t hm = (int64_t)((hu & 0x7fffffu) | 0x800000u);      // hi = hm 2^(hex-150)
    const int shift = (hex - 150) - e;                               // >= 0: hi's grid is coarser
    const int64_t r = (int64_t)m - (shift < 63 ? (hm << shift) : 0);
    const float lo = r >= 0 ? f_from_parts(sign, e, (uint64_t)r, 53)
                            : f_from_parts(sign ^ 0x80000000u, e, (uint64_t)(-r), 53);
    return df(hi, lo);
}
__device__ __forceinline__ double widen_f(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
    const uint32_t e = (u >> 23) & 0xffu;
    if (e == 0) return __longlong_as_double((long long)sign);       // zero (subnormals flushed)
    const uint64_t ed = e == 0xffu ? 2047ull : (uint64_t)(e + 896u);
    return __longlong_as_double((long long)(sign | (ed << 52) | ((uint64_t)(u & 0x7fffffu) << 29)));
}
// df -> double: the two exact widenings and one FP64 addition
__device__ __forceinline__ double df_to_double(df v) { return widen_f(v.hi) + widen_f(v.lo); }

// Input conversion of the passes: a density or restricted value of type TIN
// to the pass type T.
template <typename T, typename TIN> __device__ __forceinline__ T conv_in(TIN v) { return (T)v; }
template <> __device__ __forceinline__ df conv_in<df, double>(double v) { return df_from_double(v); }

template <typename T> struct is_df { static constexpr bool value = false; };
template <> struct is_df<df> { static constexpr bool value = true; };

// The input (density) type that goes with a pass type: double for df.
template <typename T> struct InOf { using type = T; };
template <> struct InOf<df> { using type = double; };

// Read-only cached load of a pass-type value.
template <typename T> __device__ __forceinline__ T ldg_t(const T* p) { return __ldg(p); }
template <> __device__ __forceinline__ df ldg_t<df>(const df* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return df(v.x, v.y);
}

}  // namespace nm
