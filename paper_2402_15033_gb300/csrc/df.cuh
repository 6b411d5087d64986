// Double-float arithmetic on the FP32 pipe for FP64-accurate dot products.
//
// On GB300 the FP64 pipe issues about 2 operations per SM per clock, the FP32
// pipe 128 (measured: 1.19 vs 74 TFLOP/s), so the Gram reductions and block
// updates of the two-stage orthogonalization are carried out on unevaluated
// sums of two FP32 numbers (hi + lo, 48 significant bits):
//
//   split   x (FP64) -> (h, l): h = x truncated to 24 bits, l = the next 29 bits
//           rounded to 24; built from the bit pattern with integer operations
//           (no FP64 instruction).  |x - h - l| <= 2^-47 |x| for 2^-74 <= |x| < 2^128;
//           smaller magnitudes keep h only (absolute error < 2^-98), larger ones
//           overflow to infinity; NaN and infinity propagate.
//   product (ah + al)(bh + bl) = p + e exactly up to the al*bl term (< 2^-48):
//           p = ah*bh rounded, e = fma(ah, bh, -p) + ah*bl + al*bh (Dekker 1971,
//           with the fused multiply-add form of the error of a product).
//   sum     (hi, lo) += p + e: Knuth's TwoSum of hi and p, the low parts added,
//           then a fast renormalization (Dekker's FastTwoSum), so |lo| <= ulp(hi)/2
//           and each accumulation step errs by O(2^-48) relative.
//   to FP64 hi + lo assembled into the FP64 bit pattern with integer operations
//           (one rounding, to nearest).
//
// Every FP32 operation uses an explicit _rn intrinsic so the compiler cannot
// contract a product and a sum into an FMA, which would break the error-free
// transformations.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gm {

struct DD {
    float hi, lo;
};

__device__ __forceinline__ void split_f64(double x, float& h, float& l) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sgn = (unsigned)(b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7FF);                 // biased FP64 exponent
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;     // 52 fraction bits
    if (e == 0x7FF) {                                        // Inf or NaN
        h = __uint_as_float(sgn | 0x7F800000u | (m ? 0x400000u : 0u));
        l = 0.f;
        return;
    }
    const int eh = e - 1023 + 127;                           // FP32 biased exponent of h
    if (e == 0 || eh <= 0) {                                 // zero, FP64 subnormal or below FP32 range
        h = __uint_as_float(sgn);
        l = 0.f;
        return;
    }
    if (eh >= 255) {                                         // beyond FP32 range
        h = __uint_as_float(sgn | 0x7F800000u);
        l = 0.f;
        return;
    }
    h = __uint_as_float(sgn | ((unsigned)eh << 23) | (unsigned)(m >> 29));
    const unsigned r = (unsigned)(m & 0x1FFFFFFFull);        // the next 29 fraction bits
    const int el = e - 948;                                  // FP32 biased exponent of 2^(E-52)
    if (r == 0 || el <= 0) {
        l = __uint_as_float(sgn);
        return;
    }
    l = __fmul_rn(__uint2float_rn(r), __uint_as_float((unsigned)el << 23));
    l = __uint_as_float(__float_as_uint(l) | sgn);
}

__device__ __forceinline__ void split_val(double x, float& h, float& l) { split_f64(x, h, l); }
__device__ __forceinline__ void split_val(float x, float& h, float& l) { h = x; l = 0.f; }

// (hi, lo) += (ah + al) * (bh + bl)
__device__ __forceinline__ void dd_mac(DD& a, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    const float s = __fadd_rn(a.hi, p);
    const float v = __fsub_rn(s, a.hi);
    float t = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(p, v));
    t = __fadd_rn(t, __fadd_rn(a.lo, e));
    a.hi = __fadd_rn(s, t);
    a.lo = __fsub_rn(t, __fsub_rn(a.hi, s));
}

// (hi, lo) += x * (bh + bl) for an FP32 x (no low part)
__device__ __forceinline__ void dd_mac1(DD& a, float x, float bh, float bl) {
    const float p = __fmul_rn(x, bh);
    float e = __fmaf_rn(x, bh, -p);
    e = __fmaf_rn(x, bl, e);
    const float s = __fadd_rn(a.hi, p);
    const float v = __fsub_rn(s, a.hi);
    float t = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(p, v));
    t = __fadd_rn(t, __fadd_rn(a.lo, e));
    a.hi = __fadd_rn(s, t);
    a.lo = __fsub_rn(t, __fsub_rn(a.hi, s));
}

// FP64 value of hi + lo (|lo| <= ulp(hi)/2 after dd_mac), integer assembly,
// rounded to nearest even.
__device__ __forceinline__ double dd_to_double(float hi, float lo) {
    const unsigned bh = __float_as_uint(hi);
    const int eh = (int)((bh >> 23) & 0xFF);
    if (eh == 0xFF) return (double)hi;                        // Inf / NaN (rare path)
    if (eh == 0) {
        // hi is zero (the accumulators never hold FP32 subnormals in range)
        const unsigned bl = __float_as_uint(lo);
        const int el = (int)((bl >> 23) & 0xFF);
        if (el == 0) return 0.0;
        const unsigned long long d = ((unsigned long long)(bl >> 31) << 63) |
                                     ((unsigned long long)(el - 127 + 1023) << 52) |
                                     ((unsigned long long)(bl & 0x7FFFFFu) << 29);
        return __longlong_as_double((long long)d);
    }
    // hi = +-H * 2^(Eh-52) with H = (1.f) << 29 (53-bit), Eh = eh - 127
    long long H = (long long)((bh & 0x7FFFFFu) | 0x800000u) << 29;
    if (bh >> 31) H = -H;
    const unsigned bl = __float_as_uint(lo);
    const int el = (int)((bl >> 23) & 0xFF);
    long long S = H;
    if (el != 0) {
        // lo = +-L * 2^(El-23), L 24-bit; in units of 2^(Eh-52): shift = El - Eh + 29
        long long L = (long long)((bl & 0x7FFFFFu) | 0x800000u);
        const int sh = el - eh + 29;
        if (sh >= 0) L <<= sh; else L = sh > -40 ? (L >> (-sh)) : 0;   // |lo| <= ulp(hi)/2: sh <= 5
        S += (bl >> 31) ? -L : L;
    }
    const unsigned long long sgn = S < 0 ? (1ull << 63) : 0ull;
    unsigned long long M = (unsigned long long)(S < 0 ? -S : S);
    if (M == 0) return 0.0;
    // normalize to 53 significant bits: the leading one at bit 52
    const int lz = __clzll((long long)M);                    // 63 - position of the leading one
    int E = eh - 127 + 1023 + (11 - lz);                      // biased FP64 exponent
    if (lz < 11) {
        const int r = 11 - lz;                                // drop r bits, round to nearest even
        const unsigned long long half = 1ull << (r - 1);
        const unsigned long long rem = M & ((1ull << r) - 1);
        M >>= r;
        if (rem > half || (rem == half && (M & 1))) ++M;
        if (M >> 53) { M >>= 1; ++E; }
    } else {
        M <<= (lz - 11);
    }
    const unsigned long long d = sgn | ((unsigned long long)E << 52) | (M & 0xFFFFFFFFFFFFFull);
    return __longlong_as_double((long long)d);
}

__device__ __forceinline__ double dd_value(const DD& a) { return dd_to_double(a.hi, a.lo); }

template <typename T> __device__ __forceinline__ T dd_store(const DD& a);
template <> __device__ __forceinline__ double dd_store<double>(const DD& a) { return dd_to_double(a.hi, a.lo); }
template <> __device__ __forceinline__ float dd_store<float>(const DD& a) { return __fadd_rn(a.hi, a.lo); }

}  // namespace gm
