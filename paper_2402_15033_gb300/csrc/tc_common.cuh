// Exact integer slicing of FP64 values for the bf16 tensor cores (the
// error-free splitting of Ozaki, Ogita, Oishi and Rump, 2012), shared by the
// tensor-core Gram (gram_tc.cuh) and block update (update_tc.cuh).
//
// A value x is sliced against a common biased exponent eb of its group (a
// chunk column for the Gram, a row for the update), eb >= x's own exponent:
// F = round(|x| 2^(54 - e)) (e = eb - 1023; |F| < 2^55) is written in balanced
// base 256, F = sum_{p=0..6} d_p 256^(6-p), d_1..d_6 in [-128, 127], d_0 in
// [-128, 128], so that x = sum_p d_p 2^(e - 6 - 8p) up to the rounding of F and
// every digit is exact in bf16.  A dot product of two sliced vectors of at most
// 64 terms is 2^(e_x + e_y - 12) sum_{t=0..6} 2^(-8t) I_t with
// I_t = sum_{p+q=t} sum_terms d_p d'_q; every digit product is an integer of
// magnitude <= 2^14 and every partial sum of I_t is at most (t+1) 64 2^14 < 2^24,
// so mma.sync (bf16 inputs, FP32 accumulators) forms each I_t exactly.  Digit
// pairs with p + q > 6 weigh less than 2^-51 of the largest product and are not
// formed.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gm {

constexpr int kTcSlices = 7;                  // balanced base-256 digits
constexpr int kTcWp = 34;                     // 16-byte units per (column, digit half): 32 pairs + 2 pad
constexpr int kTcBadExp = 1 << 20;            // exponent marking a NaN or infinity in the group

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                               uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Biased FP64 exponent field of x.
__device__ __forceinline__ int tc_bexp(double x) { return (__double2hiint(x) >> 20) & 0x7FF; }

// Signed F = round(|x| 2^(54 - e)) * sign(x) for the chunk-column biased
// exponent eb >= the value's own (rounding half up); zero and subnormals give 0.
__device__ __forceinline__ long long tc_fixed(double x, int eb) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const int e = (int)(hi >> 20) & 0x7FF;
    unsigned long long m = ((unsigned long long)((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;
    if (e == 0) m = 0;
    const int d = min(max(eb - e, 0), 63);
    const unsigned long long F = ((m << 2) + ((1ull << d) >> 1)) >> d;
    return (hi >> 31) ? -(long long)F : (long long)F;
}

// FP32 bit patterns of the seven balanced base-256 digits of F (most
// significant first); each bf16 digit is the high half.  Adding 128 at every
// lower digit position makes each byte of the sum the digit plus 128, with the
// carries of the balanced representation; a byte b becomes the float b - 128
// by one byte permute into 1.5 * 2^23 and one exact subtraction.
__device__ __forceinline__ void tc_digits(long long F, uint32_t (&dig)[kTcSlices]) {
    const long long Gv = F + 0x808080808080ll;
    const uint32_t lo = (uint32_t)Gv;
    const uint32_t hi = (uint32_t)((unsigned long long)Gv >> 32);
    const float off = -12583040.0f;              // -(1.5 * 2^23 + 128)
    dig[6] = __float_as_uint(__fadd_rn(__uint_as_float(__byte_perm(lo, 0x4B400000u, 0x7650)), off));
    dig[5] = __float_as_uint(__fadd_rn(__uint_as_float(__byte_perm(lo, 0x4B400000u, 0x7651)), off));
    dig[4] = __float_as_uint(__fadd_rn(__uint_as_float(__byte_perm(lo, 0x4B400000u, 0x7652)), off));
    dig[3] = __float_as_uint(__fadd_rn(__uint_as_float(__byte_perm(lo, 0x4B400000u, 0x7653)), off));
    dig[2] = __float_as_uint(__fadd_rn(__uint_as_float(__byte_perm(hi, 0x4B400000u, 0x7650)), off));
    dig[1] = __float_as_uint(__fadd_rn(__uint_as_float(__byte_perm(hi, 0x4B400000u, 0x7651)), off));
    dig[0] = __float_as_uint(__fadd_rn(__int_as_float(0x4B400000 + ((int)hi >> 16)), -12582912.0f));
}

__device__ __forceinline__ double tc_pow2(int e) {   // e in [-1022, 1023]
    return __longlong_as_double((long long)(e + 1023) << 52);
}

// S = sum_t I_t 2^(8(5-t)) for t <= 4, plus I_5 + I_6 / 256 rounded (0.75 units
// at most: the tail weighs 2^-40 of I_0 and the fold is one FP32 rounding),
// from the seven exact accumulators; |S| < 2^61 for sums of at most 64 terms.
__device__ __forceinline__ long long tc_combine(float a0, float a1, float a2, float a3, float a4, float a5, float a6) {
    const long long hi = (long long)__float2int_rn(a0) * 65536 + (long long)__float2int_rn(a1) * 256 +
                         __float2int_rn(a2);
    const long long lo = (long long)__float2int_rn(a3) * 65536 + (long long)__float2int_rn(a4) * 256 +
                         __float2int_rn(__fmaf_rn(a6, 0.00390625f, a5));
    return hi * 16777216 + lo;
}

// acc + S * 2^s for |S| < 2^62: one rounding of S to FP64, then an exact
// power-of-two product and one rounding of the sum; results outside the normal
// range scale in steps.
__device__ __forceinline__ double tc_accum(double acc, long long S, int s) {
    const double d = __ll2double_rn(S);
    if (s >= -1022 && s <= 1023 - 62) return fma(d, tc_pow2(s), acc);
    double v = d;
    int rest = s;
    while (rest != 0) {
        const int step = rest > 1000 ? 1000 : (rest < -1000 ? -1000 : rest);
        v *= tc_pow2(step);
        rest -= step;
    }
    return acc + v;
}

// S * 2^s for |S| < 2^62 (one rounding of S; results outside the normal range
// scale in steps).
__device__ __forceinline__ double tc_scaled(long long S, int s) {
    const double d = __ll2double_rn(S);
    if (s >= -1022 && s <= 1023 - 62) return d * tc_pow2(s);
    double v = d;
    int rest = s;
    while (rest != 0) {
        const int step = rest > 1000 ? 1000 : (rest < -1000 ? -1000 : rest);
        v *= tc_pow2(step);
        rest -= step;
    }
    return v;
}

// Two rows' (or two K terms') digits packed as one bf16x2 word per digit, in
// the two 16-byte units (digits 0-3 and 4-6) of a (column, pair) slot.
__device__ __forceinline__ void tc_pack(const uint32_t (&d0)[kTcSlices], const uint32_t (&d1)[kTcSlices],
                                        uint4& lo, uint4& hi) {
    lo = make_uint4(__byte_perm(d0[0], d1[0], 0x7632), __byte_perm(d0[1], d1[1], 0x7632),
                    __byte_perm(d0[2], d1[2], 0x7632), __byte_perm(d0[3], d1[3], 0x7632));
    hi = make_uint4(__byte_perm(d0[4], d1[4], 0x7632), __byte_perm(d0[5], d1[5], 0x7632),
                    __byte_perm(d0[6], d1[6], 0x7632), 0u);
}

// The 28 digit-pair MMAs of one k-step: A (16 x 16) and B (16 x 8) fragments of
// the seven digit slices, as loaded from the two units of each fragment position.
__device__ __forceinline__ void tc_mma_step(float (&acc)[kTcSlices][4], const uint4& a0l, const uint4& a0h,
                                            const uint4& a1l, const uint4& a1h, const uint4& a2l,
                                            const uint4& a2h, const uint4& a3l, const uint4& a3h,
                                            const uint4& b0l, const uint4& b0h, const uint4& b1l,
                                            const uint4& b1h) {
    const uint32_t A[kTcSlices][4] = {{a0l.x, a1l.x, a2l.x, a3l.x}, {a0l.y, a1l.y, a2l.y, a3l.y},
                                      {a0l.z, a1l.z, a2l.z, a3l.z}, {a0l.w, a1l.w, a2l.w, a3l.w},
                                      {a0h.x, a1h.x, a2h.x, a3h.x}, {a0h.y, a1h.y, a2h.y, a3h.y},
                                      {a0h.z, a1h.z, a2h.z, a3h.z}};
    const uint32_t B[kTcSlices][2] = {{b0l.x, b1l.x}, {b0l.y, b1l.y}, {b0l.z, b1l.z}, {b0l.w, b1l.w},
                                      {b0h.x, b1h.x}, {b0h.y, b1h.y}, {b0h.z, b1h.z}};
#pragma unroll
    for (int p = 0; p < kTcSlices; ++p)
#pragma unroll
        for (int r = 0; r < kTcSlices - p; ++r)
            mma_bf16_16816(acc[p + r], A[p][0], A[p][1], A[p][2], A[p][3], B[r][0], B[r][1]);
}

}  // namespace gm
