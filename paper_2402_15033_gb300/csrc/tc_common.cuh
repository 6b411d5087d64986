// Exact integer slicing of FP64 values for the bf16 tensor cores (the
// error-free splitting of Ozaki, Ogita, Oishi and Rump, 2012), shared by the
// tensor-core Gram (gram_tc.cuh) and block update (update_tc.cuh).
//
// A value x is sliced against a common biased exponent eb of its group (a
// chunk column for the Gram, a row for the update), eb >= x's own exponent:
// F = trunc(|x| 2^(54 - e)) (e = eb - 1023; F < 2^55) is written in balanced
// base 256, F = sum_{p=0..6} d_p 256^(6-p) with |d_p| <= 128, signed like x, so
// that x = sum_p d_p 2^(e - 6 - 8p) within 2^(e - 54) (55 bits for the
// group's largest entries) and every digit is exact in bf16.  A dot product of two sliced vectors of at most
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

// The seven digits of x against the group's biased exponent eb (>= x's own),
// as FP32 bit patterns whose high halves are the bf16 digits: F =
// trunc(|x| 2^(54 - e)) (e = eb - 1023; zero and subnormals give 0) is shifted
// into place with two 32-bit funnel shifts, 128 is added at every lower digit
// position (each byte of the sum is then the balanced digit plus 128, the
// carries included), and a byte b becomes the float +-(b - 128) by one byte
// permute into the signed constant +-1.5 * 2^23 and one exact addition.
__device__ __forceinline__ void tc_slice(double x, int eb, uint32_t (&dig)[kTcSlices]) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const int e = (int)(hi >> 20) & 0x7FF;
    const uint32_t mh = e ? ((hi & 0xFFFFFu) | 0x100000u) : 0u;
    const uint32_t ml = e ? lo : 0u;
    const int d = min(eb - e, 63);
    const uint32_t h = (mh << 2) | (ml >> 30), l = ml << 2;          // the mantissa times 4 (55 bits)
    const uint32_t fl = __funnelshift_rc(l, h, d) >> max(d - 32, 0);
    const uint32_t fh = __funnelshift_rc(h, 0u, d);
    const unsigned long long G = (((unsigned long long)fh << 32) | fl) + 0x808080808080ull;
    const uint32_t gl = (uint32_t)G, gh = (uint32_t)(G >> 32);
    const bool neg = (hi >> 31) != 0;
    const uint32_t magic = neg ? 0xCB400000u : 0x4B400000u;
    const float off = neg ? 12583040.0f : -12583040.0f;
    const float off0 = neg ? 12582912.0f : -12582912.0f;
    dig[6] = __float_as_uint(__fadd_rn(__uint_as_float(__byte_perm(gl, magic, 0x7650)), off));
    dig[5] = __float_as_uint(__fadd_rn(__uint_as_float(__byte_perm(gl, magic, 0x7651)), off));
    dig[4] = __float_as_uint(__fadd_rn(__uint_as_float(__byte_perm(gl, magic, 0x7652)), off));
    dig[3] = __float_as_uint(__fadd_rn(__uint_as_float(__byte_perm(gl, magic, 0x7653)), off));
    dig[2] = __float_as_uint(__fadd_rn(__uint_as_float(__byte_perm(gh, magic, 0x7650)), off));
    dig[1] = __float_as_uint(__fadd_rn(__uint_as_float(__byte_perm(gh, magic, 0x7651)), off));
    dig[0] = __float_as_uint(__fadd_rn(__uint_as_float(magic + (gh >> 16)), off0));
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

// S * 2^s in FP64 for |S| < 2^62 by integer operations (rounded to nearest
// even), so that only the accumulation itself uses the FP64 pipe; results
// outside the normal range go through FP64 multiplications by powers of two.
__device__ __forceinline__ double tc_int_to_double(long long S, int s) {
    if (S == 0) return 0.0;
    const unsigned long long sgn = S < 0 ? (1ull << 63) : 0ull;
    unsigned long long M = (unsigned long long)(S < 0 ? -S : S);
    int msb = 63 - __clzll((long long)M);
    if (msb > 52) {
        const int r = msb - 52;
        const unsigned long long half = 1ull << (r - 1);
        const unsigned long long rem = M & ((1ull << r) - 1);
        M >>= r;
        if (rem > half || (rem == half && (M & 1))) ++M;
        if (M >> 53) { M >>= 1; ++msb; }
    } else {
        M <<= (52 - msb);
    }
    const int be = msb + s + 1023;
    if (be >= 1 && be <= 2046)
        return __longlong_as_double((long long)(sgn | ((unsigned long long)be << 52) | (M & 0xFFFFFFFFFFFFFull)));
    double v = __longlong_as_double((long long)(sgn | ((unsigned long long)(msb + 1023) << 52) |
                                                (M & 0xFFFFFFFFFFFFFull)));
    int rest = s;
    while (rest != 0) {
        const int step = rest > 1000 ? 1000 : (rest < -1000 ? -1000 : rest);
        v *= __longlong_as_double((long long)(step + 1023) << 52);
        rest -= step;
    }
    return v;
}

// acc + S * 2^s for |S| < 2^62: S rounded once to FP64 and added with one
// fused multiply-add (the power-of-two product is exact); scales outside the
// normal range take the integer conversion.
__device__ __forceinline__ double tc_accum(double acc, long long S, int s) {
    if (s >= -1022 && s <= 1023 - 62) return fma(__ll2double_rn(S), tc_pow2(s), acc);
    return acc + tc_int_to_double(S, s);
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

// Asynchronous copies of a 64-row chunk of [Q(:, 0:k), V(:, 0:kx-k)] (columns
// cb and up) into a column-major shared tile (ld 64): thread t copies rows
// 2(t % 32), +1 of columns t / 32, t / 32 + nw, ... (nw = blockDim / 32),
// walking the column pointers by increments; rows at or beyond n are
// zero-filled.  Q, V and
// their leading dimensions are 16-byte aligned (row0 is even).
__device__ __forceinline__ void tc_stage64(const double* Q, int64_t ldq, int k, const double* V, int64_t ldv,
                                           int kx, int64_t row0, int64_t n, double* tile, int cb = 0) {
    const int q = threadIdx.x & 31, c0 = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t row = row0 + 2 * q;
    const int bytes = row + 2 <= n ? 16 : (row < n ? 8 : 0);
    const unsigned dst0 = (unsigned)__cvta_generic_to_shared(tile + 2 * q);
    int c = c0;
    if (c < cb) c += (cb - c + nw - 1) / nw * nw;   // columns below cb are not staged
    for (const double* p = Q + (int64_t)c * ldq + row; c < k; c += nw, p += (int64_t)nw * ldq)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst0 + (unsigned)c * 512u),
                     "l"(bytes ? p : Q), "r"(bytes) : "memory");
    for (const double* p = V + (int64_t)(c - k) * ldv + row; c < kx; c += nw, p += (int64_t)nw * ldv)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst0 + (unsigned)c * 512u),
                     "l"(bytes ? p : V), "r"(bytes) : "memory");
}

// ---- digit basis: the seven digit slices of basis columns, kept in HBM so that
// a column is sliced once however often it is read.  For 64-row chunk ch and
// column c, units [(ch * capc + c) * 64, +64) hold the 32 row pairs' digits
// 0-3 (units 0-31) and 4-6 (units 32-63) in the shared-memory unit format of the
// Gram kernel (without its padding), and exps[ch * tc_dex_stride(capc) + c] the
// chunk column's unbiased exponent (kTcBadExp for a NaN or infinity).  The
// exponents follow the units in one buffer; a chunk's row of exponents starts
// on a 16-byte boundary, so that one bulk copy can fetch it.
__host__ __device__ inline size_t tc_digits_units(int64_t n, int capc) {
    return (size_t)((n + 63) / 64) * (size_t)capc * 64;
}
__host__ __device__ inline int tc_dex_stride(int capc) { return (capc + 3) & ~3; }
__host__ __device__ inline size_t tc_digits_bytes(int64_t n, int capc) {
    return tc_digits_units(n, capc) * 16 + (size_t)((n + 63) / 64) * (size_t)tc_dex_stride(capc) * sizeof(int) + 256;
}

// Slice column c of a 64-row chunk (lane l holds rows 2l, 2l+1: x0, x1) into
// the digit basis; one warp.
__device__ __forceinline__ void tc_digits_store(double x0, double x1, int64_t ch, int c, int capc, uint4* units,
                                                int* exps) {
    const int lane = threadIdx.x & 31;
    int eb = max(tc_bexp(x0), tc_bexp(x1));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, off));
    const bool bad = eb == 0x7FF;
    if (bad || eb == 0) eb = 1023;
    uint32_t d0[kTcSlices], d1[kTcSlices];
    tc_slice(x0, eb, d0);
    tc_slice(x1, eb, d1);
    uint4 lo, hi;
    tc_pack(d0, d1, lo, hi);
    uint4* u = units + ((size_t)ch * capc + c) * 64;
    u[lane] = lo;
    u[32 + lane] = hi;
    if (lane == 0) exps[(size_t)ch * tc_dex_stride(capc) + c] = bad ? kTcBadExp : eb - 1023;
}

}  // namespace gm
