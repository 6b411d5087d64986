// Exact integer slicing of FP64 values for the f16 tensor cores (the
// error-free splitting of Ozaki, Ogita, Oishi and Rump, 2012), shared by the
// tensor-core Gram (gram_tc.cuh, gram_tcq.cuh) and block update (update_tc.cuh,
// update_tcd.cuh).
//
// A value x is sliced against a common biased exponent eb of its group (a
// chunk column for the Gram, a row for the update), eb >= x's own exponent:
// with E = eb - 1023 (so |x| < 2^(E+1) for the group's largest entries),
// F = trunc(|x| 2^(53 - E)) < 2^54 keeps 54 significant bits of the largest
// entries (53 of FP64 plus one).  The signed integer Fs = +-F is written in
// balanced base 256,
//     Fs = sum_{p=0..6} d_p 256^(6-p),  d_p in [-128, 127] for p >= 1,  |d_0| <= 64,
// so that x = 2^(E-5) sum_p d_p 2^(-8p) within 2^(E-53), and every digit is an
// integer exact in f16.  The digits come out of one 64-bit addition: the low
// seven bytes of G = Fs + 0x0080808080808080 are d_p + 128 (byte 6 - p holds
// digit p), each a biased byte in [0, 255]; a byte b becomes the f16 value
// b - 128 by placing it under the f16 exponent of 1024 (bits 0x6400 | b, the
// value 1024 + b exactly) and subtracting 1152 (exact).
//
// A dot product of two sliced vectors of at most 64 terms is
//     2^(E_x + E_y - 10) sum_{t=0..6} 2^(-8t) I_t,   I_t = sum_{p+q=t} sum_terms d_p d'_q;
// every digit product is an integer of magnitude <= 2^14 and every partial
// sum of I_t is at most (t+1) 64 2^14 < 2^24, so mma.sync (f16 inputs, FP32
// accumulators) forms each I_t exactly.  Digit pairs with p + q > 6 weigh less
// than 2^-51 of the largest product and are not formed.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gm {

constexpr int kTcSlices = 7;                  // balanced base-256 digits
constexpr int kTcWp = 34;                     // 16-byte units per (column, digit half): 32 pairs + 2 pad
constexpr int kTcBadExp = 1 << 20;            // exponent marking a NaN or infinity in the group
constexpr int kTcZeroExp = -(1 << 20);        // stored exponent of an all-zero chunk column (digits all zero)
constexpr int kTcShift = 50;                  // x_i x_j = S 2^(E_i + E_j - kTcShift), S from tc_combine
constexpr uint32_t kTcF16Hi = 0x64646464u;    // f16 exponent byte of 1024, for the widening permutes
constexpr uint32_t kTcF16Bias = 0x64806480u;  // f16x2 (1152, 1152)

__device__ __forceinline__ void mma_f16_16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                              uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Biased FP64 exponent field of x.
__device__ __forceinline__ int tc_bexp(double x) { return (__double2hiint(x) >> 20) & 0x7FF; }

// The seven biased digit bytes of x against the group's biased exponent eb
// (>= x's own): G = Fs + 0x0080808080808080 (low word .x: digits 6, 5, 4, 3 in
// bytes 0-3; high word .y: digits 2, 1, 0 in bytes 0-2, byte 3 zero).  Zero
// and subnormal inputs give Fs = 0.  F = (2m) >> (eb - e) for the 53-bit
// significand m, by two 32-bit funnel shifts.
__device__ __forceinline__ uint2 tc_slice(double x, int eb) {
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const int e = (int)(hi >> 20) & 0x7FF;
    const uint32_t mh = e ? ((hi & 0xFFFFFu) | 0x100000u) : 0u;
    const uint32_t ml = e ? lo : 0u;
    const int d = min(eb - e, 63);
    const uint32_t h = (mh << 1) | (ml >> 31), l = ml << 1;          // twice the significand (54 bits)
    const uint32_t fl = __funnelshift_rc(l, h, d) >> max(d - 32, 0);
    const uint32_t fh = __funnelshift_rc(h, 0u, d);
    unsigned long long F = ((unsigned long long)fh << 32) | fl;
    if (hi >> 31) F = 0ull - F;
    const unsigned long long G = F + 0x0080808080808080ull;
    return make_uint2((uint32_t)G, (uint32_t)(G >> 32));
}

// f16x2 digits from a word of biased bytes [b0, b1, b2, b3]: (b0, b1) with
// SEL = 0x4140, (b2, b3) with SEL = 0x4342.
template <uint32_t SEL>
__device__ __forceinline__ uint32_t tc_widen(uint32_t w) {
    const uint32_t t = __byte_perm(w, kTcF16Hi, SEL);
    uint32_t r;
    asm("sub.rn.f16x2 %0, %1, %2;\n" : "=r"(r) : "r"(t), "r"(kTcF16Bias));
    return r;
}

__device__ __forceinline__ double tc_pow2(int e) {   // e in [-1022, 1023]
    return __longlong_as_double((long long)(e + 1023) << 52);
}

// S = sum_t I_t 2^(8(5-t)) for t <= 4, plus I_5 + I_6 / 256 rounded (0.75 units
// at most: the tail weighs 2^-40 of I_0 and the fold is one FP32 rounding),
// from the seven exact accumulators; |S| < 2^59 for sums of at most 64 terms.
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

// Two rows' (or two K terms') digits as one f16x2 word per digit, in the two
// 16-byte units (digits 0-3 and 4-6) of a (column, pair) slot of the shared
// memory tiles: word p = (digit p of a, digit p of b).
__device__ __forceinline__ void tc_pack(uint2 a, uint2 b, uint4& lo, uint4& hi) {
    const uint32_t l01 = __byte_perm(a.x, b.x, 0x5140);   // bytes 0, 1 of a and b: digits 6, 5
    const uint32_t l23 = __byte_perm(a.x, b.x, 0x7362);   // bytes 2, 3: digits 4, 3
    const uint32_t h01 = __byte_perm(a.y, b.y, 0x5140);   // bytes 4, 5: digits 2, 1
    const uint32_t h23 = __byte_perm(a.y, b.y, 0x7362);   // byte 6: digit 0
    lo = make_uint4(tc_widen<0x4140>(h23), tc_widen<0x4342>(h01), tc_widen<0x4140>(h01), tc_widen<0x4342>(l23));
    hi = make_uint4(tc_widen<0x4140>(l23), tc_widen<0x4342>(l01), tc_widen<0x4140>(l01), 0u);
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
            mma_f16_16816(acc[p + r], A[p][0], A[p][1], A[p][2], A[p][3], B[r][0], B[r][1]);
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

// ---- digit basis: the seven biased digit bytes of basis columns, kept in HBM
// so that a column is sliced once however often it is read (7 bytes per value
// against FP64's 8).  For 64-row chunk ch and column c the 448 bytes at unit
// (ch * capc + c) * kTcB8Units are 28 units of 16 bytes: unit 4p + g (digit p,
// row group g = 0..3) holds, in its word w = 0..3, the biased digit p of rows
// 16w + 2g, +1, +8, +9 as bytes 0-3: exactly the rows that lane (., g) of an
// mma.sync fragment reads in k-step w, so a Gram lane widens each byte once
// and the update lane takes rows r, r+8 of two columns with one permute.
// exps[ch * tc_dex_stride(capc) + c] holds the chunk column's unbiased exponent
// E (kTcBadExp for a NaN or infinity, kTcZeroExp for a chunk column whose
// entries are all zero or subnormal: its digits are all zero, and the marker
// keeps it out of any largest-exponent scan).  The exponents follow the units
// in one buffer; a chunk's row of exponents starts on a 16-byte boundary.
constexpr int kTcB8Units = 28;                // 16-byte units per (chunk, column)
constexpr int kTcB8Bytes = kTcB8Units * 16;   // 448

__host__ __device__ inline size_t tc_digits_units(int64_t n, int capc) {
    return (size_t)((n + 63) / 64) * (size_t)capc * kTcB8Units;
}
__host__ __device__ inline int tc_dex_stride(int capc) { return (capc + 3) & ~3; }
__host__ __device__ inline size_t tc_digits_bytes(int64_t n, int capc) {
    return tc_digits_units(n, capc) * 16 + (size_t)((n + 63) / 64) * (size_t)tc_dex_stride(capc) * sizeof(int) + 256;
}

// The digit-basis word of digit p for the four rows r, r+1, r+8, r+9 from
// their slices: bytes [a_p, b_p, c_p, d_p].
template <int P>
__device__ __forceinline__ uint32_t tc_b8_word(uint2 a, uint2 b, uint2 c, uint2 d) {
    constexpr int byte = 6 - P;                       // byte of G that holds digit P
    constexpr int bb = byte & 3;                      // its byte within the low or high word
    constexpr uint32_t sel = (uint32_t)(bb | ((bb + 4) << 4));   // [x.bb, y.bb, ., .]
    const uint32_t ab = byte < 4 ? __byte_perm(a.x, b.x, sel) : __byte_perm(a.y, b.y, sel);
    const uint32_t cd = byte < 4 ? __byte_perm(c.x, d.x, sel) : __byte_perm(c.y, d.y, sel);
    return __byte_perm(ab, cd, 0x5410);
}

// Slice and store the digits of one chunk column per half warp: called by all
// 32 lanes of a warp (each half warp its own column), lane h = 4w + g of the
// half holding rows 16w + 2g, +1, +8, +9 (x[0..3]; zeros past n).  The
// column's exponent is the largest of its 64 rows.  units points at the
// column's 28 units, *ex at its exponent.
__device__ __forceinline__ void tc_b8_store(const double (&x)[4], uint4* units, int* ex) {
    const int h = threadIdx.x & 15;
    const int w = h >> 2, g = h & 3;
    int eb = max(max(tc_bexp(x[0]), tc_bexp(x[1])), max(tc_bexp(x[2]), tc_bexp(x[3])));
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, off));
    const bool bad = eb == 0x7FF, zero = eb == 0;
    if (bad || zero) eb = 1023;
    const uint2 s0 = tc_slice(x[0], eb), s1 = tc_slice(x[1], eb), s2 = tc_slice(x[2], eb), s3 = tc_slice(x[3], eb);
    uint32_t* u = reinterpret_cast<uint32_t*>(units) + g * 4 + w;   // unit 4p + g, word w
    u[0 * 16] = tc_b8_word<0>(s0, s1, s2, s3);
    u[1 * 16] = tc_b8_word<1>(s0, s1, s2, s3);
    u[2 * 16] = tc_b8_word<2>(s0, s1, s2, s3);
    u[3 * 16] = tc_b8_word<3>(s0, s1, s2, s3);
    u[4 * 16] = tc_b8_word<4>(s0, s1, s2, s3);
    u[5 * 16] = tc_b8_word<5>(s0, s1, s2, s3);
    u[6 * 16] = tc_b8_word<6>(s0, s1, s2, s3);
    if (h == 0) *ex = bad ? kTcBadExp : (zero ? kTcZeroExp : eb - 1023);
}

}  // namespace gm
