// Wide Gram block [P; G] = [Q, V]^T V of BCGS-PIP (§IV-C, Fig. 4a) for stage 2
// of the two-stage scheme (§V: CholQR of the big panel), every column of
// X = [Q, V] (kx = k + nb <= 64, nb > 8) in the digit basis, on the
// fifth-generation tensor cores (tcgen05.mma, accumulators in tensor memory).
// Digits, exponents and the digit-weight sums I_t (t <= 6, exact FP32
// integers) are those of gram_tc.cuh (tc_common.cuh).
//
// MMAs.  The chunk's digit planes X_0..X_7 of all kx columns are widened into
// one 128-byte-swizzled K-major tile (plane q in rows 64 q .. 64 q + 63, the
// chunk's 64 rows in the digit basis's order along K), so that stack a (rows
// 128 a .. +127: planes 2a in TMEM lanes c, 2a + 1 in lanes 64 + c) is an A
// operand and any run of consecutive planes a B operand.  Accumulator block r
// (64 TMEM columns 64 r .. 64 r + 63, r = 0..6) collects every product of
// stack a with plane q = r - 2a, so that lane 64 d + c, column 64 r + j' holds
// the part of digit weight r + d of X_c^T X_j' whose X_c plane has parity d.
// Per 16-row k-step six MMAs (M = 128):
//   a = 0, planes 0..3 -> blocks 0..3 (N = 256)   a = 0, planes 4..6 -> 4..6 (192)
//   a = 1, planes 0..3 -> blocks 2..5 (N = 256)   a = 1, plane 4    -> 6    (64)
//   a = 2, planes 0..2 -> blocks 4..6 (N = 192)   a = 3, plane 0    -> 6    (64)
// cover every pair of weight p + q <= 6; the extra products (weights above 6,
// including everything plane 7 touches) land in cells never read.  A cell sums
// at most 4 x 64 digit products, so |cell| <= 2^22.
//
// Combine without FP64 per chunk.  Lane (d, c) forms, per column j', its
// partial S_d = sum_r block r 2^(8(5 - r - d)) (64-bit integer, the 2^-8 tail
// rounded once as in tc_combine; FP32 to integer by an exact addition), and
// adds it to its own 128-bit fixed-point accumulator of the pair (c, j') (one
// set per plane parity d, summed at the end), so the lanes never wait on each
// other.  The CTA's chunks are pre-scanned for each column's largest exponent
// Emax_c (all-zero chunk columns, whose digits are zero, carry a marker and are
// skipped), and S_d 2^(E_c + E_j' - 50) is accumulated exactly as the integer
// S_d 2^(48 - (Emax_c - E_c) - (Emax_j' - E_j')) (units 2^(Emax_c + Emax_j' - 98);
// contributions more than 2^-48 below a unit of the largest chunk are
// truncated); the CTA's sums are rounded to FP64 once at the end, and the CTAs'
// partial blocks are reduced in FP64 as for every Gram.  Only the needed
// entries (c <= j', j' >= k) are kept; a warp skips a group of 8 columns that
// lies wholly below the diagonal for its 32 rows.
//
// One CTA per SM, warp-specialized, every hand-off an mbarrier with a bounded
// wait: warp 0 bulk-copies (TMA) the chunk's kx x 448 digit bytes and
// exponents; warp 1 issues the MMAs into the single accumulator (448 of 512
// TMEM columns); warps 2-5 widen the digits into the A tile (two stages);
// warps 6-13 combine, two per TMEM lane quarter, each taking every other group
// of 8 columns j'.
#pragma once
#include "pip_body.cuh"
#include "tc_common.cuh"
#include "t5_common.cuh"

namespace gm {

constexpr int kW5Threads = 448;
constexpr int kW5MinNB = 9;                       // narrower blocks: gram_t5.cuh / gram_tcq.cuh
constexpr int kW5MaxKX = 64;
constexpr int kW5Stack = 16384;                   // 128 rows x 64 K f16, 128-byte swizzle
constexpr int kW5ATile = 4 * kW5Stack;            // planes 0..7
constexpr int kW5Pairs = 2080;                    // needed entries: at most 64 * 65 / 2
constexpr int kW5Group = 8;                       // columns j' per combine group
constexpr int kW5Slicers = 4;                     // slicer warps (2..5)
constexpr int kW5Combiners = 8;                   // combiner warps (6..13)
constexpr int kW5DshZero = 1 << 20;               // exponent gap of an all-zero (or invalid) chunk column
constexpr size_t kW5A = 0;
constexpr size_t kW5Acc = kW5A + 2 * (size_t)kW5ATile;                  // int128 accumulators, plane parity 0, 1
constexpr size_t kW5Raw = kW5Acc + 2 * (size_t)kW5Pairs * 16;           // one raw stage follows (size per call)
__host__ __device__ inline int w5_raw_bytes(int kx) { return kx * kTcB8Bytes + 256; }   // digits + exponents
__host__ __device__ inline size_t w5_smem(int kx) { return kW5Raw + (size_t)w5_raw_bytes(kx) + 1024; }

// Index of the needed entry (c, j') (c <= j', k <= j' < kx) in the accumulators.
__host__ __device__ inline int w5_pair(int c, int jp, int k) { return (jp * (jp + 1) - k * (k + 1)) / 2 + c; }

// x + 1.5 2^23 for an FP32 x with |x| <= 2^22 lies in [2^23, 2^24], where the
// FP32 spacing is 1: for an integer x the sum is exact and its bit pattern is
// 0x4B400000 + x (at 2^24 too: the exponent field takes the carry); any other
// x is rounded to the nearest integer, ties to even.
constexpr int kW5Magic = 0x4B400000;
__device__ __forceinline__ int w5_bits(uint32_t xbits) {
    return __float_as_int(__fadd_rn(__uint_as_float(xbits), 12582912.0f));
}
// tc_combine's S = sum_t I_t 2^(8(5-t)) for t <= 4 plus I_5 + I_6 / 256 rounded,
// for cells of |I_t| <= 2^22, from the biased bit patterns B_t = 0x4B400000 +
// I_t (the FP32 -> integer conversion unit is slower than these additions):
// the top two weights in 32 bits (the true value fits; the wrap-around of the
// intermediate products cancels), the lower four by 64-bit multiply-adds.
__device__ __forceinline__ long long w5_combine(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t a4,
                                                uint32_t a5, uint32_t a6) {
    const float t = __fmaf_rn(__uint_as_float(a6), 0.00390625f, __uint_as_float(a5));
    const uint32_t u = (uint32_t)w5_bits(a0) * 256u + (uint32_t)w5_bits(a1) - 257u * (uint32_t)kW5Magic;
    long long low = (long long)w5_bits(__float_as_uint(t)) - (long long)kW5Magic * (16777216ll + 65536 + 256 + 1);
    low += (long long)w5_bits(a4) * 256;
    low += (long long)w5_bits(a3) * 65536;
    low += (long long)w5_bits(a2) * 16777216;
    return (long long)((unsigned long long)(long long)(int)u << 32) + low;
}

// acc (128-bit, little-endian pair, 16-byte aligned) += S 2^sh, |S| < 2^62, sh <= 48.
__device__ __forceinline__ void w5_add(unsigned long long* acc, long long S, int sh) {
    long long lo, hi;
    if (sh >= 0) {
        lo = (long long)((unsigned long long)S << sh);
        hi = (S >> (63 - sh)) >> 1;
    } else {
        lo = -sh < 63 ? (S >> -sh) : (S >> 63);
        hi = S >> 63;
    }
    ulonglong2 a = *reinterpret_cast<ulonglong2*>(acc);
    asm("add.cc.u64 %0, %0, %2;\n addc.u64 %1, %1, %3;\n" : "+l"(a.x), "+l"(a.y) : "l"(lo), "l"(hi));
    *reinterpret_cast<ulonglong2*>(acc) = a;
}

// One virtual CTA's partial block over the chunks b, b+G, ...: entry (c, j) of
// [Q(:, 0:k), V(:, 0:nb)]^T V (c <= k + j) goes to slot[c * nb + j] (NaN
// everywhere if a wait timed out).  Every column of [Q, V] is in the digit
// basis (dig, dex, capc; columns 0 .. kx-1).  kW5Threads threads; nb >=
// kW5MinNB, k + nb <= kW5MaxKX; dynamic shared memory w5_smem(k + nb).
__device__ void gram_w5_part(int64_t n, int k, int nb, int b, int G, double* slot, char* smem,
                             const uint4* __restrict__ dig, const int* __restrict__ dex, int capc) {
    // [0] raw full, [1] raw empty, [2..3] A full (stage), [4..5] MMAs done (stage), [6] accumulator read
    __shared__ __align__(8) uint64_t bars[7];
    __shared__ uint32_t tslot;
    __shared__ int dsh[4][kW5MaxKX];            // Emax_c - E_c of chunk i in slot i % 4 (kW5DshZero: no digits)
    __shared__ int emax[kW5MaxKX];              // the CTA's largest exponent per column
    __shared__ int colbad[kW5MaxKX];            // a NaN or infinity in the column (some chunk of the CTA)
    __shared__ int s_fail;
    uint64_t* raw_full = bars;
    uint64_t* raw_empty = bars + 1;
    uint64_t* a_full = bars + 2;
    uint64_t* d_full = bars + 4;
    uint64_t* tm_empty = bars + 6;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kx = k + nb;
    smem += (1024 - (t5_smem(smem) & 1023)) & 1023;   // swizzle atoms are 1024-aligned
    const int64_t nchunks = (n + 63) / 64;
    const int nmine = (int64_t)b < nchunks ? (int)((nchunks - 1 - b) / G + 1) : 0;
    const int capx = tc_dex_stride(capc);
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(smem + kW5Acc);
    char* raw = smem + kW5Raw;

    if (tid == 0) {
        t5_bar_init(raw_full, 1);
        t5_bar_init(raw_empty, kW5Slicers);
        for (int q = 0; q < 2; ++q) {
            t5_bar_init(&a_full[q], kW5Slicers);
            t5_bar_init(&d_full[q], 1);
        }
        t5_bar_init(tm_empty, kW5Combiners);
        t5_bar_init_fence();
        s_fail = 0;
    }
    for (int c = tid; c < kW5MaxKX; c += kW5Threads) {
        emax[c] = -(1 << 30);
        colbad[c] = 0;
    }
    for (int e = tid; e < 2 * kW5Pairs; e += kW5Threads) reinterpret_cast<ulonglong2*>(acc)[e] = make_ulonglong2(0ull, 0ull);
    if (warp == 0) t5_tmem_alloc(&tslot, 512);
    t5_fence_before_sync();
    __syncthreads();
    t5_fence_after_sync();
    const uint32_t tm = tslot;
    // the CTA's column exponents: largest per column (all-zero chunk columns
    // skipped), and NaN/infinity marks
    for (int e = tid; e < nmine * kx; e += kW5Threads) {
        const int i = e / kx, c = e - i * kx;
        const int ex = __ldg(dex + (size_t)(b + (int64_t)i * G) * capx + c);
        if (ex == kTcBadExp) colbad[c] = 1;
        else if (ex != kTcZeroExp) atomicMax(&emax[c], ex);
    }
    __syncthreads();

    if (warp == 0) {
        // ---- producer: the chunk's kx x 448 digit bytes and its exponents, two bulk copies
        const uint32_t exb = (uint32_t)((4 * kx + 15) & ~15);
        if (lane == 0) {
            int issued = 0;
            for (int i = 0; i < nmine; ++i, ++issued) {
                if (i > 0 && !t5_bar_wait(raw_empty, (uint32_t)((i - 1) & 1))) s_fail = 1;
                if (s_fail) break;
                const int64_t ch = b + (int64_t)i * G;
                t5_bar_arrive_tx(raw_full, (uint32_t)kx * kTcB8Bytes + exb);
                t5_bulk_g2s(raw, dig + (size_t)ch * capc * kTcB8Units, (uint32_t)kx * kTcB8Bytes, raw_full);
                t5_bulk_g2s(raw + kx * kTcB8Bytes, dex + (size_t)ch * capx, exb, raw_full);
            }
            // the last copy has landed before the CTA leaves (bounded)
            if (issued > 0) t5_bar_wait(raw_full, (uint32_t)((issued - 1) & 1));
        }
    } else if (warp == 1) {
        // ---- MMA issue: six MMAs per k-step into the seven weight blocks
        if (lane == 0) {
            int done = 0;
            for (int i = 0; i < nmine; ++i) {
                const int s = i & 1, u = i >> 1;
                if (!t5_bar_wait(&a_full[s], (uint32_t)(u & 1))) s_fail = 1;
                if (!s_fail && i > 0 && !t5_bar_wait(tm_empty, (uint32_t)((i - 1) & 1))) s_fail = 1;
                if (s_fail) break;
                t5_fence_after_sync();
                const uint32_t A = t5_smem(smem + kW5A + (size_t)s * kW5ATile);
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    // (stack a, first plane q0, planes, first block): block r gets stack a x plane r - 2a
                    const int ma[6] = {0, 0, 1, 1, 2, 3}, mq[6] = {0, 4, 0, 4, 0, 0}, mn[6] = {4, 3, 4, 1, 3, 1};
#pragma unroll
                    for (int x = 0; x < 6; ++x) {
                        const int a = ma[x], q0 = mq[x], np = mn[x], r0 = 2 * a + q0;
                        const uint64_t ad = t5_sdesc(A + a * kW5Stack + 32 * ks, 16, 1024, kT5Swizzle128);
                        const uint64_t bd = t5_sdesc(A + q0 * 8192 + 32 * ks, 16, 1024, kT5Swizzle128);
                        // the first MMA into each block overwrites it: blocks 0..3 (x = 0), 4..6 (x = 1) at ks = 0
                        const uint32_t accum = (ks > 0 || x >= 2) ? 1u : 0u;
                        t5_mma(tm + 64 * r0, ad, bd, t5_idesc_f16(128, 64 * np, 0, 0), accum);
                    }
                }
                t5_commit(&d_full[s]);
                ++done;
            }
            // the last MMAs into the accumulator have completed before it is freed (bounded)
            for (int q = done - 1; q >= 0 && q >= done - 2; --q) t5_bar_wait(&d_full[q & 1], (uint32_t)((q >> 1) & 1));
        }
    } else if (warp < 2 + kW5Slicers) {
        // ---- slicers (128 threads): lane = unit 4p + g of columns sw, sw + 8, ... for
        // sw = warp - 2 and warp + 2; plane p in rows 64 p + c; odd p stores its two
        // halves in the other order
        const int st = tid - 64;
        const int wp = lane >> 2, wg = lane & 3;
        const int ch0 = 2 * wg + (wp & 1), ch1 = ch0 ^ 1;
        for (int i = 0; i < nmine; ++i) {
            const int s = i & 1, u = i >> 1;
            // the raw tile has landed; the A stage is free once chunk i - 2's MMAs are done
            bool ok = t5_bar_wait(raw_full, (uint32_t)(i & 1));
            if (ok && u > 0) ok = t5_bar_wait(&d_full[s], (uint32_t)((u - 1) & 1));
            if (!ok) s_fail = 1;
            if (s_fail) break;
            char* A = smem + kW5A + (size_t)s * kW5ATile;
            if (wp < kTcSlices) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int sw = warp - 2 + 4 * h;
                    const uint32_t rowb = (uint32_t)((wp * 64 + sw) >> 3) * 1024 + (uint32_t)(sw * 128);
                    const char* src = raw + sw * kTcB8Bytes + lane * 16;
                    char* d0 = A + rowb + ((ch0 ^ sw) << 4);
                    char* d1 = A + rowb + ((ch1 ^ sw) << 4);
#pragma unroll 2
                    for (int c = sw; c < kx; c += 8, src += 8 * kTcB8Bytes, d0 += 1024, d1 += 1024) {
                        const uint4 w = *reinterpret_cast<const uint4*>(src);
                        const uint4 lo = make_uint4(tc_widen<0x4140>(w.x), tc_widen<0x4342>(w.x),
                                                    tc_widen<0x4140>(w.y), tc_widen<0x4342>(w.y));
                        const uint4 hi = make_uint4(tc_widen<0x4140>(w.z), tc_widen<0x4342>(w.z),
                                                    tc_widen<0x4140>(w.w), tc_widen<0x4342>(w.w));
                        *reinterpret_cast<uint4*>(d0) = (wp & 1) ? hi : lo;
                        *reinterpret_cast<uint4*>(d1) = (wp & 1) ? lo : hi;
                    }
                }
            }
            // exponent gaps of chunk i into slot i % 4, which is free: chunk i - 4's
            // combiners finished before they released the accumulator of chunk i - 3,
            // which chunk i - 2's MMAs waited for
            for (int c = st; c < kx; c += 32 * kW5Slicers) {
                const int ex = reinterpret_cast<const int*>(raw + kx * kTcB8Bytes)[c];
                dsh[i & 3][c] = (ex == kTcZeroExp || ex == kTcBadExp) ? kW5DshZero : emax[c] - ex;
            }
            t5_fence_async_smem();
            __syncwarp();
            if (lane == 0) {
                t5_bar_arrive(raw_empty);
                t5_bar_arrive(&a_full[s]);
            }
        }
    } else {
        // ---- combiners (256 threads): TMEM lane L = 32 (warp % 4) + lane = 64 d + c;
        // the warp takes groups hh, hh + 2, ... that reach its rows' diagonal
        const int qb = 32 * (warp & 3), hh = (warp - 2 - kW5Slicers) >> 2;
        const int L = qb + lane, d = L >> 6, c = L & 63;
        const int jlo = max(c, k);                        // needed columns: jlo <= j' < kx
        const int wlo = max(qb & 63, k);                  // the warp's smallest needed column
        const int ngr = (kx + kW5Group - 1) / kW5Group;
        int glast = -1;                                   // the warp's last group (-1: none)
        for (int g = hh; g < ngr; g += 2)
            if ((qb & 63) < kx && g * kW5Group + kW5Group - 1 >= wlo) glast = g;
        unsigned long long* accd = acc + (size_t)d * 2 * kW5Pairs;
        const int tk = k * (k + 1) / 2;
        for (int i = 0; i < nmine && !s_fail; ++i) {
            const int s = i & 1, u = i >> 1;
            if (!t5_bar_wait(&d_full[s], (uint32_t)(u & 1))) s_fail = 1;
            if (s_fail) break;
            t5_fence_after_sync();
            if (glast < 0) {
                __syncwarp();
                if (lane == 0) t5_bar_arrive(tm_empty);
                continue;
            }
            const int* ds = dsh[i & 3];
            const int dc = c < kx ? ds[c] : kW5DshZero;
            for (int g = hh; g <= glast; g += 2) {
                const int j0 = g * kW5Group;
                if (j0 + kW5Group - 1 < wlo) continue;        // wholly below the diagonal for this warp
                // this lane's weight sums for columns j0 .. j0 + 7: block r, weight r + d
                uint32_t v[7][8];
#pragma unroll
                for (int r = 0; r < 7; ++r)
                    if (r < 6 || d == 0) t5_ld8(tm + ((uint32_t)qb << 16) + (uint32_t)(64 * r + j0), v[r]);
                t5_ld_wait();
                if (g == glast) {
                    // the accumulator is free for the next chunk's MMAs
                    t5_fence_before_sync();
                    __syncwarp();
                    if (lane == 0) t5_bar_arrive(tm_empty);
                }
#pragma unroll
                for (int jj = 0; jj < kW5Group; ++jj) {
                    const int jp = j0 + jj;
                    if (jp < jlo || jp >= kx) continue;
                    const long long S = d == 0
                        ? w5_combine(v[0][jj], v[1][jj], v[2][jj], v[3][jj], v[4][jj], v[5][jj], v[6][jj])
                        : w5_combine(0u, v[0][jj], v[1][jj], v[2][jj], v[3][jj], v[4][jj], v[5][jj]);
                    w5_add(accd + 2 * (jp * (jp + 1) / 2 - tk + c), S, 48 - dc - ds[jp]);
                }
            }
        }
    }
    __syncthreads();
    // the CTA's sums, rounded to FP64 once: (hi 2^64 + lo) 2^(Emax_c + Emax_j' - 98)
    for (int e = tid; e < kx * nb; e += kW5Threads) {
        const int cc = e / nb, j = e - cc * nb, jp = k + j;
        if (cc > jp) continue;
        double val;
        if (s_fail || colbad[cc] || colbad[jp]) {
            val = __longlong_as_double(0x7FF8000000000000ll);
        } else {
            const int p = w5_pair(cc, jp, k);
            const ulonglong2 a0 = reinterpret_cast<const ulonglong2*>(acc)[p];
            const ulonglong2 a1 = reinterpret_cast<const ulonglong2*>(acc)[kW5Pairs + p];
            unsigned long long lo = a0.x, hi = a0.y;
            asm("add.cc.u64 %0, %0, %2;\n addc.u64 %1, %1, %3;\n" : "+l"(lo), "+l"(hi) : "l"(a1.x), "l"(a1.y));
            const bool neg = (long long)hi < 0;
            if (neg) {   // magnitude of the two's-complement value
                lo = ~lo + 1ull;
                hi = ~hi + (lo == 0ull ? 1ull : 0ull);
            }
            val = fma((double)hi, 0x1p64, (double)lo);
            val = neg ? -val : val;
            if (val != 0.0) val = ldexp(val, emax[cc] + emax[jp] - 98);
        }
        slot[cc * nb + j] = val;
    }
    t5_fence_before_sync();
    __syncthreads();
    if (warp == 0) t5_tmem_dealloc(tm, 512);
}

}  // namespace gm
