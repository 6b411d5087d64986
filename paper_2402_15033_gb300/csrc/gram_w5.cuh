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
// Combine without FP64 per chunk.  The two lanes of row c, (0, c) and (1, c),
// sit in TMEM quarters q and q ^ 2 (warps paired by rank); per group of 8
// columns each hands the partner the cells of the partner's four columns
// through shared memory, so that (0, c) completes the even columns and (1, c)
// the odd ones: I_t = cell(0, t) + cell(1, t - 1), each cell converted to an
// integer by one exact FP32 addition (|cell| <= 2^22) and the two added as
// integers, then S = sum_t I_t 2^(8(5 - t)) (64-bit integer, the 2^-8 tail
// rounded to nearest in integer arithmetic).  The CTA's chunks are
// pre-scanned for each column's largest exponent Emax_c (all-zero chunk
// columns, whose digits are zero, carry a marker and are skipped), and
// S 2^(E_c + E_j' - 50) is accumulated exactly as the 128-bit fixed-point
// integer S 2^(48 - (Emax_c - E_c) - (Emax_j' - E_j')) (units
// 2^(Emax_c + Emax_j' - 98); contributions more than 2^-48 below a unit of the
// largest chunk are truncated); the CTA's sums are rounded to FP64 once at the
// end, and the CTAs' partial blocks are reduced in FP64 as for every Gram.
// Only the needed entries (c <= j', j' >= k) are kept; a warp pair skips a
// group of 8 columns that lies wholly below the diagonal for its 32 rows.
//
// One CTA per SM, warp-specialized, every hand-off an mbarrier with a bounded
// wait.  A warp runs on sub-partition (warp % 4), whose TMEM lane quarter it
// alone may read; the quarters of the rows c < 32 carry twice the combine work
// of the others (the triangle), so they get three combiner warps each and the
// other two quarters two combiner warps plus the slicers:
//   warp 0: bulk copies (TMA) of the chunk's kx x 448 digit bytes and exponents
//           into three raw stages (two chunks in flight ahead of the slicers);
//   warp 2: issues the MMAs into the single accumulator (448 of 512 columns);
//   warps 1, 3, 5, 7: widen the digits into the A tile (one stage: the MMAs of
//           a chunk are done long before its combine frees the accumulator);
//   warps 4, 8, 12 | 9, 13 | 6, 10, 14 | 11, 15: combine TMEM lane quarters
//           0 | 1 | 2 | 3, each warp every third (or second) group of 8 columns.
#pragma once
#include "pip_body.cuh"
#include "tc_common.cuh"
#include "t5_common.cuh"

namespace gm {

constexpr int kW5Threads = 512;
constexpr int kW5MinNB = 9;                       // narrower blocks: gram_t5.cuh / gram_tcq.cuh
constexpr int kW5MaxKX = 64;
constexpr int kW5Stack = 16384;                   // 128 rows x 64 K f16, 128-byte swizzle
constexpr int kW5ATile = 4 * kW5Stack;            // planes 0..7
constexpr int kW5Pairs = 2080;                    // needed entries: at most 64 * 65 / 2
constexpr int kW5Group = 8;                       // columns j' per combine group
constexpr int kW5Slicers = 4;                     // slicer warps
constexpr int kW5Combiners = 10;                  // combiner warps
constexpr int kW5RawStages = 3;
constexpr int kW5DshZero = 1 << 20;               // exponent gap of an all-zero (or invalid) chunk column
constexpr int kW5Pairs5 = 5;                      // combiner warp pairs (quarters 0|2 x 3, 1|3 x 2)
constexpr int kW5XFloats = 2 * 4 * 8 * 32;        // per warp pair: 2 directions x 4 columns x 8 cells x 32 lanes
constexpr size_t kW5A = 0;
constexpr size_t kW5Acc = kW5A + (size_t)kW5ATile;                      // int128 accumulators
constexpr size_t kW5Xb = kW5Acc + (size_t)kW5Pairs * 16;                // cell exchange of the warp pairs
constexpr size_t kW5Raw = kW5Xb + (size_t)kW5Pairs5 * kW5XFloats * 4;   // raw stages follow (size per call)
__host__ __device__ inline int w5_raw_bytes(int kx) { return kx * kTcB8Bytes + 256; }   // digits + exponents
__host__ __device__ inline size_t w5_smem(int kx) { return kW5Raw + kW5RawStages * (size_t)w5_raw_bytes(kx) + 1024; }

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
// S = sum_t I_t 2^(8(5-t)) for t <= 4, plus I_5 + I_6 / 256 rounded to nearest
// (halves up) in integer arithmetic, from the seven exact integer weight sums
// (|I_t| < 2^23): the top two weights in 32 bits, the lower four by 64-bit
// multiply-adds.
__device__ __forceinline__ long long w5_combine(const int (&I)[7]) {
    const int u = I[0] * 256 + I[1];
    long long low = (long long)I[5] + ((I[6] + 128) >> 8);
    low += (long long)I[4] * 256;
    low += (long long)I[3] * 65536;
    low += (long long)I[2] * 16777216;
    return (long long)((unsigned long long)(long long)u << 32) + low;
}

// a (128-bit, little-endian pair) += S 2^sh, |S| < 2^62, sh <= 48, without
// branches: T = S >> r (floor, r = -sh clamped to [0, 63]), then T << l for l =
// max(sh, 0) as a sign-extended 128-bit value.
__device__ __forceinline__ void w5_add2(ulonglong2& a, long long S, int sh) {
    const int l = max(sh, 0), r = min(max(-sh, 0), 63);
    const long long T = S >> r;
    const long long lo = (long long)((unsigned long long)T << l);
    const long long hi = (T >> (63 - l)) >> 1;
    asm("add.cc.u64 %0, %0, %2;\n addc.u64 %1, %1, %3;\n" : "+l"(a.x), "+l"(a.y) : "l"(lo), "l"(hi));
}

// One combine group of a warp pair (lane (D, c) of TMEM quarter q and lane
// (1 - D, c) of quarter q ^ 2): v[t] holds this lane's part of weight t for
// columns j0 .. j0 + 7.  The lane sends the cells of the columns its partner
// completes (D = 0 sends the odd ones, D = 1 the even ones) through xs, takes
// the partner's cells of its own four columns, converts both cells of each
// weight to integers (each at most 4 x 64 x 2^14 = 2^22, the exact range of
// w5_bits; their sum can exceed it) and adds them as integers, combines and
// accumulates.  n counts the pair's exchange rounds (x_full / x_empty phases).
template <int D>
__device__ __forceinline__ void w5_group(const uint32_t (&v)[7][8], float* xs, uint64_t* x_full, uint64_t* x_empty,
                                         int& n, int& fail, unsigned long long* acc, const int* ds, int dc, int c,
                                         int j0, int jlo, int kx, int base, int lane) {
    if (n > 0 && !t5_bar_wait(x_empty, (uint32_t)((n - 1) & 1))) fail = 1;
    float4* out = reinterpret_cast<float4*>(xs) + D * 256;          // direction D: 4 columns x 2 quads x 32 lanes
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int jj = 2 * h + 1 - D;
        out[(2 * h) * 32 + lane] = make_float4(__uint_as_float(v[0][jj]), __uint_as_float(v[1][jj]),
                                               __uint_as_float(v[2][jj]), __uint_as_float(v[3][jj]));
        out[(2 * h + 1) * 32 + lane] = make_float4(__uint_as_float(v[4][jj]), __uint_as_float(v[5][jj]),
                                                   __uint_as_float(v[6][jj]), 0.f);
    }
    __syncwarp();
    if (lane == 0) t5_bar_arrive(x_full);
    if (!t5_bar_wait(x_full, (uint32_t)(n & 1))) fail = 1;
    const float4* in = reinterpret_cast<const float4*>(xs) + (1 - D) * 256;
    long long S[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int jj = 2 * h + D;
        const float4 p0 = in[(2 * h) * 32 + lane], p1 = in[(2 * h + 1) * 32 + lane];
        const float w[7] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z};
        int I[7];
#pragma unroll
        for (int t = 0; t < 7; ++t) I[t] = w5_bits(v[t][jj]) + w5_bits(__float_as_uint(w[t])) - 2 * kW5Magic;
        S[h] = w5_combine(I);
    }
    __syncwarp();
    if (lane == 0) t5_bar_arrive(x_empty);
    ++n;
    // the accumulators of this lane's needed columns: all loads before any store
    const int4 dj0 = *reinterpret_cast<const int4*>(ds + j0);
    const int4 dj1 = *reinterpret_cast<const int4*>(ds + j0 + 4);
    const int dj[8] = {dj0.x, dj0.y, dj0.z, dj0.w, dj1.x, dj1.y, dj1.z, dj1.w};
    ulonglong2 a[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int jj = 2 * h + D, jp = j0 + jj;
        const int p = (jp >= jlo && jp < kx) ? base + jj * j0 + jj * (jj + 1) / 2 : 0;
        a[h] = reinterpret_cast<const ulonglong2*>(acc)[p];
    }
#pragma unroll
    for (int h = 0; h < 4; ++h) w5_add2(a[h], S[h], 48 - dc - dj[2 * h + D]);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int jj = 2 * h + D, jp = j0 + jj;
        if (jp >= jlo && jp < kx) reinterpret_cast<ulonglong2*>(acc)[base + jj * j0 + jj * (jj + 1) / 2] = a[h];
    }
}

// One virtual CTA's partial block over the chunks b, b+G, ...: entry (c, j) of
// [Q(:, 0:k), V(:, 0:nb)]^T V (c <= k + j) goes to slot[c * nb + j] (NaN
// everywhere if a wait timed out).  Every column of [Q, V] is in the digit
// basis (dig, dex, capc; columns 0 .. kx-1).  kW5Threads threads; nb >=
// kW5MinNB, k + nb <= kW5MaxKX; dynamic shared memory w5_smem(k + nb).
__device__ void gram_w5_part(int64_t n, int k, int nb, int b, int G, double* slot, char* smem,
                             const uint4* __restrict__ dig, const int* __restrict__ dex, int capc) {
    // [0..2] raw full, [3..5] raw empty (stage), [6] A full, [7] MMAs done, [8] accumulator read,
    // [9..13] exchange written, [14..18] exchange read (warp pair)
    __shared__ __align__(8) uint64_t bars[9 + 2 * kW5Pairs5];
    __shared__ uint32_t tslot;
    __shared__ __align__(16) int dsh[4][kW5MaxKX];   // Emax_c - E_c of chunk i in slot i % 4 (kW5DshZero: no digits)
    __shared__ int emax[kW5MaxKX];              // the CTA's largest exponent per column
    __shared__ int colbad[kW5MaxKX];            // a NaN or infinity in the column (some chunk of the CTA)
    __shared__ int s_fail;
    uint64_t* raw_full = bars;
    uint64_t* raw_empty = bars + kW5RawStages;
    uint64_t* a_full = bars + 2 * kW5RawStages;
    uint64_t* d_full = a_full + 1;
    uint64_t* tm_empty = a_full + 2;
    uint64_t* x_full = a_full + 3;
    uint64_t* x_empty = x_full + kW5Pairs5;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kx = k + nb;
    smem += (1024 - (t5_smem(smem) & 1023)) & 1023;   // swizzle atoms are 1024-aligned
    const int64_t nchunks = (n + 63) / 64;
    const int nmine = (int64_t)b < nchunks ? (int)((nchunks - 1 - b) / G + 1) : 0;
    const int capx = tc_dex_stride(capc);
    const int rawb = w5_raw_bytes(kx);
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(smem + kW5Acc);
    char* const A = smem + kW5A;

    if (tid == 0) {
        for (int q = 0; q < kW5RawStages; ++q) {
            t5_bar_init(&raw_full[q], 1);
            t5_bar_init(&raw_empty[q], kW5Slicers);
        }
        t5_bar_init(a_full, kW5Slicers);
        t5_bar_init(d_full, 1);
        t5_bar_init(tm_empty, kW5Combiners);
        for (int q = 0; q < kW5Pairs5; ++q) {
            t5_bar_init(&x_full[q], 2);
            t5_bar_init(&x_empty[q], 2);
        }
        t5_bar_init_fence();
        s_fail = 0;
    }
    for (int c = tid; c < kW5MaxKX; c += kW5Threads) {
        emax[c] = -(1 << 30);
        colbad[c] = 0;
    }
    for (int e = tid; e < kW5Pairs; e += kW5Threads) reinterpret_cast<ulonglong2*>(acc)[e] = make_ulonglong2(0ull, 0ull);
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
                const int r = i % kW5RawStages, u = i / kW5RawStages;
                if (u > 0 && !t5_bar_wait(&raw_empty[r], (uint32_t)((u - 1) & 1))) s_fail = 1;
                if (s_fail) break;
                const int64_t ch = b + (int64_t)i * G;
                char* rt = smem + kW5Raw + (size_t)r * rawb;
                t5_bar_arrive_tx(&raw_full[r], (uint32_t)kx * kTcB8Bytes + exb);
                t5_bulk_g2s(rt, dig + (size_t)ch * capc * kTcB8Units, (uint32_t)kx * kTcB8Bytes, &raw_full[r]);
                t5_bulk_g2s(rt + kx * kTcB8Bytes, dex + (size_t)ch * capx, exb, &raw_full[r]);
            }
            // the last copy into each stage has landed before the CTA leaves (bounded)
            for (int q = issued - 1; q >= 0 && q >= issued - kW5RawStages; --q)
                t5_bar_wait(&raw_full[q % kW5RawStages], (uint32_t)((q / kW5RawStages) & 1));
        }
    } else if (warp == 2) {
        // ---- MMA issue: six MMAs per k-step into the seven weight blocks
        if (lane == 0) {
            int done = 0;
            const uint32_t As = t5_smem(A);
            for (int i = 0; i < nmine; ++i) {
                if (!t5_bar_wait(a_full, (uint32_t)(i & 1))) s_fail = 1;
                if (!s_fail && i > 0 && !t5_bar_wait(tm_empty, (uint32_t)((i - 1) & 1))) s_fail = 1;
                if (s_fail) break;
                t5_fence_after_sync();
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    // (stack a, first plane q0, planes, first block): block r gets stack a x plane r - 2a
                    const int ma[6] = {0, 0, 1, 1, 2, 3}, mq[6] = {0, 4, 0, 4, 0, 0}, mn[6] = {4, 3, 4, 1, 3, 1};
#pragma unroll
                    for (int x = 0; x < 6; ++x) {
                        const int a = ma[x], q0 = mq[x], np = mn[x], r0 = 2 * a + q0;
                        const uint64_t ad = t5_sdesc(As + a * kW5Stack + 32 * ks, 16, 1024, kT5Swizzle128);
                        const uint64_t bd = t5_sdesc(As + q0 * 8192 + 32 * ks, 16, 1024, kT5Swizzle128);
                        // the first MMA into each block overwrites it: blocks 0..3 (x = 0), 4..6 (x = 1) at ks = 0
                        const uint32_t accum = (ks > 0 || x >= 2) ? 1u : 0u;
                        t5_mma(tm + 64 * r0, ad, bd, t5_idesc_f16(128, 64 * np, 0, 0), accum);
                    }
                }
                t5_commit(d_full);
                ++done;
            }
            // the last MMAs have completed before the accumulator is freed (bounded)
            if (done > 0) t5_bar_wait(d_full, (uint32_t)((done - 1) & 1));
        }
    } else if ((warp & 1) && warp < 8) {
        // ---- slicers (warps 1, 3, 5, 7): lane = unit 4p + g of columns sw, sw + 8, ...
        // for sw = si and si + 4; plane p in rows 64 p + c; odd p stores its two
        // halves in the other order
        const int si = warp >> 1, st = 32 * si + lane;
        const int wp = lane >> 2, wg = lane & 3;
        const int ch0 = 2 * wg + (wp & 1), ch1 = ch0 ^ 1;
        for (int i = 0; i < nmine; ++i) {
            const int r = i % kW5RawStages, u = i / kW5RawStages;
            // the raw tile has landed; the A tile is free once chunk i - 1's MMAs are done
            bool ok = t5_bar_wait(&raw_full[r], (uint32_t)(u & 1));
            if (ok && i > 0) ok = t5_bar_wait(d_full, (uint32_t)((i - 1) & 1));
            if (!ok) s_fail = 1;
            if (s_fail) break;
            const char* rt = smem + kW5Raw + (size_t)r * rawb;
            if (wp < kTcSlices) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int sw = si + 4 * h;
                    const uint32_t rowb = (uint32_t)((wp * 64 + sw) >> 3) * 1024 + (uint32_t)(sw * 128);
                    const char* src = rt + sw * kTcB8Bytes + lane * 16;
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
            // combiners finished before they released the accumulator of chunk i - 2,
            // which chunk i - 1's MMAs waited for
            for (int c = st; c < kx; c += 32 * kW5Slicers) {
                const int ex = reinterpret_cast<const int*>(rt + kx * kTcB8Bytes)[c];
                dsh[i & 3][c] = (ex == kTcZeroExp || ex == kTcBadExp) ? kW5DshZero : emax[c] - ex;
            }
            t5_fence_async_smem();
            __syncwarp();
            if (lane == 0) {
                t5_bar_arrive(&raw_empty[r]);
                t5_bar_arrive(a_full);
            }
        }
    } else {
        // ---- combiners (10 warps): TMEM lane L = 32 q + lane = 64 d + c, q = warp % 4;
        // quarter q's warps (first warp f, nq of them, rank rk) take groups rk, rk + nq, ...
        // that reach their rows' diagonal
        const int q = warp & 3, qb = 32 * q;
        const int f = (q == 0) ? 4 : (q == 1) ? 9 : (q == 2) ? 6 : 11;
        const int nq = (q & 1) ? 2 : 3, rk = (warp - f) >> 2;
        const int L = qb + lane, d = L >> 6, c = L & 63;
        const int jlo = max(c, k);                        // needed columns: jlo <= j' < kx
        const int wlo = max(qb & 63, k);                  // the warp's smallest needed column
        const int ngr = (kx + kW5Group - 1) / kW5Group;
        int glast = -1;                                   // the warp's last group (-1: none)
        for (int g = rk; g < ngr; g += nq)
            if ((qb & 63) < kx && g * kW5Group + kW5Group - 1 >= wlo) glast = g;
        // the warp pair (quarter q and q ^ 2, same rank): its exchange slot and barriers
        const int pi = (q & 1) ? 3 + rk : rk;
        float* xs = reinterpret_cast<float*>(smem + kW5Xb) + (size_t)pi * kW5XFloats;
        int nx = 0;                                       // the pair's exchange rounds so far
        const int tk = k * (k + 1) / 2;
        for (int i = 0; i < nmine && !s_fail; ++i) {
            if (!t5_bar_wait(d_full, (uint32_t)(i & 1))) s_fail = 1;
            if (s_fail) break;
            t5_fence_after_sync();
            if (glast < 0) {
                __syncwarp();
                if (lane == 0) t5_bar_arrive(tm_empty);
                continue;
            }
            const int* ds = dsh[i & 3];
            const int dc = c < kx ? ds[c] : kW5DshZero;
            for (int g = rk; g <= glast; g += nq) {
                const int j0 = g * kW5Group;
                if (j0 + kW5Group - 1 < wlo) continue;        // wholly below the diagonal for this warp
                // this lane's weight sums for columns j0 .. j0 + 7: v[t] holds weight t
                // (block t - d; weight 0 of the odd planes is empty)
                uint32_t v[7][8];
                const uint32_t ta = tm + ((uint32_t)qb << 16) + (uint32_t)j0;
                if (d == 0) {
#pragma unroll
                    for (int r = 0; r < 7; ++r) t5_ld8(ta + 64 * r, v[r]);
                } else {
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) v[0][jj] = 0u;
#pragma unroll
                    for (int r = 0; r < 6; ++r) t5_ld8(ta + 64 * r, v[r + 1]);
                }
                t5_ld_wait();
                if (g == glast) {
                    // the accumulator is free for the next chunk's MMAs
                    t5_fence_before_sync();
                    __syncwarp();
                    if (lane == 0) t5_bar_arrive(tm_empty);
                }
                const int base = j0 * (j0 + 1) / 2 - tk + c;   // pair index of (c, j0)
                if (d == 0)
                    w5_group<0>(v, xs, &x_full[pi], &x_empty[pi], nx, s_fail, acc, ds, dc, c, j0, jlo, kx, base, lane);
                else
                    w5_group<1>(v, xs, &x_full[pi], &x_empty[pi], nx, s_fail, acc, ds, dc, c, j0, jlo, kx, base, lane);
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
            const ulonglong2 a0 = reinterpret_cast<const ulonglong2*>(acc)[w5_pair(cc, jp, k)];
            unsigned long long lo = a0.x, hi = a0.y;
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
