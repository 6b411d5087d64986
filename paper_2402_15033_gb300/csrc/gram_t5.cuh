// Narrow tall-skinny Gram block [P; G] = [Q, V]^T V of BCGS-PIP (§IV-C,
// Fig. 4a, first step) on the fifth-generation tensor cores (tcgen05.mma,
// accumulators in tensor memory), for 32 < k + nb <= 64, nb <= 8, every column
// of Q read from the digit basis.  The arithmetic is that of gram_tc.cuh: per
// 64-row chunk each column has one exponent, the balanced base-256 digits are
// exact f16 integers, the digit-weight sums I_t = sum_{p+q=t} X_p^T V_q
// (t <= 6) of a chunk are exact FP32 integers, combined in 64-bit integers and
// added to the FP64 output with one rounding (tc_common.cuh).
//
// MMA shape M = 128 TMEM lanes, K = 16 rows.  The digit planes X_0..X_7 of the
// chunk's kx <= 64 columns are stacked in pairs to 128-row A operands: stack a
// holds planes 2a (lanes c) and 2a + 1 (lanes 64 + c).  The B operand holds
// V's digit planes 0..7, row (q, j) = plane q of V column j.  Stack a
// multiplies planes 0 .. 7 - 2a of B (N = 64 - 16 a) into accumulator columns
// 16 a and up, so that lane 64 d + c, column (w, j) collects
//     sum_a X_{2a + d}(:, c)^T V_{w - 2a}(:, j),  digit weight w + d.
// Its weights t = w + d <= 6 are the chunk's partial sums of I_t over the
// planes of parity d; weights above 6 (including everything plane 7 or a row
// j >= nb of B touches, which therefore never needs clearing) are not read.
// The chunk's rows enter K in the digit basis's own order (row 16w + 2g +
// {0,1,8,9} at K index 16g + 4w + {0..3}), the same permutation for both
// operands.  Operands use the 128-byte swizzle (t5_common.cuh): an A or B row
// holds the chunk's 64 K values, eight rows per 1024-byte atom.
//
// Each lane writes its weight sums (w <= 6, 56 FP32 values) to an exchange
// tile in the stage's A tile, free once the stage's MMAs are done; the owner
// of (c, j) adds I_t = lane (0, c) column (t, j) + lane (1, c) column (t - 1, j)
// (exact), combines S = sum_t I_t 2^(8(5-t)) (64-bit integer, tc_combine),
// releases the stage and adds S 2^(E_c + E_j - 50) to its FP64 sum.
//
// One CTA per SM, warp-specialized, two stages of everything (raw bytes, A and
// B tiles, TMEM accumulator), every hand-off an mbarrier:
//   warp 0      producer: bulk-copies (TMA) a chunk's Q digit bytes (448 per
//               column, contiguous in the digit basis) and exponents;
//   warp 1      issues a chunk's 16 MMAs and commits them;
//   warps 2-9   slicers: widen Q's digit bytes into the A tile; warps 2-5 also
//               slice V's rows (a half warp per column, prefetched a chunk
//               ahead) into A and B;
//   warps 10-13 combiners: exchange, release the stage, combine, accumulate.
// Role-internal hand-offs are mbarriers too (never bar.sync), so that a role
// that gives up after a timed-out wait cannot leave another waiting forever.
#pragma once
#include "pip_body.cuh"
#include "tc_common.cuh"
#include "t5_common.cuh"

namespace gm {

constexpr int kG5Threads = 448;                    // producer, MMA, 8 slicer and 4 combiner warps
constexpr int kG5MaxNB = 8;
constexpr int kG5MinKX = 33;                       // narrower blocks: gram_tcq.cuh
constexpr int kG5MaxKX = 64;
constexpr int kG5RedLd = 60;                       // floats per TMEM lane in the exchange tile (56 used)
constexpr int kG5Stack = 16384;                    // A: one stack = 128 rows x 64 K (128-byte swizzle)
constexpr int kG5ATile = 4 * kG5Stack;
constexpr int kG5BTile = 8 * 1024;                 // B: V's digit planes 0..7, 8 rows (j) each
constexpr int kG5RawTile = kG5MaxKX * kTcB8Bytes + 256;   // digit bytes + exponents
constexpr size_t kG5A = 0;
constexpr size_t kG5B = kG5A + 2 * (size_t)kG5ATile;
constexpr size_t kG5Raw = kG5B + 2 * (size_t)kG5BTile;
constexpr size_t kG5Smem = kG5Raw + 2 * (size_t)kG5RawTile + 1024;   // + alignment of the tiles to 1024 bytes
static_assert((size_t)128 * kG5RedLd * 4 <= (size_t)kG5ATile, "exchange tile fits in the A tile");

// One virtual CTA's partial block over the chunks b, b+G, ...: entry (c, j) of
// [Q(:, 0:k), V(:, 0:nb)]^T V goes to slot[c * nb + j] (NaN everywhere if a
// wait timed out).  Q is the digit basis (dig, dex, capc).  kG5Threads
// threads; kG5MinKX <= k + nb <= kG5MaxKX, nb <= kG5MaxNB; V and ldv 16-byte
// aligned; dynamic shared memory kG5Smem.
__device__ void gram_t5_part(int64_t n, const double* __restrict__ V, int64_t ldv, int k, int nb, int b, int G,
                             double* slot, char* smem, const uint4* __restrict__ dig, const int* __restrict__ dex,
                             int capc) {
    // [0..1] raw full, [2..3] raw empty, [4..5] A/B full, [6..7] MMAs done, [8..9] stage exchanged,
    // [10..11] exchange tile written
    __shared__ __align__(8) uint64_t bars[12];
    __shared__ uint32_t tslot;
    __shared__ int exq[2][kG5MaxKX];            // a stage's Q column exponents
    __shared__ int vex[2][kG5MaxNB];            // its V column exponents
    __shared__ int s_fail;
    uint64_t* raw_full = bars;
    uint64_t* raw_empty = bars + 2;
    uint64_t* a_full = bars + 4;
    uint64_t* d_full = bars + 6;
    uint64_t* s_empty = bars + 8;
    uint64_t* x_ready = bars + 10;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kx = k + nb;
    smem += (1024 - (t5_smem(smem) & 1023)) & 1023;   // swizzle atoms are 1024-aligned
    const int64_t nchunks = (n + 63) / 64;
    const int nmine = (int64_t)b < nchunks ? (int)((nchunks - 1 - b) / G + 1) : 0;
    const int capx = tc_dex_stride(capc);
    const int npair = kx * nb;

    if (tid == 0) {
        for (int q = 0; q < 2; ++q) {
            t5_bar_init(&raw_full[q], 1);
            t5_bar_init(&raw_empty[q], 8);
            t5_bar_init(&a_full[q], 8);
            t5_bar_init(&d_full[q], 1);
            t5_bar_init(&s_empty[q], 4);
            t5_bar_init(&x_ready[q], 4);
        }
        t5_bar_init_fence();
        s_fail = 0;
    }
    if (warp == 0) t5_tmem_alloc(&tslot, 128);
    t5_fence_before_sync();
    __syncthreads();
    t5_fence_after_sync();
    const uint32_t tm = tslot;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};

    if (warp == 0) {
        // ---- producer: the chunk's k x 448 digit bytes and its exponents, two bulk copies
        const uint32_t exb = (uint32_t)((4 * k + 15) & ~15);
        if (lane == 0) {
            for (int i = 0; i < nmine; ++i) {
                const int s = i & 1, u = i >> 1;
                if (u > 0 && !t5_bar_wait(&raw_empty[s], (uint32_t)((u - 1) & 1))) s_fail = 1;
                if (s_fail) break;
                const int64_t ch = b + (int64_t)i * G;
                char* rt = smem + kG5Raw + (size_t)s * kG5RawTile;
                t5_bar_arrive_tx(&raw_full[s], (uint32_t)k * kTcB8Bytes + exb);
                if (k) t5_bulk_g2s(rt, dig + (size_t)ch * capc * kTcB8Units, (uint32_t)k * kTcB8Bytes, &raw_full[s]);
                if (exb) t5_bulk_g2s(rt + kG5MaxKX * kTcB8Bytes, dex + (size_t)ch * capx, exb, &raw_full[s]);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issue: stack a multiplies B's planes 0 .. 7 - 2a into columns 16 a and up
        if (lane == 0) {
            for (int i = 0; i < nmine; ++i) {
                const int s = i & 1, u = i >> 1;
                if (!t5_bar_wait(&a_full[s], (uint32_t)(u & 1))) s_fail = 1;
                if (s_fail) break;
                t5_fence_after_sync();
                const uint32_t A = t5_smem(smem + kG5A + (size_t)s * kG5ATile);
                const uint32_t B = t5_smem(smem + kG5B + (size_t)s * kG5BTile);
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const uint32_t idesc = t5_idesc_f16(128, 64 - 16 * a, 0, 0);
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        const uint64_t ad = t5_sdesc(A + a * kG5Stack + 32 * ks, 16, 1024, kT5Swizzle128);
                        const uint64_t bd = t5_sdesc(B + 32 * ks, 16, 1024, kT5Swizzle128);
                        t5_mma(tm + 64 * s + 16 * a, ad, bd, idesc, (uint32_t)((a | ks) != 0));
                    }
                }
                t5_commit(&d_full[s]);
            }
        }
    } else if (warp < 10) {
        // ---- slicers (256 threads)
        const int st = tid - 64, sw = warp - 2;
        const int vj = st >> 4, h = st & 15, hw = h >> 2, hg = h & 3;       // V (warps 2-5): half warp per column
        const bool vcol = vj < nb;                                          // this half warp slices a column
        const unsigned hmask = 0xFFFFu << (lane & 16);
        const int kch = 2 * hg + (hw >> 1), kof = (hw & 1) * 8;             // K indices 16 hg + 4 hw + 0..3
        // Q: lane = unit 4p + g of columns sw, sw + 8, ...: the two 16-byte halves of
        // the widened unit go to chunks 2g and 2g + 1 of row 64 (p % 2) + c of stack
        // p / 2; odd p stores its halves in the other order, so that each store
        // instruction of a quarter warp covers eight distinct bank groups
        const int wp = lane >> 2, wg = lane & 3;
        const int ch0 = 2 * wg + (wp & 1), ch1 = ch0 ^ 1;
        const uint32_t rowb = (uint32_t)((wp >> 1) * kG5Stack + ((64 * (wp & 1) + sw) >> 3) * 1024 + sw * 128);
        const uint32_t off0 = rowb + (uint32_t)((ch0 ^ sw) << 4), off1 = rowb + (uint32_t)((ch1 ^ sw) << 4);
        // V rows 16 hw + 2 hg, +1, +8, +9 of column vj of chunk ch (zeros past n)
        auto load_v = [&](int64_t ch, double (&x)[4]) {
            x[0] = x[1] = x[2] = x[3] = 0.0;
            const double* vp = V + (size_t)vj * ldv;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int64_t r = ch * 64 + 16 * hw + 2 * hg + 8 * hh;
                if (r + 1 < n) {
                    const double2 t = __ldg(reinterpret_cast<const double2*>(vp + r));
                    x[2 * hh] = t.x;
                    x[2 * hh + 1] = t.y;
                } else if (r < n) {
                    x[2 * hh] = __ldg(vp + r);
                }
            }
        };
        double xn[4] = {0.0, 0.0, 0.0, 0.0};
        if (vcol && nmine > 0) load_v(b, xn);
        for (int i = 0; i < nmine; ++i) {
            const int s = i & 1, u = i >> 1;
            double x[4] = {xn[0], xn[1], xn[2], xn[3]};
            if (vcol && i + 1 < nmine) load_v(b + (int64_t)(i + 1) * G, xn);
            // the raw tile has landed; the stage is free once chunk i - 2's exchange is read
            bool ok = t5_bar_wait(&raw_full[s], (uint32_t)(u & 1));
            if (ok && u > 0) ok = t5_bar_wait(&s_empty[s], (uint32_t)((u - 1) & 1));
            if (!ok) s_fail = 1;
            if (s_fail) break;
            char* A = smem + kG5A + (size_t)s * kG5ATile;
            char* B = smem + kG5B + (size_t)s * kG5BTile;
            const char* rt = smem + kG5Raw + (size_t)s * kG5RawTile;
            // Q's digit units widened into the A tile (plane 7 is never read);
            // column c = sw + 8 t sits one swizzle atom (1024 bytes) after c - 8
            if (wp < kTcSlices) {
                const char* src = rt + sw * kTcB8Bytes + lane * 16;
                char* d0 = A + off0;
                char* d1 = A + off1;
#pragma unroll 2
                for (int c = sw; c < k; c += 8, src += 8 * kTcB8Bytes, d0 += 1024, d1 += 1024) {
                    const uint4 w = *reinterpret_cast<const uint4*>(src);
                    const uint4 lo = make_uint4(tc_widen<0x4140>(w.x), tc_widen<0x4342>(w.x), tc_widen<0x4140>(w.y),
                                                tc_widen<0x4342>(w.y));
                    const uint4 hi = make_uint4(tc_widen<0x4140>(w.z), tc_widen<0x4342>(w.z), tc_widen<0x4140>(w.w),
                                                tc_widen<0x4342>(w.w));
                    *reinterpret_cast<uint4*>(d0) = (wp & 1) ? hi : lo;
                    *reinterpret_cast<uint4*>(d1) = (wp & 1) ? lo : hi;
                }
            }
            for (int c = st; c < k; c += 256) exq[s][c] = reinterpret_cast<const int*>(rt + kG5MaxKX * kTcB8Bytes)[c];
            __syncwarp();
            if (lane == 0) t5_bar_arrive(&raw_empty[s]);
            // V: exponent of each column over the chunk, digit planes into A (column k + j) and B
            if (vcol) {
                int eb = max(max(tc_bexp(x[0]), tc_bexp(x[1])), max(tc_bexp(x[2]), tc_bexp(x[3])));
#pragma unroll
                for (int off = 8; off > 0; off >>= 1) eb = max(eb, __shfl_xor_sync(hmask, eb, off));
                const bool bad = eb == 0x7FF;
                if (bad || eb == 0) eb = 1023;
                if (h == 0) vex[s][vj] = bad ? kTcBadExp : eb - 1023;
                const uint2 s0 = tc_slice(x[0], eb), s1 = tc_slice(x[1], eb), s2 = tc_slice(x[2], eb),
                            s3 = tc_slice(x[3], eb);
                uint32_t wd[kTcSlices];
                wd[0] = tc_b8_word<0>(s0, s1, s2, s3);
                wd[1] = tc_b8_word<1>(s0, s1, s2, s3);
                wd[2] = tc_b8_word<2>(s0, s1, s2, s3);
                wd[3] = tc_b8_word<3>(s0, s1, s2, s3);
                wd[4] = tc_b8_word<4>(s0, s1, s2, s3);
                wd[5] = tc_b8_word<5>(s0, s1, s2, s3);
                wd[6] = tc_b8_word<6>(s0, s1, s2, s3);
                const int c = k + vj;
                char* bq = B + t5_sw128(vj, kch) + kof;
                char* aq0 = A + t5_sw128(c, kch) + kof;          // plane 2a: row c of stack a
                char* aq1 = A + t5_sw128(64 + c, kch) + kof;     // plane 2a + 1: row 64 + c
#pragma unroll
                for (int p = 0; p < kTcSlices; ++p) {
                    const uint2 f = make_uint2(tc_widen<0x4140>(wd[p]), tc_widen<0x4342>(wd[p]));
                    *reinterpret_cast<uint2*>(bq + p * 1024) = f;
                    *reinterpret_cast<uint2*>(((p & 1) ? aq1 : aq0) + (p >> 1) * kG5Stack) = f;
                }
            }
            t5_fence_async_smem();
            __syncwarp();
            if (lane == 0) t5_bar_arrive(&a_full[s]);
        }
    } else {
        // ---- combiners (128 threads): thread ct holds TMEM lane L = 32 (warp % 4) + lane
        const int ct = tid - 320, L = 32 * (warp & 3) + lane;
        int roff[4], cc[4], jj[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int q = ct + m * 128;
            cc[m] = q / nb;
            jj[m] = q - cc[m] * nb;
            roff[m] = cc[m] * kG5RedLd + jj[m];
        }
        for (int i = 0; i < nmine; ++i) {
            const int s = i & 1, u = i >> 1;
            if (!t5_bar_wait(&d_full[s], (uint32_t)(u & 1))) s_fail = 1;
            if (s_fail) break;
            t5_fence_after_sync();
            float* red = reinterpret_cast<float*>(smem + kG5A + (size_t)s * kG5ATile);
            {
                float* rowp = red + L * kG5RedLd;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t r[16];
                    t5_ld16(tm + 64 * s + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(q * 16), r);
                    t5_ld_wait();
#pragma unroll
                    for (int e = 0; e < 16; e += 4)
                        if (q * 16 + e < 56)
                            *reinterpret_cast<uint4*>(rowp + q * 16 + e) = make_uint4(r[e], r[e + 1], r[e + 2], r[e + 3]);
                }
            }
            t5_fence_before_sync();
            __syncwarp();
            if (lane == 0) t5_bar_arrive(&x_ready[s]);
            if (!t5_bar_wait(&x_ready[s], (uint32_t)(u & 1))) s_fail = 1;
            if (s_fail) break;
            // per (c, j): I_t = lane (0, c) column (t, j) + lane (1, c) column (t - 1, j),
            // combined exactly, then the FP64 accumulation S * 2^(E_c + E_j - 50)
            long long S[4];
            int ec[4], ej[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                S[m] = 0;
                ec[m] = ej[m] = 0;
                if (ct + m * 128 < npair) {
                    const float* rp = red + roff[m];
                    float I[kTcSlices];
                    I[0] = rp[0];
#pragma unroll
                    for (int t = 1; t < kTcSlices; ++t) I[t] = rp[t * 8] + rp[64 * kG5RedLd + (t - 1) * 8];
                    S[m] = tc_combine(I[0], I[1], I[2], I[3], I[4], I[5], I[6]);
                    const int c = cc[m];
                    ec[m] = c < k ? exq[s][c] : vex[s][c - k];
                    ej[m] = vex[s][jj[m]];
                }
            }
            __syncwarp();
            if (lane == 0) t5_bar_arrive(&s_empty[s]);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                if (ct + m * 128 < npair)
                    acc[m] = max(ec[m], ej[m]) == kTcBadExp ? __longlong_as_double(0x7FF8000000000000ll)
                                                            : tc_accum(acc[m], S[m], ec[m] + ej[m] - kTcShift);
            }
        }
    }
    __syncthreads();
    if (s_fail) {
        // a wait timed out: give copies and MMAs still in flight time to land (bounded)
        if (tid == 0) {
            for (int q = 0; q < 2; ++q) {
                t5_bar_wait(&raw_full[q], 0u);
                t5_bar_wait(&d_full[q], 0u);
            }
        }
        __syncthreads();
    }
    if (tid >= 320) {
        const int ct = tid - 320;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int q = ct + m * 128;
            if (q < npair) slot[q] = s_fail ? __longlong_as_double(0x7FF8000000000000ll) : acc[m];
        }
    }
    t5_fence_before_sync();
    __syncthreads();
    if (warp == 0) t5_tmem_dealloc(tm, 128);
}

}  // namespace gm
