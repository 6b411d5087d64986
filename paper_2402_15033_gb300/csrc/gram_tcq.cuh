// Narrow tall-skinny Gram block [P; G] = [Q, V]^T V (nb <= 8) on the f16
// tensor cores, with every column of Q read from the digit basis (the biased
// digit bytes of tc_common.cuh, 7 bytes per value) and V sliced in registers.
// Same arithmetic as gram_tc.cuh: per 64-row chunk each column has one
// exponent, each digit product is exact, the seven digit-pair sums of a chunk
// are exact FP32 integers, combined in 64-bit integers and added to the FP64
// output with one rounding.
//
// Work split.  Every warp owns whole chunks (the CTA's warps take its chunks
// b, b+G, ... in turn) and runs them on its own, with no barrier: the per-chunk
// work is a long chain of dependent steps (slice, 28 MMAs per k-step, combine),
// so the SM's throughput comes from eight chunks in progress at once.  Per
// chunk a warp slices its V columns once (lane (g, t) holds rows 16 ks + 2t,
// +1, +8, +9 of column g for the four k-steps, and the four lanes of a column
// reduce its exponent by shuffles) into B fragments kept in registers, then
// walks the M-tiles (16 columns of [Q, V]), combining every M-tile's outputs
// once.  A V column of the G block is an A operand too: its digits come from
// the lanes holding it as a B operand.
//
// Memory.  The digit basis stores digit p of rows 16 ks + 2t, +1, +8, +9 as
// one word of unit 4p + t, so lane (g, t) of an M-tile needs exactly units
// 4p + t (p = 0..6) of its two columns: 14 units of 16 bytes, which it copies
// with cp.async into a private three-stage ring, two M-tiles ahead of the
// MMAs, together with the two columns' exponents.  Each lane reads back only
// what it copied, so completion needs no barrier (cp.async.wait_group per
// thread); each digit byte is widened to f16 once, by one byte permute and one
// f16x2 subtraction per pair of rows.  The chunk's V rows travel the same way
// into a per-warp buffer, issued as soon as the previous chunk's V is sliced.
#pragma once
#include "pip_body.cuh"
#include "tc_common.cuh"

namespace gm {

constexpr int kGqWarps = 8;
constexpr int kGqThreads = 32 * kGqWarps;
constexpr int kGqDepth = 3;                       // ring stages per warp (M-tile items)
constexpr int kGqASlots = 15;                     // per lane per stage: 2 columns x 7 digit units + exponents
constexpr int kGqMaxNB = 8;
constexpr int kGqMaxKX = 64;
constexpr size_t kGqRingBytes = (size_t)kGqDepth * kGqASlots * 32 * 16;
constexpr size_t kGqVBytes = (size_t)8 * 32 * 16;            // one chunk's V rows, 8 double pairs per lane
constexpr size_t kGqWarpBytes = kGqRingBytes + kGqVBytes;

__host__ __device__ inline size_t gram_tcq_smem(int) { return (size_t)kGqWarps * kGqWarpBytes; }

__device__ __forceinline__ void gq_cp16(unsigned dst, const void* src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void gq_cp4(unsigned dst, const void* src, int bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}

// One virtual CTA's partial block over the chunks b, b+G, ...: entry (c, j) of
// [Q(:, 0:k), V(:, 0:nb)]^T V goes to slot[c * nb + j].  Q is the digit basis
// (dig, dex, capc; columns 0..k-1 valid for every chunk).  kGqThreads threads;
// nb <= 8, k + nb <= 64; V and ldv 16-byte aligned; dynamic shared memory
// gram_tcq_smem(k).
__device__ void gram_tcq_part(int64_t n, const double* __restrict__ V, int64_t ldv, int k, int nb, int b, int G,
                              double* slot, char* smem, const uint4* __restrict__ dig,
                              const int* __restrict__ dex, int capc) {
    const int kx = k + nb;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const int nmt = (kx + 15) / 16;                   // items (M-tiles) per chunk
    char* wbase = smem + (size_t)warp * kGqWarpBytes;
    const unsigned ring_s = (unsigned)__cvta_generic_to_shared(wbase);
    const unsigned v_s = ring_s + (unsigned)kGqRingBytes;
    const uint4* ring = reinterpret_cast<const uint4*>(wbase) + lane;
    const uint4* vbuf = reinterpret_cast<const uint4*>(wbase + kGqRingBytes) + lane;
    const int64_t nchunks = (n + 63) / 64;
    const int64_t mine = nchunks > b ? (nchunks - 1 - b) / G + 1 : 0;          // chunks of this CTA
    const int64_t tw = mine > warp ? (mine - 1 - warp) / kGqWarps + 1 : 0;     // chunks of this warp
    const int nitems = (int)(tw * nmt);
    const int capx = tc_dex_stride(capc);
    auto chunk_of = [&](int t) { return b + (warp + (int64_t)t * kGqWarps) * (int64_t)G; };

    // item j = (chunk t, M-tile m): the digit units 4p + tig of columns
    // 16m + gid and 16m + gid + 8 (zeros for V columns and past k), and their exponents
    auto issue = [&](int j, int t, int m) {
        const int64_t ci = chunk_of(t);
        const unsigned st = ring_s + (unsigned)(((j % kGqDepth) * kGqASlots * 32 + lane) * 16);
        const uint4* base = dig + (size_t)ci * capc * kTcB8Units + tig;
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const int c = 16 * m + gid + 8 * cc;
            const bool ok = c < k;
            const uint4* cu = base + (size_t)(ok ? c : 0) * kTcB8Units;
#pragma unroll
            for (int p = 0; p < kTcSlices; ++p)
                gq_cp16(st + (unsigned)((cc * kTcSlices + p) * 512), cu + 4 * p, ok ? 16 : 0);
            gq_cp4(st + 14 * 512 + 4 * cc, dex + (size_t)ci * capx + (ok ? c : 0), ok ? 4 : 0);
        }
    };
    // the chunk's V values: rows 16 ks + 2 tig + {0, 1} and + 8 of column gid (zeros past n)
    auto issue_v = [&](int t) {
        const int64_t ci = chunk_of(t);
        const bool col = gid < nb;
        const double* vp = V + (int64_t)(col ? gid : 0) * ldv;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t rr = ci * 64 + (q >> 1) * 16 + 2 * tig + 8 * (q & 1);
            const int bytes = !col ? 0 : (rr + 2 <= n ? 16 : (rr < n ? 8 : 0));
            gq_cp16(v_s + (unsigned)((q * 32 + lane) * 16), bytes ? vp + rr : V, bytes);
        }
    };

    double out[4][4];   // [M-tile][fragment entry]
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int e = 0; e < 4; ++e) out[m][e] = 0.0;

    int it_t = 0, it_m = 0;   // issue cursor (chunk, M-tile)
    auto advance = [&]() {
        if (++it_m == nmt) { it_m = 0; ++it_t; }
    };
    // prologue: items 0 .. kGqDepth - 2, V of chunk 0 with item 0
#pragma unroll
    for (int j = 0; j < kGqDepth - 1; ++j) {
        if (j < nitems) {
            issue(j, it_t, it_m);
            if (j == 0) issue_v(0);
        }
        advance();
        cp_async_commit();
    }
    uint32_t bv[4][kTcSlices][2];   // B fragments: [k-step][digit][rows +0/+1, +8/+9]
    int ev = 0;                     // exponent of V column gid in the current chunk
    int j = 0;                      // consume cursor (item index)
    for (int t = 0; t < (int)tw; ++t) {
        // M-tiles unrolled, so that out[m] stays in registers
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            if (m >= nmt) break;
            // item j's copies (and, at a chunk start, the chunk's V) have landed:
            // V(t) was committed in item j's group or, for one-tile chunks, in the
            // group right after it
            if (nmt >= 2 || m != 0 || t == 0) asm volatile("cp.async.wait_group %0;\n" ::"n"(kGqDepth - 2) : "memory");
            else asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            if (m == 0) {
                // slice the chunk's V: exponent of column gid over its 64 rows, then the digits
                uint4 v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = vbuf[q * 32];
                int eb = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    eb = max(eb, max(((int)v[q].y >> 20) & 0x7FF, ((int)v[q].w >> 20) & 0x7FF));
                eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, 1));
                eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, 2));
                const bool bad = eb == 0x7FF;          // NaN or infinity in the chunk
                if (bad || eb == 0) eb = 1023;         // all zero (or subnormal): every digit is zero
                ev = bad ? kTcBadExp : eb - 1023;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const uint4 x = v[2 * ks + hh];
                        uint4 lo, hi;
                        tc_pack(tc_slice(__hiloint2double((int)x.y, (int)x.x), eb),
                                tc_slice(__hiloint2double((int)x.w, (int)x.z), eb), lo, hi);
                        bv[ks][0][hh] = lo.x;
                        bv[ks][1][hh] = lo.y;
                        bv[ks][2][hh] = lo.z;
                        bv[ks][3][hh] = lo.w;
                        bv[ks][4][hh] = hi.x;
                        bv[ks][5][hh] = hi.y;
                        bv[ks][6][hh] = hi.z;
                    }
                }
                __syncwarp();
                // the V buffer is free: the next chunk's V streams in
                if (t + 1 < (int)tw) issue_v(t + 1);
            }
            if (j + kGqDepth - 1 < nitems) issue(j + kGqDepth - 1, it_t, it_m);
            advance();
            cp_async_commit();

            const uint4* rs = ring + (size_t)(j % kGqDepth) * kGqASlots * 32;
            const uint4 eq = rs[14 * 32];
            const int m0 = 16 * m;
            int vl[2];
            bool isv[2];
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                const int c = m0 + gid + 8 * cc;
                isv[cc] = c >= k && c < kx;
                vl[cc] = (((c - k) & 7) << 2) | tig;
            }
            const bool vtile = m0 + 15 >= k;   // warp-uniform: the M-tile holds V columns
            // even and odd k-steps accumulate separately (each sum stays an exact
            // integer below 2^23), so that consecutive MMAs never wait on each other
            float acc[kTcSlices][4], acc1[kTcSlices][4];
#pragma unroll
            for (int tt = 0; tt < kTcSlices; ++tt)
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[tt][i] = acc1[tt][i] = 0.f;
#pragma unroll
            for (int p = 0; p < kTcSlices; ++p) {
                const uint4 u0 = rs[p * 32], u1 = rs[(kTcSlices + p) * 32];
                const uint32_t w0[4] = {u0.x, u0.y, u0.z, u0.w}, w1[4] = {u1.x, u1.y, u1.z, u1.w};
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    uint32_t a0 = tc_widen<0x4140>(w0[ks]), a2 = tc_widen<0x4342>(w0[ks]);
                    uint32_t a1 = tc_widen<0x4140>(w1[ks]), a3 = tc_widen<0x4342>(w1[ks]);
                    if (vtile) {
                        // V columns of the G block: their digits from the lanes holding them as B
                        const uint32_t s0 = __shfl_sync(0xffffffffu, bv[ks][p][0], vl[0]);
                        const uint32_t s2 = __shfl_sync(0xffffffffu, bv[ks][p][1], vl[0]);
                        const uint32_t s1 = __shfl_sync(0xffffffffu, bv[ks][p][0], vl[1]);
                        const uint32_t s3 = __shfl_sync(0xffffffffu, bv[ks][p][1], vl[1]);
                        if (isv[0]) { a0 = s0; a2 = s2; }
                        if (isv[1]) { a1 = s1; a3 = s3; }
                    }
#pragma unroll
                    for (int r = 0; r < kTcSlices - p; ++r) {
                        if (ks & 1) mma_f16_16816(acc1[p + r], a0, a1, a2, a3, bv[ks][r][0], bv[ks][r][1]);
                        else mma_f16_16816(acc[p + r], a0, a1, a2, a3, bv[ks][r][0], bv[ks][r][1]);
                    }
                }
            }
#pragma unroll
            for (int tt = 0; tt < kTcSlices; ++tt)
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[tt][i] += acc1[tt][i];
            // the M-tile's chunk contribution S * 2^(E_i + E_j - 50)
            const int ej0 = __shfl_sync(0xffffffffu, ev, (2 * tig) << 2);
            const int ej1 = __shfl_sync(0xffffffffu, ev, (2 * tig + 1) << 2);
            int ei[2];
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                const int evc = __shfl_sync(0xffffffffu, ev, vl[cc] & ~3);
                ei[cc] = (m0 + gid + 8 * cc) < k ? (int)(cc ? eq.y : eq.x) : evc;
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int row = m0 + gid + ((e & 2) ? 8 : 0);
                const int col = 2 * tig + (e & 1);
                if (row >= kx || col >= nb || !needed(row, col, k)) continue;
                const long long S = tc_combine(acc[0][e], acc[1][e], acc[2][e], acc[3][e], acc[4][e], acc[5][e],
                                               acc[6][e]);
                const int e1 = ei[(e & 2) ? 1 : 0], e2 = (e & 1) ? ej1 : ej0;
                out[m][e] = max(e1, e2) == kTcBadExp ? __longlong_as_double(0x7FF8000000000000ll)
                                                     : tc_accum(out[m][e], S, e1 + e2 - kTcShift);
            }
            ++j;
        }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();

    // the warps' sums of each M-tile, added in warp order
    double* red = reinterpret_cast<double*>(smem);   // [warp][m][e][lane]
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int e = 0; e < 4; ++e) red[((warp * 4 + m) * 4 + e) * 32 + lane] = out[m][e];
    __syncthreads();
    if (warp >= nmt) return;
    const int m = warp;   // warp m writes M-tile m
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kGqWarps; ++w) s += red[((w * 4 + m) * 4 + e) * 32 + lane];
        const int row = 16 * m + gid + ((e & 2) ? 8 : 0);
        const int col = 2 * tig + (e & 1);
        if (row < kx && col < nb) slot[row * nb + col] = s;
    }
}

}  // namespace gm
