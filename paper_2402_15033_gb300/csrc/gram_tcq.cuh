// Narrow tall-skinny Gram block [P; G] = [Q, V]^T V (nb <= 8) on the bf16
// tensor cores, with every column of Q read from the digit basis (the exact
// slices of tc_common.cuh) and V sliced in registers.  Same arithmetic as
// gram_tc.cuh: per 64-row chunk each column has one exponent, each digit
// product is exact, the seven digit-pair sums of a chunk are exact FP32
// integers, combined in 64-bit integers and added to the FP64 output with one
// rounding.
//
// Work split.  Every warp owns whole chunks (the CTA's warps take its chunks
// b, b+G, ... in turn) and runs them on its own, with no barrier: the per-chunk
// work is a long chain of dependent steps (slice, 28 MMAs per k-step, combine),
// so the SM's throughput comes from eight chunks in progress at once.  Per
// chunk a warp slices its V columns once (lane (g, t) holds rows 16 ks + 2t,
// +1, +8, +9 of column g, and the four lanes of a column reduce its exponent
// over the 64 rows by shuffles), keeps the B fragments of the four k-steps in
// registers, and then walks the M-tiles (16 columns of [Q, V]), four k-steps
// each, combining every M-tile's outputs once.  A V column of the G block is an
// A operand too: its digits come from the lanes holding it as a B operand.
//
// Memory.  Each lane copies exactly the 16-byte digit units its A fragments
// need for one (M-tile, k-step) (two columns x two row pairs x two digit
// halves) with cp.async into a private four-stage ring in shared memory, three
// steps ahead of the MMAs, and reads back only what it copied, so completion
// needs no barrier (cp.async.wait_group per thread).  The V values of a chunk
// and the Q exponents travel in the same copy groups.
#pragma once
#include "pip_body.cuh"
#include "tc_common.cuh"

namespace gm {

constexpr int kGqWarps = 8;
constexpr int kGqThreads = 32 * kGqWarps;
constexpr int kGqDepth = 4;                       // ring stages per warp ((M-tile, k-step) items)
constexpr int kGqASlots = 9;                      // per lane per stage: 8 Q units + the exponent pair
constexpr int kGqMaxNB = 8;
constexpr int kGqMaxKX = 64;
constexpr size_t kGqRingBytes = (size_t)kGqDepth * kGqASlots * 32 * 16;
constexpr size_t kGqVRingBytes = (size_t)2 * 8 * 32 * 16;    // two chunks' V values, 8 pieces per lane
constexpr size_t kGqWarpBytes = kGqRingBytes + kGqVRingBytes;

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
    const int nmt = (kx + 15) / 16;
    const int ipc = 4 * nmt;                          // items per chunk: (M-tile, k-step)
    char* wbase = smem + (size_t)warp * kGqWarpBytes;
    const unsigned ring_s = (unsigned)__cvta_generic_to_shared(wbase);
    const unsigned vring_s = ring_s + (unsigned)kGqRingBytes;
    const uint4* ring = reinterpret_cast<const uint4*>(wbase) + lane;
    const uint4* vring = reinterpret_cast<const uint4*>(wbase + kGqRingBytes) + lane;
    const int64_t nchunks = (n + 63) / 64;
    const int64_t mine = nchunks > b ? (nchunks - 1 - b) / G + 1 : 0;          // chunks of this CTA
    const int64_t tw = mine > warp ? (mine - 1 - warp) / kGqWarps + 1 : 0;     // chunks of this warp
    const int nitems = (int)(tw * ipc);
    const int capx = tc_dex_stride(capc);
    auto chunk_of = [&](int t) { return b + (warp + (int64_t)t * kGqWarps) * (int64_t)G; };

    // item j = (chunk t, r = 4 mt + ks); the issuing side runs kGqDepth - 1 items ahead
    auto issue = [&](int j, int t, int r) {
        const int mt = r >> 2, ks = r & 3;
        const int64_t ci = chunk_of(t);
        const unsigned st = ring_s + (unsigned)((((j & (kGqDepth - 1)) * kGqASlots) * 32 + lane) * 16);
        const uint4* base = dig + (size_t)ci * capc * 64;
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const int c = 16 * mt + gid + 8 * cc;
            const bool ok = c < k;
            const uint4* cu = base + (size_t)(ok ? c : 0) * 64 + ks * 8 + tig;
#pragma unroll
            for (int pp = 0; pp < 2; ++pp)
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    gq_cp16(st + (unsigned)((cc * 4 + pp * 2 + h) * 512), cu + h * 32 + 4 * pp, ok ? 16 : 0);
            if (ks == 0)
                gq_cp4(st + 8 * 512 + 4 * cc, dex + (size_t)ci * capx + (ok ? c : 0), ok ? 4 : 0);
        }
        if (r == 0) {
            // the chunk's V values: rows 16 ks + 2 tig + {0, 1} and + 8 of column gid
            const bool col = gid < nb;
            const double* vp = V + (int64_t)(col ? gid : 0) * ldv;
            const unsigned vs = vring_s + (unsigned)((((t & 1) * 8) * 32 + lane) * 16);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int64_t rr = ci * 64 + (q >> 1) * 16 + 2 * tig + 8 * (q & 1);
                const int bytes = !col ? 0 : (rr + 2 <= n ? 16 : (rr < n ? 8 : 0));   // zeros past n
                gq_cp16(vs + (unsigned)(q * 512), bytes ? vp + rr : V, bytes);
            }
        }
    };

    double out[4][4];   // [M-tile][fragment entry] (indexed by the runtime M-tile: local memory)
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int e = 0; e < 4; ++e) out[m][e] = 0.0;

    int it_t = 0, it_r = 0;   // issue cursor (chunk, item in chunk)
    auto advance = [&](int& t, int& r) {
        if (++r == ipc) { r = 0; ++t; }
    };
#pragma unroll
    for (int j = 0; j < kGqDepth - 1; ++j) {
        if (j < nitems) issue(j, it_t, it_r);
        advance(it_t, it_r);
        cp_async_commit();
    }
    uint4 bl[4], bh[4], cl[4], ch[4];   // B fragments per k-step: pairs pA (b*) and pB (c*), digit halves
    int j = 0;                           // consume cursor (item index)
    // issue the item kGqDepth - 1 ahead of item j, then wait for item j's copies
    auto step = [&]() {
        if (j + kGqDepth - 1 < nitems) issue(j + kGqDepth - 1, it_t, it_r);
        advance(it_t, it_r);
        cp_async_commit();
        asm volatile("cp.async.wait_group %0;\n" ::"n"(kGqDepth - 1) : "memory");
    };
    for (int t = 0; t < (int)tw; ++t) {
        int ev = 0;   // exponent of V column gid in this chunk
        for (int m = 0; m < nmt; ++m) {
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
            float acc[kTcSlices][4];
#pragma unroll
            for (int tt = 0; tt < kTcSlices; ++tt)
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[tt][i] = 0.f;
            int eq[2] = {0, 0};   // exponents of this lane's two A columns
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                step();
                const uint4* rs = ring + (size_t)(j & (kGqDepth - 1)) * kGqASlots * 32;
                if (ks == 0 && m == 0) {
                    // the chunk's V: exponent of column gid over its 64 rows, then the digits
                    const uint4* vr = vring + (size_t)(t & 1) * 8 * 32;
                    int eb = 0;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const uint4 v = vr[q * 32];
                        eb = max(eb, max(((int)v.y >> 20) & 0x7FF, ((int)v.w >> 20) & 0x7FF));
                    }
                    eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, 1));
                    eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, 2));
                    const bool bad = eb == 0x7FF;          // NaN or infinity in the chunk
                    if (bad || eb == 0) eb = 1023;         // all zero (or subnormal): every digit is zero
                    ev = bad ? kTcBadExp : eb - 1023;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint4 v0 = vr[(2 * q) * 32], v1 = vr[(2 * q + 1) * 32];
                        uint32_t d0[kTcSlices], d1[kTcSlices];
                        tc_slice(__hiloint2double((int)v0.y, (int)v0.x), eb, d0);
                        tc_slice(__hiloint2double((int)v0.w, (int)v0.z), eb, d1);
                        tc_pack(d0, d1, bl[q], bh[q]);
                        tc_slice(__hiloint2double((int)v1.y, (int)v1.x), eb, d0);
                        tc_slice(__hiloint2double((int)v1.w, (int)v1.z), eb, d1);
                        tc_pack(d0, d1, cl[q], ch[q]);
                    }
                }
                if (ks == 0) {
                    const uint4 e = rs[8 * 32];
                    eq[0] = (int)e.x;
                    eq[1] = (int)e.y;
                }
                uint4 a[2][2][2];   // [column c0 / c0 + 8][pair pA / pB][digit half]
#pragma unroll
                for (int cc = 0; cc < 2; ++cc)
#pragma unroll
                    for (int pp = 0; pp < 2; ++pp)
#pragma unroll
                        for (int h = 0; h < 2; ++h) a[cc][pp][h] = rs[(cc * 4 + pp * 2 + h) * 32];
                if (vtile) {
                    // V columns of the G block: their digits from the lanes holding them as B
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc) {
                        uint32_t* lo0 = &a[cc][0][0].x;
                        uint32_t* hi0 = &a[cc][0][1].x;
                        uint32_t* lo1 = &a[cc][1][0].x;
                        uint32_t* hi1 = &a[cc][1][1].x;
                        const uint32_t* s0l = &bl[ks].x;
                        const uint32_t* s0h = &bh[ks].x;
                        const uint32_t* s1l = &cl[ks].x;
                        const uint32_t* s1h = &ch[ks].x;
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            const uint32_t u0 = __shfl_sync(0xffffffffu, s0l[p], vl[cc]);
                            const uint32_t u1 = __shfl_sync(0xffffffffu, s1l[p], vl[cc]);
                            if (isv[cc]) { lo0[p] = u0; lo1[p] = u1; }
                        }
#pragma unroll
                        for (int p = 0; p < 3; ++p) {
                            const uint32_t u0 = __shfl_sync(0xffffffffu, s0h[p], vl[cc]);
                            const uint32_t u1 = __shfl_sync(0xffffffffu, s1h[p], vl[cc]);
                            if (isv[cc]) { hi0[p] = u0; hi1[p] = u1; }
                        }
                    }
                }
                tc_mma_step(acc, a[0][0][0], a[0][0][1], a[1][0][0], a[1][0][1], a[0][1][0], a[0][1][1],
                            a[1][1][0], a[1][1][1], bl[ks], bh[ks], cl[ks], ch[ks]);
                ++j;
            }
            // the M-tile's chunk contribution S * 2^(e_i + e_j - 52)
            const int ej0 = __shfl_sync(0xffffffffu, ev, (2 * tig) << 2);
            const int ej1 = __shfl_sync(0xffffffffu, ev, (2 * tig + 1) << 2);
            int ei[2];
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                const int evc = __shfl_sync(0xffffffffu, ev, vl[cc] & ~3);
                ei[cc] = (m0 + gid + 8 * cc) < k ? eq[cc] : evc;
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
                                                     : tc_accum(out[m][e], S, e1 + e2 - 52);
            }
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
