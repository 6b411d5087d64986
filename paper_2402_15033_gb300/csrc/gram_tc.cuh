// Tall-skinny Gram block [P; G] = [Q, V]^T V on the f16 tensor cores with
// exact integer slicing (the error-free splitting of Ozaki, Ogita, Oishi and
// Rump, 2012): FP64 inputs, results of FP64 quality, for k + nb <= 64.
//
// Per 64-row chunk and column c let E_c be the largest binary exponent in the
// chunk (|x| < 2^(E_c+1)).  Each value is truncated to the integer
// F = trunc(|x| 2^(53 - E_c)) (< 2^54, 54 significant bits for the largest
// entries) and written, signed like x, in balanced base 256 (tc_common.cuh):
//     +-F = sum_{p=0..6} d_p 256^(6-p),  |d_p| <= 128,
// so x = sum_p d_p 2^(E_c - 5 - 8p) within 2^(E_c - 53), and every digit is
// exact in f16.  For a column pair (i, j) the chunk's contribution is
//     x_i^T y_j = 2^(E_i + E_j - 10) sum_{t=0..6} 2^(-8t) I_t,
//     I_t = sum_{p+q=t} sum_rows d_p d'_q,
// and each I_t is accumulated by mma.sync m16n8k16 (f16 inputs, FP32
// accumulators).  Every product is an integer of magnitude <= 2^14, and every
// partial sum is bounded by (t+1) * 64 * 2^14 <= 7 * 2^20 < 2^24, so the FP32
// accumulation is exact.  Pairs with p + q > 6 weigh less than 2^-51 of the
// largest product and are not formed (28 products per output instead of 49).
// After each chunk the seven exact sums are combined in 64-bit integers
// (|S| < 2^59), converted to FP64 (one rounding) and added to the output, scaled
// by 2^(E_i + E_j - 50), with one fused multiply-add.  The per-chunk error is a
// few units of 2^-53 of the chunk's largest product, below the rounding error
// of an FP64 dot product of the same rows.  Subnormal inputs count as zero; a
// NaN or infinity in a column makes every entry of that column's row and
// column of the block NaN, as FP64 arithmetic would.
//
// Two CTAs share an SM, so one slices while the other multiplies.  Within a
// CTA, chunks arrive by asynchronous copies (cp.async) into a raw tile, which
// is free once the chunk is sliced: the next chunk streams in during the MMAs.
// Columns held in the digit basis arrive as their 448 digit bytes in the same
// tile slot and are only widened.  The slices of a column are stored as two
// 16-byte units per row pair (f16 digits 0-3 and 4-6), so a thread loads the
// seven digit words of an MMA fragment position with two 128-bit shared
// loads, free of bank conflicts.
#pragma once
#include "pip_body.cuh"
#include "tc_common.cuh"

namespace gm {

constexpr int kTcRows = 64;                   // rows per chunk (kTcWp holds its 32 row pairs)
constexpr int kTcCols = 72;                   // slice columns kept (tiles may read up to k + 8 ceil(nb/8) - 1 <= 71)
constexpr int kTcMaxTiles = 3;                // 16 x 8 output tiles per warp; k + nb <= 64 needs <= 23
constexpr int kTcMaxKX = 64;
constexpr size_t kTcSliceBytes = (size_t)kTcCols * 2 * kTcWp * 16;

__host__ __device__ constexpr size_t gram_tc_smem(int kx) {
    return (size_t)kx * kTcRows * sizeof(double)      // raw FP64 chunk
           + kTcSliceBytes                            // digit slices (columns >= kx stay zero)
           + kTcCols * sizeof(int);                   // column exponents
}

// Output tiles of the (k+nb) x nb block kept by the symmetric-G rule: M-tiles of
// 16 X columns, N-tiles of 8 Y columns, skipping tiles strictly below the
// diagonal of the G block.
__host__ __device__ inline bool tc_tile_needed(int mt, int nt, int k) { return !(16 * mt - k > 8 * nt + 7); }
__host__ __device__ inline int tc_tile_count(int k, int nb) {
    int cnt = 0;
    for (int mt = 0; mt < (k + nb + 15) / 16; ++mt)
        for (int nt = 0; nt < (nb + 7) / 8; ++nt) cnt += tc_tile_needed(mt, nt, k);
    return cnt;
}

// One virtual CTA's partial block of [Q(:, 0:k), V(:, 0:nb)]^T V(:, 0:nb) over
// the 64-row chunks b, b+G, ...; entry (c, j) goes to slot[c * nb + j].  The
// first kc columns of [Q, V] may come from a digit basis (dig, dex, capc:
// tc_b8_store) instead of being staged and sliced.  256 threads (8 warps);
// k + nb <= 64; dynamic shared memory gram_tc_smem(k + nb).
__device__ void gram_tc_part(int64_t n, const double* __restrict__ Q, int64_t ldq, int k,
                             const double* __restrict__ V, int64_t ldv, int nb, int b, int G,
                             double* slot, double* smem, const uint4* __restrict__ dig = nullptr,
                             const int* __restrict__ dex = nullptr, int capc = 0, int kc = 0) {
    const int kx = k + nb;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gid = lane >> 2, tig = lane & 3;
    double* raw = smem;                                                        // [kx][64]
    uint4* sl = reinterpret_cast<uint4*>(raw + (size_t)kx * kTcRows);          // [72][2][kTcWp] units
    int* ex = reinterpret_cast<int*>(reinterpret_cast<char*>(sl) + kTcSliceBytes);   // [72] unbiased exponents

    for (int e = threadIdx.x; e < kTcCols * 2 * kTcWp; e += blockDim.x) sl[e] = make_uint4(0u, 0u, 0u, 0u);

    // Wide blocks: tiles round robin over the 8 warps.  Narrow blocks (nb <= 8,
    // at most 4 tiles) give each tile a warp pair that splits the chunk's rows
    // (k-steps 0-1 and 2-3): half the chain of dependent MMAs per accumulator,
    // every warp busy; the pair's FP64 sums are added in a fixed order at the end.
    const bool narrow = nb <= 8;
    const int khalf = narrow ? (warp & 1) : 0;
    const int ks0 = narrow ? 2 * khalf : 0, ks1 = narrow ? ks0 + 2 : kTcRows / 16;
    int my_mt[kTcMaxTiles], my_nt[kTcMaxTiles], ntile = 0;
    {
        const int who = narrow ? (warp >> 1) : warp, nwho = narrow ? 4 : 8;
        int cnt = 0;
        for (int mt = 0; mt < (kx + 15) / 16; ++mt)
            for (int nt = 0; nt < (nb + 7) / 8; ++nt) {
                if (!tc_tile_needed(mt, nt, k)) continue;
                if (cnt % nwho == who && ntile < kTcMaxTiles) { my_mt[ntile] = mt; my_nt[ntile] = nt; ++ntile; }
                ++cnt;
            }
    }
    double out[kTcMaxTiles][4];
#pragma unroll
    for (int q = 0; q < kTcMaxTiles; ++q)
#pragma unroll
        for (int i = 0; i < 4; ++i) out[q][i] = 0.0;

    const int64_t nchunks = (n + kTcRows - 1) / kTcRows;
    // the raw tile of chunk ch: FP64 rows of columns kc and up, and the 448
    // digit bytes of each column below kc in that column's 512-byte slot
    auto stage = [&](int64_t ch) {
        if (kc < kx) tc_stage64(Q, ldq, k, V, ldv, kx, ch * kTcRows, n, raw, kc);
        if (kc > 0) {
            const uint4* src = dig + (size_t)ch * capc * kTcB8Units;
            for (int e = threadIdx.x; e < kc * kTcB8Units; e += blockDim.x) {
                const int c = e / kTcB8Units, u = e - c * kTcB8Units;
                cp_async16(reinterpret_cast<uint4*>(raw + (size_t)c * kTcRows) + u, src + e, 16);
            }
        }
        cp_async_commit();
    };
    if ((int64_t)b < nchunks) stage(b);
    for (int64_t ci = b; ci < nchunks; ci += G) {
        cp_async_wait_all();
        __syncthreads();
        // 0. columns held in the digit basis: widen digit p of rows 16w + 2g,
        //    +1 (pair 8w + g) and +8, +9 (pair 8w + g + 4) into the slice units
        for (int e = threadIdx.x; e < kc * 16; e += blockDim.x) {
            const int c = e >> 4, g = (e >> 2) & 3, w = e & 3;
            const uint32_t* src = reinterpret_cast<const uint32_t*>(raw + (size_t)c * kTcRows) + g * 4 + w;
            uint32_t wd[kTcSlices];
#pragma unroll
            for (int p = 0; p < kTcSlices; ++p) wd[p] = src[p * 16];
            uint4* u = sl + (size_t)c * 2 * kTcWp + 8 * w + g;
            u[0] = make_uint4(tc_widen<0x4140>(wd[0]), tc_widen<0x4140>(wd[1]), tc_widen<0x4140>(wd[2]),
                              tc_widen<0x4140>(wd[3]));
            u[kTcWp] = make_uint4(tc_widen<0x4140>(wd[4]), tc_widen<0x4140>(wd[5]), tc_widen<0x4140>(wd[6]), 0u);
            u[4] = make_uint4(tc_widen<0x4342>(wd[0]), tc_widen<0x4342>(wd[1]), tc_widen<0x4342>(wd[2]),
                              tc_widen<0x4342>(wd[3]));
            u[4 + kTcWp] = make_uint4(tc_widen<0x4342>(wd[4]), tc_widen<0x4342>(wd[5]), tc_widen<0x4342>(wd[6]), 0u);
        }
        for (int c = threadIdx.x; c < kc; c += blockDim.x) ex[c] = dex[(size_t)ci * tc_dex_stride(capc) + c];
        // 1. per other column (one warp): exponent of the chunk maximum, then the
        //    digit slices; lane l holds rows 2l and 2l + 1
        for (int c = kc + warp; c < kx; c += 8) {
            const double2 v = reinterpret_cast<const double2*>(raw + (size_t)c * kTcRows)[lane];
            int eb = max(tc_bexp(v.x), tc_bexp(v.y));
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, off));
            const bool bad = eb == 0x7FF;          // NaN or infinity in the chunk
            if (bad || eb == 0) eb = 1023;         // all zero (or subnormal): every digit is zero
            if (lane == 0) ex[c] = bad ? kTcBadExp : eb - 1023;
            uint4* u = sl + (size_t)c * 2 * kTcWp + lane;
            tc_pack(tc_slice(v.x, eb), tc_slice(v.y, eb), u[0], u[kTcWp]);
        }
        __syncthreads();
        // the raw tile is free: the next chunk streams in during the MMAs
        if (ci + G < nchunks) stage(ci + G);
        // 2. exact digit products on the tensor cores, one output tile at a time
#pragma unroll
        for (int q = 0; q < kTcMaxTiles; ++q) {
            if (q >= ntile) break;
            const int m0 = 16 * my_mt[q], n0 = 8 * my_nt[q];
            // unit of (column, digit half 0, row pair tig): Y column j is X column k + j
            const uint4* pa = sl + (size_t)(m0 + gid) * 2 * kTcWp + tig;
            const uint4* pb = sl + (size_t)(k + n0 + gid) * 2 * kTcWp + tig;
            constexpr int C8 = 8 * 2 * kTcWp;      // eight columns further
            float acc[kTcSlices][4];
#pragma unroll
            for (int t = 0; t < kTcSlices; ++t)
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[t][i] = 0.f;
#pragma unroll 1
            for (int ks = ks0; ks < ks1; ++ks) {
                const int w = ks * 8;
                // digits 0-3 (.x..w) and 4-6 of the four A and two B fragment positions
                tc_mma_step(acc, pa[w], pa[w + kTcWp], pa[C8 + w], pa[C8 + w + kTcWp], pa[w + 4], pa[w + 4 + kTcWp],
                            pa[C8 + w + 4], pa[C8 + w + 4 + kTcWp], pb[w], pb[w + kTcWp], pb[w + 4],
                            pb[w + 4 + kTcWp]);
            }
            // 3. the chunk's contribution S * 2^(e_i + e_j - 52), S from the seven exact sums
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int row = m0 + gid + ((i & 2) ? 8 : 0);       // X column
                const int col = n0 + 2 * tig + (i & 1);             // Y column
                if (row >= kx || col >= nb || !needed(row, col, k)) continue;
                const long long S = tc_combine(acc[0][i], acc[1][i], acc[2][i], acc[3][i], acc[4][i], acc[5][i],
                                               acc[6][i]);
                const int ei = ex[row], ej = ex[k + col];
                out[q][i] = max(ei, ej) == kTcBadExp ? __longlong_as_double(0x7FF8000000000000ll)
                                                     : tc_accum(out[q][i], S, ei + ej - kTcShift);
            }
        }
    }
    cp_async_wait_all();
    if (narrow) {
        // the pair's second warp hands its sums to the first through the (now
        // idle) digit slices; the first adds them in a fixed order
        double* red = reinterpret_cast<double*>(sl);
        __syncthreads();
        if (khalf == 1) {
#pragma unroll
            for (int q = 0; q < kTcMaxTiles; ++q) {
                if (q >= ntile) break;
#pragma unroll
                for (int i = 0; i < 4; ++i) red[(((warp >> 1) * kTcMaxTiles + q) * 4 + i) * 32 + lane] = out[q][i];
            }
        }
        __syncthreads();
        if (khalf == 1) return;
#pragma unroll
        for (int q = 0; q < kTcMaxTiles; ++q) {
            if (q >= ntile) break;
#pragma unroll
            for (int i = 0; i < 4; ++i) out[q][i] += red[(((warp >> 1) * kTcMaxTiles + q) * 4 + i) * 32 + lane];
        }
    }
#pragma unroll
    for (int q = 0; q < kTcMaxTiles; ++q) {
        if (q >= ntile) break;
        const int m0 = 16 * my_mt[q], n0 = 8 * my_nt[q];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int row = m0 + gid + ((i & 2) ? 8 : 0);
            const int col = n0 + 2 * tig + (i & 1);
            if (row < kx && col < nb) slot[row * nb + col] = out[q][i];
        }
    }
}

}  // namespace gm
