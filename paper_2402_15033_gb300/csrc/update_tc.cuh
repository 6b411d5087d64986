// Block update of BCGS-PIP (§IV-C, Fig. 4a, last step) on the f16 tensor
// cores by exact slicing (tc_common.cuh):
//     V <- (V - Q P) T^{-1} = [Q, V] W,   W = [-P T^{-1}; T^{-1}]   (kx = k + nb <= 64).
// Every CTA forms W in FP64 from R (T^{-1} by substitution), slices its columns
// once, and then streams 64-row chunks of X = [Q, V]: each row is sliced against
// its own largest exponent (the output of a row is a dot product along that
// row), the digit products run on the tensor cores with FP32 accumulators that
// stay exact, and every output is S * 2^(e_row + f_col - 50) rounded once to
// FP64 (the scaling of tc_common.cuh).
//
// Equilibration: a row mixes Q entries (unit columns) with V entries whose
// column norms ||V_j|| = ||R(:, j)|| can be far from one; slicing such a row
// against its largest entry would cost the small ones bits that W then
// amplifies.  V's columns are therefore sliced as V_j 2^(-g_j) and W's rows
// scaled by 2^(g_j), g_j = floor(log2 ||R(:, j)||): both exact.  The result
// then carries a few units of 2^-53 of sum_c |X_rc| |W_cj| at the row and
// column scales, the FP64 level.
#pragma once
#include "pip_body.cuh"
#include "tc_common.cuh"

namespace gm {

constexpr int kTuRows = 64;                   // rows per chunk (a warp pair covers them, one row per lane)
constexpr int kTuMaxKX = 64;
constexpr int kTuMaxTiles = 2;                // 4 M-tiles x N-tiles: <= 16 over 8 warps (nb <= 32), <= 32 over 16

__host__ __device__ constexpr int tu_nbp(int nb) { return (nb + 7) / 8 * 8; }
// shared memory: raw chunk, X slices, W slices, integer tables
__host__ __device__ constexpr size_t update_tc_smem(int kx, int nb, bool digits = false) {
    return (size_t)kx * kTuRows * sizeof(double) + (size_t)kTuRows * 2 * kTcWp * 16 +
           (size_t)tu_nbp(nb) * 2 * kTcWp * 16 + (64 + 64 + kTuRows + 8 * kTuRows) * sizeof(int) +
           (digits ? (size_t)nb * kTuRows * sizeof(double) : 0);   // output tile of the digit-basis writes
}

// Row r's unit for K pair w (two consecutive columns) in the X slices; the low
// two bits of w are permuted by row so that both the slicing stores (32 rows,
// one pair) and the fragment loads (8 rows x 4 pairs) are free of bank conflicts.
__device__ __forceinline__ int tu_xunit(int r, int half, int w) {
    return (r * 2 + half) * kTcWp + (w ^ ((r >> 1) & 3));
}

__device__ __forceinline__ int tu_colshift(double nrm2) {
    const int e = tc_bexp(nrm2);
    if (e == 0 || e == 0x7FF) return 0;
    return (e - 1023) >> 1;                       // floor(log2 ||v||) or one less
}

// X = [Q(:, 0:k), V(:, 0:nb)] rows in 64-row chunks b, b+G, ...; V overwritten;
// with DIG the new columns' digits also go to digit-basis columns k .. k+nb-1.
// blockDim.x = 32 * NW, NW >= 8.
template <bool DIG>
__device__ void update_tc_body(int64_t n, const double* __restrict__ Q, int64_t ldq, int k, double* V,
                               int64_t ldv, int nb, const double* __restrict__ R, int ldr, int mode, int b, int G,
                               char* smem, uint4* dig, int* dex, int capc) {
    const int kx = k + nb, nbp = tu_nbp(nb);
    const int NW = blockDim.x >> 5;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const int nks = (kx + 15) / 16;               // K steps; pairs w < 8 nks are sliced (zeros past kx)
    double* raw = reinterpret_cast<double*>(smem);                                       // [kx][64]
    uint4* xu = reinterpret_cast<uint4*>(smem + (size_t)kx * kTuRows * sizeof(double));   // [64][2][kTcWp]
    uint4* wu = xu + kTuRows * 2 * kTcWp;                                                  // [nbp][2][kTcWp]
    int* cshift = reinterpret_cast<int*>(wu + (size_t)nbp * 2 * kTcWp);                    // [64]
    int* fexp = cshift + 64;                                                               // [64]
    int* rexp = fexp + 64;                                                                 // [64]
    int* epart = rexp + kTuRows;                                                           // [8][64]
    double* otile = reinterpret_cast<double*>(epart + 8 * kTuRows);                        // [nb][64]

    // ---- W = [-P T^{-1}; T^{-1}] scaled by the column shifts, in FP64, then sliced
    double* Ts = reinterpret_cast<double*>(wu);   // nb x nb (T), then T^{-1}, in the W-slice region
    double* Ti = Ts + nb * nb;
    double* Wd = reinterpret_cast<double*>(xu);   // kx x nb, in the X-slice region
    double* Dinv = raw;                           // nb reciprocals
    const bool notrsm = (mode & kPipNoTrsm) != 0;
    for (int c = tid; c < kx; c += blockDim.x) {
        int g = 0;
        if (c >= k && !notrsm) {
            const int j = c - k;
            double s2 = 0.0;
            for (int i = 0; i <= k + j; ++i) {
                const double v = R[i + (size_t)j * ldr];
                s2 = fma(v, v, s2);
            }
            g = tu_colshift(s2);
        }
        cshift[c] = g;
    }
    for (int e = tid; e < nb * nb; e += blockDim.x) {
        const int i = e % nb, l = e / nb;
        Ts[e] = notrsm ? (i == l ? 1.0 : 0.0) : (i <= l ? R[(k + i) + (size_t)l * ldr] : 0.0);
    }
    __syncthreads();
    for (int i = tid; i < nb; i += blockDim.x) Dinv[i] = 1.0 / Ts[i + i * nb];
    __syncthreads();
    for (int j = tid; j < nb; j += blockDim.x) {          // column j of T^{-1} by back substitution
        for (int i = nb - 1; i > j; --i) Ti[i + j * nb] = 0.0;
        Ti[j + j * nb] = Dinv[j];
        for (int i = j - 1; i >= 0; --i) {
            double s = 0.0;
            for (int l = i + 1; l <= j; ++l) s = fma(Ts[i + l * nb], Ti[l + j * nb], s);
            Ti[i + j * nb] = -s * Dinv[i];
        }
    }
    __syncthreads();
    for (int e = tid; e < kx * nb; e += blockDim.x) {
        const int c = e % kx, j = e / kx;
        double w;
        if (c < k) {
            double s = 0.0;
            for (int l = 0; l <= j; ++l) s = fma(R[c + (size_t)l * ldr], Ti[l + j * nb], s);
            w = -s;
        } else {
            w = Ti[(c - k) + j * nb];
        }
        Wd[e] = w * tc_pow2(cshift[c]);
    }
    __syncthreads();
    for (int e = tid; e < nbp * 2 * kTcWp; e += blockDim.x) wu[e] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    // slice W column j against its own exponent: lane = K pair (rows 2l, 2l + 1 of W)
    for (int j = warp; j < nb; j += NW) {
        const int c0 = 2 * lane, c1 = 2 * lane + 1;
        const double w0 = c0 < kx ? Wd[c0 + j * kx] : 0.0;
        const double w1 = c1 < kx ? Wd[c1 + j * kx] : 0.0;
        int eb = max(tc_bexp(w0), tc_bexp(w1));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, off));
        const bool bad = eb == 0x7FF;
        if (bad || eb == 0) eb = 1023;
        if (lane == 0) fexp[j] = bad ? kTcBadExp : eb - 1023;
        uint4* u = wu + (size_t)j * 2 * kTcWp + lane;
        tc_pack(tc_slice(w0, eb), tc_slice(w1, eb), u[0], u[kTcWp]);
    }
    __syncthreads();

    // ---- output tiles: M-tiles of 16 rows (2 per chunk) x N-tiles of 8 columns
    int my_mt[kTuMaxTiles], my_nt[kTuMaxTiles], ntile = 0;
    {
        int cnt = 0;
        for (int nt = 0; nt < nbp / 8; ++nt)
            for (int mt = 0; mt < kTuRows / 16; ++mt) {
                if (cnt % NW == warp && ntile < kTuMaxTiles) { my_mt[ntile] = mt; my_nt[ntile] = nt; ++ntile; }
                ++cnt;
            }
    }
    const int fa = (gid >> 1) & 3;               // the row permutation of tu_xunit for rows m0 + gid (+8)

    const int64_t nchunks = (n + kTuRows - 1) / kTuRows;
    if ((int64_t)b < nchunks) {
        tc_stage64(Q, ldq, k, V, ldv, kx, (int64_t)b * kTuRows, n, raw);
        cp_async_commit();
    }
    const int half = warp & 1, grp = warp >> 1, ngrp = NW >> 1;
    const int r = half * 32 + lane;              // this thread's row of the chunk (slicing phases)
    for (int64_t ci = b; ci < nchunks; ci += G) {
        const int64_t row0 = ci * kTuRows;
        cp_async_wait_all();
        __syncthreads();
        // 1. row exponents of the shifted columns: thread (row r, K pairs grp, grp + ngrp, ...)
        int emax = -100000;                       // no nonzero value seen
        for (int w = grp; w < 8 * nks; w += ngrp) {
            const int c0 = 2 * w, c1 = 2 * w + 1;
            const double x0 = c0 < kx ? raw[c0 * kTuRows + r] : 0.0;
            const double x1 = c1 < kx ? raw[c1 * kTuRows + r] : 0.0;
            const int e0 = tc_bexp(x0), e1 = tc_bexp(x1);
            if (e0 == 0x7FF || e1 == 0x7FF) emax = 0x7FF + 4096;
            if (e0) emax = max(emax, e0 - cshift[c0]);
            if (e1) emax = max(emax, e1 - cshift[min(c1, kx - 1)]);
        }
        epart[grp * kTuRows + r] = emax;
        __syncthreads();
        int eb = -100000;
        for (int q = 0; q < ngrp; ++q) eb = max(eb, epart[q * kTuRows + r]);
        const bool bad = eb > 0x7FF + 2048;      // above any shifted exponent: a NaN/inf in the row
        if (bad || eb == -100000) eb = 1023;      // NaN/inf row, or an all-zero row (digits all zero)
        if (grp == 0) rexp[r] = bad ? kTcBadExp : eb - 1023;
        // 2. slices of the row against eb (+ the column shift)
        for (int w = grp; w < 8 * nks; w += ngrp) {
            const int c0 = 2 * w, c1 = 2 * w + 1;
            const double x0 = c0 < kx ? raw[c0 * kTuRows + r] : 0.0;
            const double x1 = c1 < kx ? raw[c1 * kTuRows + r] : 0.0;
            tc_pack(tc_slice(x0, eb + cshift[min(c0, kx - 1)]), tc_slice(x1, eb + cshift[min(c1, kx - 1)]),
                    xu[tu_xunit(r, 0, w)], xu[tu_xunit(r, 1, w)]);
        }
        __syncthreads();
        // the raw tile is free: the next chunk streams in during the MMAs
        if (ci + G < nchunks) {
            tc_stage64(Q, ldq, k, V, ldv, kx, (ci + G) * kTuRows, n, raw);
            cp_async_commit();
        }
        // 3. digit products and the outputs of this warp's tiles
#pragma unroll
        for (int q = 0; q < kTuMaxTiles; ++q) {
            if (q >= ntile) break;
            const int m0 = 16 * my_mt[q], n0 = 8 * my_nt[q];
            const uint4* pa0 = xu + (m0 + gid) * 2 * kTcWp;
            const uint4* pa1 = xu + (m0 + gid + 8) * 2 * kTcWp;
            const uint4* pb = wu + (n0 + gid) * 2 * kTcWp + tig;
            // W rows c >= k + j are zero (T^{-1} is upper triangular): stop at the last
            // K step that reaches a nonzero row of this N-tile
            const int ks_end = min(nks, (k + n0 + 7) / 16 + 1);
            float acc[kTcSlices][4];
#pragma unroll
            for (int t = 0; t < kTcSlices; ++t)
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[t][i] = 0.f;
#pragma unroll 1
            for (int ks = 0; ks < ks_end; ++ks) {
                const int wa = ks * 8 + (tig ^ fa), wb = ks * 8;
                tc_mma_step(acc, pa0[wa], pa0[wa + kTcWp], pa1[wa], pa1[wa + kTcWp], pa0[wa + 4],
                            pa0[wa + 4 + kTcWp], pa1[wa + 4], pa1[wa + 4 + kTcWp], pb[wb], pb[wb + kTcWp],
                            pb[wb + 4], pb[wb + 4 + kTcWp]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int ro = m0 + gid + ((i & 2) ? 8 : 0);
                const int j = n0 + 2 * tig + (i & 1);
                if (j >= nb || row0 + ro >= n) continue;
                const long long S = tc_combine(acc[0][i], acc[1][i], acc[2][i], acc[3][i], acc[4][i], acc[5][i],
                                               acc[6][i]);
                const int er = rexp[ro], fj = fexp[j];
                const double v = max(er, fj) == kTcBadExp ? __longlong_as_double(0x7FF8000000000000ll)
                                                          : tc_int_to_double(S, er + fj - kTcShift);
                if (DIG) otile[j * kTuRows + ro] = v;
                else V[(size_t)j * ldv + row0 + ro] = v;
            }
        }
        if (DIG) {
            // the new columns in FP64 and in the digit basis: half warp per
            // column, lane h = 4w + g of the half holds rows 16w + 2g, +1, +8, +9
            __syncthreads();
            const int h = lane & 15, w = h >> 2, g = h & 3;
            for (int j0 = 2 * warp; j0 < nb; j0 += 2 * NW) {
                const int j = j0 + (lane >> 4);
                const bool col = j < nb;
                const int jj = col ? j : j0;
                double x[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int rr = 16 * w + 2 * g + (q & 1) + 8 * (q >> 1);
                    x[q] = row0 + rr < n ? otile[jj * kTuRows + rr] : 0.0;
                }
                if (col) {
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const int64_t r0 = row0 + 16 * w + 2 * g + 8 * hh;
                        double* dst = V + (size_t)j * ldv + r0;
                        if (r0 + 1 < n) *reinterpret_cast<double2*>(dst) = make_double2(x[2 * hh], x[2 * hh + 1]);
                        else if (r0 < n) *dst = x[2 * hh];
                    }
                }
                uint4* units = dig + ((size_t)ci * capc + k + jj) * kTcB8Units;
                int* ex = dex + (size_t)ci * tc_dex_stride(capc) + k + jj;
                // a half warp past nb repeats column j0's digits (same values, same bytes)
                tc_b8_store(x, units, ex);
            }
        }
    }
    cp_async_wait_all();
}

}  // namespace gm
