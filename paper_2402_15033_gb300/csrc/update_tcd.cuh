// Narrow block update (nb <= 8) of BCGS-PIP (§IV-C, Fig. 4a, last step) on the
// f16 tensor cores from the digit basis:
//     V <- (V - Q P) T^{-1} = [Q, V] W,   W = [-P T^{-1}; T^{-1}]   (k + nb <= 64).
// The update of the slicing kernel (update_tc.cuh) slices every row of [Q, V]
// against the row's largest exponent; here Q's columns are not sliced at all:
// their digit bytes come from the digit basis, sliced per 64-row chunk against
// each column's own exponent E_c.  Writing X = X' D with D = diag(2^(E_c)) for
// the chunk, X W = X' (D W): the chunk's W'' = D W (k + nb values per output
// column, exact power-of-two scalings of W) is sliced per output column, and
// every digit product then carries the same scale, so the seven FP32
// accumulators stay exact and the output is S * 2^(f_j - 50) rounded once to
// FP64 (tc_common.cuh), f_j the largest exponent of W'' column j.  The new
// block's V columns are sliced per chunk here like Q's in the digit basis, and
// the updated columns' digits are written back to the digit basis, so the
// next block reads them without slicing.
//
// Work per 64-row chunk: copy Q's digit bytes (448 per column, the layout of
// the digit basis, columns 464 bytes apart in shared memory), slice nb
// columns of V into the same layout and nb columns of W'' into f16 B
// fragments, 4 M-tiles x (k-steps over k + nb) MMAs, one warp per M-tile, the
// outputs staged in shared memory and written out with their digits.  A CTA is
// four warps and four CTAs share an SM, so that the slicing phases of one
// chunk (few warps, short dependent chains between barriers) overlap the MMAs
// of the others.  An A fragment takes
// rows r and r + 8 of two K columns from one digit word of each column (one
// byte permute), then widens them (two permutes and two f16x2 subtractions).
#pragma once
#include "pip_body.cuh"
#include "tc_common.cuh"

namespace gm {

constexpr int kUdRows = 64;                   // rows per chunk (= the digit basis chunk)
constexpr int kUdMaxNB = 8;
constexpr int kUdWarps = 4;                   // one warp per 16-row M-tile
constexpr int kUdThreads = 32 * kUdWarps;
constexpr int kUdXw = 116;                    // words per column of X's digit bytes in shared memory (112 + 4 pad)

__host__ __device__ constexpr size_t update_tcd_smem(int kx, int nb) {
    return (size_t)64 * kUdXw * 4                           // X digit bytes (columns past kx: zero digits)
           + (size_t)kUdMaxNB * 2 * kTcWp * 16              // W'' f16 units
           + (size_t)nb * kUdRows * sizeof(double)          // raw V chunk
           + (size_t)kx * nb * sizeof(double)               // W (FP64)
           + (size_t)nb * kUdRows * sizeof(double)          // output tile
           + (64 + kUdMaxNB) * sizeof(int);                 // E_c, f_j
}

// Q(:, 0:k) digits from the digit basis (dig, dex, capc), V(:, 0:nb) raw; the
// updated V and its digits (digit columns k .. k+nb-1) written back.
// kUdThreads threads; 64-row chunks b, b+G, ...
__device__ void update_tcd_body(int64_t n, int k, double* V, int64_t ldv, int nb, const double* __restrict__ R,
                                int ldr, int mode, int b, int G, char* smem, uint4* dig, int* dex, int capc) {
    const int kx = k + nb;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const int nks = (kx + 15) / 16;
    uint32_t* xw = reinterpret_cast<uint32_t*>(smem);                            // [64][kUdXw] digit words
    uint4* wu = reinterpret_cast<uint4*>(xw + 64 * kUdXw);                       // [8][2][kTcWp]
    double* raw = reinterpret_cast<double*>(wu + kUdMaxNB * 2 * kTcWp);          // [nb][64]
    double* W = raw + nb * kUdRows;                                              // [nb][kx]  (W[c + j kx])
    double* otile = W + kx * nb;                                                 // [nb][64]
    int* ec = reinterpret_cast<int*>(otile + nb * kUdRows);                      // [64] chunk column exponents
    int* fj = ec + 64;                                                           // [8]

    // ---- W = [-P T^{-1}; T^{-1}] in FP64 (T^{-1} by substitution; the X region is scratch)
    {
        double* Ts = reinterpret_cast<double*>(xw);
        double* Ti = Ts + nb * nb;
        double* Dinv = Ti + nb * nb;
        const bool notrsm = (mode & kPipNoTrsm) != 0;
        for (int e = tid; e < nb * nb; e += blockDim.x) {
            const int i = e % nb, l = e / nb;
            Ts[e] = notrsm ? (i == l ? 1.0 : 0.0) : (i <= l ? R[(k + i) + (size_t)l * ldr] : 0.0);
        }
        __syncthreads();
        for (int i = tid; i < nb; i += blockDim.x) Dinv[i] = 1.0 / Ts[i + i * nb];
        __syncthreads();
        for (int j = tid; j < nb; j += blockDim.x) {
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
            W[e] = w;
        }
        __syncthreads();
    }
    // columns past kx read by the last k-step hold zero digits (biased 0x80)
    for (int e = tid; e < 64 * kUdXw; e += blockDim.x) xw[e] = 0x80808080u;
    for (int e = tid; e < kUdMaxNB * 2 * kTcWp; e += blockDim.x) wu[e] = make_uint4(0u, 0u, 0u, 0u);

    // warp t: tile t (rows 16t .. 16t+15), every k-step
    const int t = warp;
    const int m0 = 16 * t;
    // rows m0 + gid and + 8 are bytes (gid & 1) and 2 + (gid & 1) of word t of unit
    // 4p + gid / 2; one permute takes them from columns c and c + 1
    const uint32_t sel = (gid & 1) ? 0x7351u : 0x6240u;
    const int uoff = (gid >> 1) * 4 + t;                   // word of digit 0 within a column

    const int64_t nchunks = (n + kUdRows - 1) / kUdRows;
    // raw V: rows 2(tid % 32), +1 of columns warp, warp + 4, ...
    auto stage_v = [&](int64_t ch) {
        const int64_t row = ch * kUdRows + 2 * lane;
        const int bytes = row + 2 <= n ? 16 : (row < n ? 8 : 0);
        for (int j = warp; j < nb; j += kUdWarps) {
            const double* p = V + (int64_t)j * ldv + row;
            cp_async16(raw + j * kUdRows + 2 * lane, bytes ? (const void*)p : (const void*)V, bytes);
        }
        cp_async_commit();
    };
    // Q's digit bytes and exponents of chunk ch from the digit basis (issued a
    // chunk ahead, as soon as the previous chunk's MMAs are done with xw)
    auto stage_q = [&](int64_t ch) {
        const uint4* src = dig + (size_t)ch * capc * kTcB8Units;
        for (int e = tid; e < k * kTcB8Units; e += blockDim.x) {
            const int c = e / kTcB8Units, u = e - c * kTcB8Units;
            cp_async16(xw + c * kUdXw + 4 * u, src + e, 16);
        }
        cp_async_commit();
        for (int c = tid; c < k; c += blockDim.x) ec[c] = dex[(size_t)ch * tc_dex_stride(capc) + c];
    };
    __syncthreads();
    if ((int64_t)b < nchunks) {
        stage_v(b);
        stage_q(b);
    }
    const int h = lane & 15, hw_w = h >> 2, hw_g = h & 3;   // half-warp roles (rows 16w + 2g, +1, +8, +9)
    for (int64_t ci = b; ci < nchunks; ci += G) {
        const int64_t row0 = ci * kUdRows;
        cp_async_wait_all();
        __syncthreads();
        // 1. V's columns sliced into digit bytes next to Q's (half warp per column)
        for (int j0 = 2 * warp; j0 < nb; j0 += 2 * kUdWarps) {
            const int jj = j0 + (lane >> 4) < nb ? j0 + (lane >> 4) : j0;
            double x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) x[q] = raw[jj * kUdRows + 16 * hw_w + 2 * hw_g + (q & 1) + 8 * (q >> 1)];
            tc_b8_store(x, reinterpret_cast<uint4*>(xw + (k + jj) * kUdXw), ec + k + jj);
        }
        __syncthreads();
        // the raw tile is free: the next chunk's V streams in
        if (ci + G < nchunks) stage_v(ci + G);
        // 2. W'' = D W per output column j (lane = K pair: rows 2l, 2l+1 of W''),
        //    sliced against its largest exponent f_j
        for (int j = warp; j < nb; j += kUdWarps) {
            const int c0 = 2 * lane, c1 = 2 * lane + 1;
            const double w0 = c0 < kx ? W[c0 + j * kx] : 0.0, w1 = c1 < kx ? W[c1 + j * kx] : 0.0;
            const int e0 = c0 < kx ? ec[c0] : 0, e1 = c1 < kx ? ec[c1] : 0;
            const int b0 = tc_bexp(w0), b1 = tc_bexp(w1);
            int bad = (e0 == kTcBadExp || e1 == kTcBadExp || b0 == 0x7FF || b1 == 0x7FF) ? 1 : 0;
            int f = -100000;
            if (b0 && e0 != kTcBadExp) f = max(f, b0 + e0);
            if (b1 && e1 != kTcBadExp) f = max(f, b1 + e1);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                f = max(f, __shfl_xor_sync(0xffffffffu, f, off));
                bad |= __shfl_xor_sync(0xffffffffu, bad, off);
            }
            if (f == -100000) f = 1023;
            if (lane == 0) fj[j] = bad ? kTcBadExp : f - 1023;
            tc_pack(tc_slice(e0 == kTcBadExp ? 0.0 : w0, f - e0), tc_slice(e1 == kTcBadExp ? 0.0 : w1, f - e1),
                    wu[(j * 2) * kTcWp + lane], wu[(j * 2 + 1) * kTcWp + lane]);
        }
        __syncthreads();
        // 3. MMAs of tile t over this warp's k-steps: A = X (rows x K columns) from
        //    the column-major digit bytes, B = W''
        float acc[kTcSlices][4];
#pragma unroll
        for (int q = 0; q < kTcSlices; ++q)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[q][e] = 0.f;
#pragma unroll 1
        for (int ks = 0; ks < nks; ++ks) {
            const int ca = 16 * ks + 2 * tig;     // K columns ca, ca+1 (a0, a1) and ca+8, ca+9 (a2, a3)
            const uint32_t* x0 = xw + ca * kUdXw + uoff;
            const uint4* pb = wu + gid * 2 * kTcWp + ks * 8 + tig;
            const uint4 b0l = pb[0], b0h = pb[kTcWp], b1l = pb[4], b1h = pb[4 + kTcWp];
            const uint32_t B[kTcSlices][2] = {{b0l.x, b1l.x}, {b0l.y, b1l.y}, {b0l.z, b1l.z}, {b0l.w, b1l.w},
                                              {b0h.x, b1h.x}, {b0h.y, b1h.y}, {b0h.z, b1h.z}};
#pragma unroll
            for (int p = 0; p < kTcSlices; ++p) {
                const uint32_t* xp = x0 + 16 * p;
                const uint32_t v01 = __byte_perm(xp[0], xp[kUdXw], sel);
                const uint32_t v89 = __byte_perm(xp[8 * kUdXw], xp[9 * kUdXw], sel);
                const uint32_t a0 = tc_widen<0x4140>(v01), a1 = tc_widen<0x4342>(v01);
                const uint32_t a2 = tc_widen<0x4140>(v89), a3 = tc_widen<0x4342>(v89);
#pragma unroll
                for (int r = 0; r < kTcSlices - p; ++r) mma_f16_16816(acc[p + r], a0, a1, a2, a3, B[r][0], B[r][1]);
            }
        }
        // 4. the outputs S * 2^(f_j - 50), S from the seven exact sums
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int r = m0 + gid + ((e & 2) ? 8 : 0);
            const int j = 2 * tig + (e & 1);
            if (j >= nb) continue;
            const long long S =
                tc_combine(acc[0][e], acc[1][e], acc[2][e], acc[3][e], acc[4][e], acc[5][e], acc[6][e]);
            const int f = fj[j];
            otile[j * kUdRows + r] = f == kTcBadExp ? __longlong_as_double(0x7FF8000000000000ll)
                                                    : tc_int_to_double(S, f - kTcShift);
        }
        __syncthreads();
        // every MMA is done with xw: the next chunk's Q digits stream in during the
        // column pass and the next chunk's slicing
        if (ci + G < nchunks) stage_q(ci + G);
        // 5. the new columns: FP64 rows and their digits (half warp per column)
        for (int j0 = 2 * warp; j0 < nb; j0 += 2 * kUdWarps) {
            const int j = j0 + (lane >> 4);
            const int jj = j < nb ? j : j0;
            double x[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int rr = 16 * hw_w + 2 * hw_g + (q & 1) + 8 * (q >> 1);
                x[q] = row0 + rr < n ? otile[jj * kUdRows + rr] : 0.0;
            }
            if (j < nb) {
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int64_t r0 = row0 + 16 * hw_w + 2 * hw_g + 8 * hh;
                    double* dst = V + (size_t)j * ldv + r0;
                    if (r0 + 1 < n) *reinterpret_cast<double2*>(dst) = make_double2(x[2 * hh], x[2 * hh + 1]);
                    else if (r0 < n) *dst = x[2 * hh];
                }
            }
            tc_b8_store(x, dig + ((size_t)ci * capc + k + jj) * kTcB8Units,
                        dex + (size_t)ci * tc_dex_stride(capc) + k + jj);
        }
    }
    cp_async_wait_all();
}

}  // namespace gm
