// Device bodies of the BCGS-PIP kernels (§IV-C, Fig. 4a), shared by the
// single-system launchers (pip.cu) and the batched engine (batch.cu).
//
// A Gram reduction is split over n into G "virtual CTAs": virtual CTA b
// reduces the interleaved 128-row (skinny) or 32-row (wide) chunks
// b, b+G, b+2G, ... of its system into one partial block (slot).  The last
// virtual CTA to arrive sums the G slots in index order and, unless told not
// to, factors G - P^T P.  The split depends only on the system's n, so a
// system gives bit-identical results alone or inside a batch.
#pragma once
#include "common.cuh"
#include "df.cuh"

namespace gm {

constexpr int kSkinnyRows = 128;   // rows per chunk, skinny path (nb <= 12)
constexpr int kWideRows = 32;      // rows per chunk, wide path
constexpr int kSLd = kMaxNB + 1;   // leading dimension of the factor in shared memory
constexpr int kSkinnyMaxNB = 12;   // wider blocks would spill 8 x nb accumulators per thread
constexpr size_t kGramSmem =
    (2 * kMaxNB * (kWideRows + 1) > kMaxNB * kSLd ? 2 * kMaxNB * (kWideRows + 1) : kMaxNB * kSLd) * sizeof(double);
static_assert(kMaxNB * kSLd >= kSkinnyMaxNB * kSkinnyRows, "skinny staging fits the epilogue buffer");

template <typename T>
__device__ __forceinline__ const T* col_ptr(const T* Q, int64_t ldq, int k, const T* V, int64_t ldv, int c) {
    return c < k ? Q + (int64_t)c * ldq : V + (int64_t)(c - k) * ldv;
}

__device__ __forceinline__ double ld_d(const double* p) { return __ldg(p); }
__device__ __forceinline__ double ld_d(const float* p) { return (double)__ldg(p); }

// Entry (c, j) of the (k+nb) x nb block [P; G] is needed unless it lies strictly
// below the diagonal of the symmetric G block.
__device__ __forceinline__ bool needed(int c, int j, int k) { return c < k || (c - k) <= j; }

// Skinny path, nb <= 12: warp w owns the group's columns w, w+8, ...; lane l owns
// rows l, l+32, ... of each chunk; the V chunk is staged in shared memory.
template <typename T, int NB>
__device__ void gram_skinny_part(int64_t n, const T* __restrict__ Q, int64_t ldq, int k,
                                 const T* __restrict__ V, int64_t ldv, int g, int b, int G,
                                 double* slot, double* smem) {
    const int kx = k + NB;
    const int ccount = min(kMaxNB, kx - g * kMaxNB);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int CPW = kMaxNB / 8;

    const T* xp[CPW];
#pragma unroll
    for (int i = 0; i < CPW; ++i) {
        const int cl = warp + 8 * i;
        xp[i] = cl < ccount ? col_ptr(Q, ldq, k, V, ldv, g * kMaxNB + cl) : nullptr;
    }
    double acc[CPW][NB];
#pragma unroll
    for (int i = 0; i < CPW; ++i)
#pragma unroll
        for (int j = 0; j < NB; ++j) acc[i][j] = 0.0;

    double* Ys = smem;  // [NB][kSkinnyRows]
    const int64_t nchunks = (n + kSkinnyRows - 1) / kSkinnyRows;
    for (int64_t ci = b; ci < nchunks; ci += G) {
        const int64_t row0 = ci * kSkinnyRows;
        __syncthreads();
        for (int e = threadIdx.x; e < NB * kSkinnyRows; e += blockDim.x) {
            const int j = e / kSkinnyRows, r = e % kSkinnyRows;
            const int64_t row = row0 + r;
            Ys[e] = row < n ? ld_d(V + (int64_t)j * ldv + row) : 0.0;
        }
        __syncthreads();
#pragma unroll 1
        for (int u = 0; u < kSkinnyRows / 32; ++u) {
            const int r = u * 32 + lane;
            const int64_t row = row0 + r;
            double v[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) v[j] = Ys[j * kSkinnyRows + r];
            const bool in = row < n;
#pragma unroll
            for (int i = 0; i < CPW; ++i) {
                if (xp[i] != nullptr) {
                    const double x = in ? ld_d(xp[i] + row) : 0.0;
#pragma unroll
                    for (int j = 0; j < NB; ++j) acc[i][j] = fma(x, v[j], acc[i][j]);
                }
            }
        }
    }
    // warp fold (fixed butterfly order) into the slot
#pragma unroll
    for (int i = 0; i < CPW; ++i) {
        if (xp[i] == nullptr) continue;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            double a = acc[i][j];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
            if (lane == 0) slot[(warp + 8 * i) * NB + j] = a;
        }
    }
}

// Wide path, nb <= 64: each thread owns a 4 x 4 tile of the group's (<= 64) x nb
// block; tiles strictly below the diagonal of the symmetric G block are skipped
// and the remaining tiles are packed onto the first threads.
template <typename T>
__device__ void gram_wide_part(int64_t n, const T* __restrict__ Q, int64_t ldq, int k,
                               const T* __restrict__ V, int64_t ldv, int nb, int g, int b, int G,
                               double* slot, double* smem) {
    const int kx = k + nb;
    const int cg0 = g * kMaxNB;
    const int ccount = min(kMaxNB, kx - cg0);
    constexpr int LD = kWideRows + 1;
    double* Xs = smem;                   // [64][LD]
    double* Ys = smem + kMaxNB * LD;     // [64][LD]

    int my_bi = -1, my_bj = -1;
    {
        int cnt = 0;
        const int nbi = (ccount + 3) / 4, nbj = (nb + 3) / 4;
        for (int bj = 0; bj < nbj && my_bi < 0; ++bj)
            for (int bi = 0; bi < nbi; ++bi) {
                const bool lower = (cg0 + 4 * bi - k) > (4 * bj + 3);
                if (lower) continue;
                if (cnt == (int)threadIdx.x) { my_bi = bi; my_bj = bj; break; }
                ++cnt;
            }
    }
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = 0.0;

    const int64_t nchunks = (n + kWideRows - 1) / kWideRows;
    for (int64_t ci = b; ci < nchunks; ci += G) {
        const int64_t row0 = ci * kWideRows;
        __syncthreads();
        for (int e = threadIdx.x; e < (ccount + nb) * kWideRows; e += blockDim.x) {
            const int c = e / kWideRows, r = e % kWideRows;
            const int64_t row = row0 + r;
            double v = 0.0;
            if (row < n) {
                const T* p = c < ccount ? col_ptr(Q, ldq, k, V, ldv, cg0 + c)
                                        : V + (int64_t)(c - ccount) * ldv;
                v = ld_d(p + row);
            }
            if (c < ccount) Xs[c * LD + r] = v; else Ys[(c - ccount) * LD + r] = v;
        }
        __syncthreads();
        if (my_bi >= 0) {
            const double* xs = Xs + 4 * my_bi * LD;
            const double* ys = Ys + 4 * my_bj * LD;
#pragma unroll 4
            for (int r = 0; r < kWideRows; ++r) {
                double a[4], c[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) { a[t] = xs[t * LD + r]; c[t] = ys[t * LD + r]; }
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int t = 0; t < 4; ++t) acc[s][t] = fma(a[s], c[t], acc[s][t]);
            }
        }
    }
    // entries outside [ccount) x [nb) multiply zero-filled or stale shared rows; drop them
    if (my_bi >= 0) {
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int cl = 4 * my_bi + s, j = 4 * my_bj + t;
                if (cl < ccount && j < nb) slot[cl * nb + j] = acc[s][t];
            }
    }
}

// Arrival and last-arrival work of column group g (of `groups`): the virtual CTA
// that completes the group sums its G slots (partial0 + b * ps, b = 0..G-1) in
// order into `gram`; the last group to complete forms S = G - P^T P and factors
// it (kernel (d)), or, with kPipGramOnly, writes [P; G] unfactored.  R = [P; T].
// With kPipShift the factored matrix is G - P^T P + sigma I, the shift of
// shifted CholQR (Fukaya, Kannan, Nakatsukasa, Zhang and Yamamoto, 2020; §II):
// sigma = 11 (nrows nb + nb (nb + 1)) u trace(G), u = 2^-53, where trace(G) =
// ||V||_F^2 bounds the block's squared 2-norm from above.
// counter holds groups + 1 arrival counters; every counter is re-armed to zero.
__device__ inline void pip_finish(int k, int nb, int g, int groups, int G, double* R, int ldr,
                                  const double* partial0, size_t ps, unsigned* counter, double* gram,
                                  int32_t* d_status, int32_t* d_skip, double* smem, int mode, int64_t nrows = 0) {
    __shared__ unsigned s_ticket;
    __shared__ int s_info;
    __shared__ double s_inv;
    const int tid = threadIdx.x;
    const int kx = k + nb;
    const int ccount = min(kMaxNB, kx - g * kMaxNB);

    __threadfence();
    __syncthreads();
    if (tid == 0) s_ticket = atomicAdd(&counter[g], 1u);
    __syncthreads();
    if (s_ticket != (unsigned)(G - 1)) return;
    __threadfence();

    // fixed-order second-level reduce of this group's slots
    for (int e = tid; e < ccount * nb; e += blockDim.x) {
        const int cl = e / nb, j = e % nb;
        const int c = g * kMaxNB + cl;
        if (!needed(c, j, k)) continue;
        const double* p = partial0 + e;
        double acc = 0.0;
#pragma unroll 8
        for (int bb = 0; bb < G; ++bb) acc += __ldcg(p + (size_t)bb * ps);
        gram[c + (size_t)j * kx] = acc;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        counter[g] = 0u;  // re-arm for the next call
        s_ticket = (groups == 1) ? 0u : atomicAdd(&counter[groups], 1u) - (unsigned)(groups - 1);
    }
    __syncthreads();
    if (s_ticket != 0u) return;   // another group's last arrival factors the Gram
    __threadfence();
    if (tid == 0 && groups > 1) counter[groups] = 0u;

    if (mode & kPipGramOnly) {
        // [P; G] as reduced (upper triangle of G), no factorization
        for (int e = tid; e < (k + nb) * nb; e += blockDim.x) {
            const int c = e % (k + nb), j = e / (k + nb);
            R[c + (size_t)j * ldr] = needed(c, j, k) ? __ldcg(gram + c + (size_t)j * kx) : 0.0;
        }
        if (tid == 0) *d_status = 0;
        return;
    }

    // S = G - P^T P (upper triangle), Pythagorean update of the Gram (Fig. 4a)
    double* S = smem;  // nb x nb, column-major, ld kSLd
    __syncthreads();
    for (int e = tid; e < nb * nb; e += blockDim.x) {
        const int i = e % nb, j = e / nb;
        if (i > j) continue;
        // the k terms subtracted in order; eight terms' loads are issued together
        const double* gi = gram + (size_t)i * kx;
        const double* gj = gram + (size_t)j * kx;
        double acc = __ldcg(gram + (k + i) + (size_t)j * kx);
        int l = 0;
        for (; l + 8 <= k; l += 8) {
            double x[8], y[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                x[q] = __ldcg(gi + l + q);
                y[q] = __ldcg(gj + l + q);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) acc -= x[q] * y[q];
        }
        for (; l < k; ++l) acc -= __ldcg(gi + l) * __ldcg(gj + l);
        S[i + j * kSLd] = acc;
    }
    if (tid == 0) s_info = 0;
    __syncthreads();
    if (mode & kPipShift) {
        if (tid == 0) {
            double tr = 0.0;
            for (int j = 0; j < nb; ++j) tr += __ldcg(gram + (k + j) + (size_t)j * kx);
            const double sig = 11.0 * ((double)nrows * nb + (double)nb * (nb + 1)) * 0x1p-53 * tr;
            for (int j = 0; j < nb; ++j) S[j + j * kSLd] += sig;
        }
        __syncthreads();
    }

    // right-looking Cholesky S = T^T T in shared memory (kernel (d))
    for (int j = 0; j < nb; ++j) {
        if (tid == 0) {
            const double d = S[j + j * kSLd];
            if (!(d > 0.0)) {
                s_info = j + 1;
            } else {
                const double r = sqrt(d);
                S[j + j * kSLd] = r;
                s_inv = 1.0 / r;
            }
        }
        __syncthreads();
        if (s_info) break;
        const double inv = s_inv;
        for (int l = j + 1 + tid; l < nb; l += blockDim.x) S[j + l * kSLd] *= inv;
        __syncthreads();
        const int rem = nb - j - 1;
        for (int p = tid; p < rem * rem; p += blockDim.x) {
            const int i = j + 1 + p % rem, l = j + 1 + p / rem;
            if (i <= l) S[i + l * kSLd] -= S[j + i * kSLd] * S[j + l * kSLd];
        }
        __syncthreads();
    }
    const int info = s_info;

    // R = [P; T]
    for (int e = tid; e < (k + nb) * nb; e += blockDim.x) {
        const int c = e % (k + nb), j = e / (k + nb);
        double v;
        if (c < k) {
            v = __ldcg(gram + c + (size_t)j * kx);
        } else {
            const int i = c - k;
            v = (i <= j) ? S[i + j * kSLd] : 0.0;
        }
        R[c + (size_t)j * ldr] = v;
    }
    if (tid == 0) {
        *d_status = info;
        if (info && d_skip) *d_skip = 1;   // the rest of a solver cycle stands down
    }
}

// P (k x NB, row-major [c][j]) and T (NB x NB, [i][j]) of R staged in shared
// memory, and 1/T_jj; with kPipNoTrsm T is the identity.
template <int NB>
__device__ void stage_pt(int k, const double* R, int ldr, int mode, double* Ps, double* Ts, double* Dinv) {
    for (int e = threadIdx.x; e < k * NB; e += blockDim.x) {
        const int c = e / NB, j = e % NB;
        Ps[e] = R[c + (size_t)j * ldr];
    }
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, j = e % NB;
        Ts[e] = (mode & kPipNoTrsm) ? (i == j ? 1.0 : 0.0) : R[(k + i) + (size_t)j * ldr];
    }
    __syncthreads();
    if (threadIdx.x < NB) Dinv[threadIdx.x] = 1.0 / Ts[threadIdx.x * NB + threadIdx.x];
    __syncthreads();
}

// One row of the skinny update: v <- (v - q P) T^{-1}, FP64 arithmetic.
template <typename T, int NB>
__device__ __forceinline__ void update_row(int64_t row, const T* __restrict__ Q, int64_t ldq, int k,
                                           T* __restrict__ V, int64_t ldv, const double* Ps, const double* Ts,
                                           const double* Dinv) {
    double w[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) w[j] = (double)V[(int64_t)j * ldv + row];
    for (int c = 0; c < k; ++c) {
        const double q = ld_d(Q + (int64_t)c * ldq + row);
#pragma unroll
        for (int j = 0; j < NB; ++j) w[j] = fma(-q, Ps[c * NB + j], w[j]);
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        double s = w[j];
#pragma unroll
        for (int i = 0; i < j; ++i) s = fma(-w[i], Ts[i * NB + j], s);
        w[j] = s * Dinv[j];
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) V[(int64_t)j * ldv + row] = (T)w[j];
}

// One row of the wide update (16 < nb <= 64): the row of V in registers, T in
// shared memory (ld kMaxNB), P read through the read-only cache.
template <typename T>
__device__ __forceinline__ void update_row_wide(int64_t row, const T* __restrict__ Q, int64_t ldq, int k,
                                                T* __restrict__ V, int64_t ldv, int nb, const double* __restrict__ R,
                                                int ldr, const double* Ts, const double* Dinv) {
    double w[kMaxNB];
#pragma unroll
    for (int j = 0; j < kMaxNB; ++j) w[j] = j < nb ? (double)V[(int64_t)j * ldv + row] : 0.0;
    for (int c = 0; c < k; ++c) {
        const double q = ld_d(Q + (int64_t)c * ldq + row);
        const double* pr = R + c;
#pragma unroll
        for (int j = 0; j < kMaxNB; ++j)
            if (j < nb) w[j] = fma(-q, __ldg(pr + (size_t)j * ldr), w[j]);
    }
#pragma unroll
    for (int j = 0; j < kMaxNB; ++j) {
        if (j < nb) {
            double s = w[j];
#pragma unroll
            for (int i = 0; i < j; ++i) s = fma(-w[i], Ts[i * kMaxNB + j], s);
            w[j] = s * Dinv[j];
        }
    }
#pragma unroll
    for (int j = 0; j < kMaxNB; ++j)
        if (j < nb) V[(int64_t)j * ldv + row] = (T)w[j];
}

// T (ld kMaxNB) and 1/T_jj of R staged for the wide update.
__device__ inline void stage_t_wide(int k, int nb, const double* R, int ldr, int mode, double* Ts, double* Dinv) {
    for (int e = threadIdx.x; e < kMaxNB * kMaxNB; e += blockDim.x) {
        const int i = e / kMaxNB, j = e % kMaxNB;
        Ts[e] = (i < nb && j < nb) ? ((mode & kPipNoTrsm) ? (i == j ? 1.0 : 0.0) : R[(k + i) + (size_t)j * ldr])
                                   : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < kMaxNB) Dinv[threadIdx.x] = threadIdx.x < nb ? 1.0 / Ts[threadIdx.x * (kMaxNB + 1)] : 0.0;
    __syncthreads();
}

// ================================================================= double-float bodies
// The same reductions and updates with FP32-pipe double-float arithmetic
// (df.cuh): products error-free, sums renormalized, ~2^-48 relative accuracy.

constexpr int kDfSkinnyMaxNB = 8;    // 8 columns x NB double-float accumulators per thread
constexpr int kDfWideRows = 64;      // rows per tile of the wide update

// ---------------------------------------------------------------- asynchronous staging
// 16-byte global -> shared copies that bypass registers (cp.async), committed
// as one group per chunk; src_bytes < 16 zero-fills the rest of the 16 bytes.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gsrc), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Issue the copies of `cols` columns x `rows` rows (rows even) starting at row0
// into a column-major shared tile of leading dimension `rows` (one element =
// 8 bytes for FP64 data; FP32 data packs two rows per 8 bytes).  Rows at or
// beyond n are zero-filled.  Column c < k comes from Q, else from V.
template <typename T>
__device__ __forceinline__ void stage_chunk_async(const T* Q, int64_t ldq, int k, const T* V, int64_t ldv,
                                                  int c0, int cols, int64_t row0, int rows, int64_t n, T* tile) {
    constexpr int per16 = 16 / sizeof(T);            // elements per 16-byte copy
    const int pieces = rows / per16;
    for (int e = threadIdx.x; e < cols * pieces; e += blockDim.x) {
        const int c = e / pieces, q = e % pieces;
        const int64_t row = row0 + (int64_t)q * per16;
        const T* src = col_ptr(Q, ldq, k, V, ldv, c0 + c);
        int bytes = 0;
        if (row < n) bytes = (int)(min((int64_t)per16, n - row) * sizeof(T));
        cp_async16(tile + (size_t)c * rows + (size_t)q * per16, bytes ? (const void*)(src + row) : (const void*)src,
                   bytes);
    }
}

// Split a staged tile in place: each 8-byte FP64 element becomes its (hi, lo)
// float pair; FP32 tiles are widened into a separate float2 tile instead.
__device__ __forceinline__ void split_tile_inplace(double* tile, int count) {
    for (int e = threadIdx.x; e < count; e += blockDim.x) {
        float h, l;
        split_f64(tile[e], h, l);
        reinterpret_cast<float2*>(tile)[e] = make_float2(h, l);
    }
}

// Skinny Gram, nb <= 8, double-float: 128-row chunks of [Q, V] staged in shared
// memory by asynchronous copies, double buffered (the next chunk streams in
// while the current one is reduced), split to (hi, lo) pairs in place; warp w
// owns the group's columns w, w+8, ...; lane l owns rows l, l+32, ...; the V
// values of a row are read from the same tile.  Shared memory: 2 x (k+NB) x 128
// x 8 bytes (<= 132 KB for k+NB = 64).
template <typename T, int NB>
__device__ void gram_skinny_part_df(int64_t n, const T* __restrict__ Q, int64_t ldq, int k,
                                    const T* __restrict__ V, int64_t ldv, int g, int b, int G,
                                    double* slot, double* smem) {
    const int kx = k + NB;
    const int cg0 = g * kMaxNB;
    const int ccount = min(kMaxNB, kx - cg0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int CPW = kMaxNB / 8;
    constexpr int RW = kSkinnyRows;
    // tile columns: the group's ccount X columns, then the NB V columns
    const int tcols = ccount + NB;
    const size_t tile_elems = (size_t)tcols * RW;
    DD acc[CPW][NB];
#pragma unroll
    for (int i = 0; i < CPW; ++i)
#pragma unroll
        for (int j = 0; j < NB; ++j) acc[i][j] = DD{0.f, 0.f};

    const int64_t nchunks = (n + RW - 1) / RW;
    // FP64: two raw 8-byte tiles, split in place.  FP32: two raw 4-byte tiles
    // after one float2 compute tile, widened from the raw tile each chunk.
    double* f2tile = smem;                                          // FP32 only
    T* raw[2];
    if (sizeof(T) == sizeof(double)) {
        raw[0] = reinterpret_cast<T*>(smem);
        raw[1] = reinterpret_cast<T*>(smem + tile_elems);
    } else {
        raw[0] = reinterpret_cast<T*>(smem + tile_elems);
        raw[1] = raw[0] + tile_elems;
    }
    auto issue = [&](int64_t ci, T* tile) {
        const int64_t row0 = ci * RW;
        stage_chunk_async<T>(Q, ldq, k, V, ldv, cg0, ccount, row0, RW, n, tile);
        stage_chunk_async<T>(V, ldv, 0, V, ldv, 0, NB, row0, RW, n, tile + (size_t)ccount * RW);
        cp_async_commit();
    };
    int cur = 0;
    if ((int64_t)b < nchunks) issue(b, raw[0]);
    for (int64_t ci = b; ci < nchunks; ci += G) {
        cp_async_wait_all();
        __syncthreads();
        double* tile;
        if (sizeof(T) == sizeof(double)) {
            tile = reinterpret_cast<double*>(raw[cur]);
            split_tile_inplace(tile, (int)tile_elems);
        } else {
            tile = f2tile;
            const float* t32 = reinterpret_cast<const float*>(raw[cur]);
            for (int e = threadIdx.x; e < (int)tile_elems; e += blockDim.x)
                reinterpret_cast<float2*>(tile)[e] = make_float2(t32[e], 0.f);
        }
        __syncthreads();
        if (ci + G < nchunks) issue(ci + G, raw[cur ^ 1]);   // overlaps the reduction below
        const float2* tf = reinterpret_cast<const float2*>(tile);
#pragma unroll 1
        for (int u = 0; u < RW / 32; ++u) {
            const int r = u * 32 + lane;
            float2 v[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) v[j] = tf[(size_t)(ccount + j) * RW + r];
#pragma unroll
            for (int i = 0; i < CPW; ++i) {
                const int cl = warp + 8 * i;
                if (cl < ccount) {
                    const float2 x = tf[(size_t)cl * RW + r];
#pragma unroll
                    for (int j = 0; j < NB; ++j) {
                        if (sizeof(T) == sizeof(float)) dd_mac1(acc[i][j], x.x, v[j].x, v[j].y);
                        else dd_mac(acc[i][j], x.x, x.y, v[j].x, v[j].y);
                    }
                }
            }
        }
        cur ^= 1;
    }
    cp_async_wait_all();
    __syncthreads();
#pragma unroll
    for (int i = 0; i < CPW; ++i) {
        const int cl = warp + 8 * i;
        if (cl >= ccount) continue;
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            double a = dd_value(acc[i][j]);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
            if (lane == 0) slot[cl * NB + j] = a;
        }
    }
}

// Shared memory of gram_skinny_part_df: two 128-row stages of the group's
// columns plus the NB V columns (FP64: 2 x 8 bytes per element; FP32: two 4-byte
// raw stages and one 8-byte compute tile), and at least what pip_finish needs.
__host__ __device__ constexpr size_t gram_skinny_df_smem(int tcols) {
    return (2 * (size_t)tcols * kSkinnyRows * sizeof(double)) > kGramSmem
               ? 2 * (size_t)tcols * kSkinnyRows * sizeof(double) : kGramSmem;
}

// Wide Gram, nb <= 64: 4 x 4 double-float tiles per thread, chunks staged pre-split.
template <typename T>
__device__ void gram_wide_part_df(int64_t n, const T* __restrict__ Q, int64_t ldq, int k,
                                  const T* __restrict__ V, int64_t ldv, int nb, int g, int b, int G,
                                  double* slot, double* smem) {
    const int kx = k + nb;
    const int cg0 = g * kMaxNB;
    const int ccount = min(kMaxNB, kx - cg0);
    constexpr int LD = kWideRows + 1;
    float2* Xs = reinterpret_cast<float2*>(smem);          // [64][LD]
    float2* Ys = Xs + kMaxNB * LD;                          // [64][LD]
    int my_bi = -1, my_bj = -1;
    {
        int cnt = 0;
        const int nbi = (ccount + 3) / 4, nbj = (nb + 3) / 4;
        for (int bj = 0; bj < nbj && my_bi < 0; ++bj)
            for (int bi = 0; bi < nbi; ++bi) {
                const bool lower = (cg0 + 4 * bi - k) > (4 * bj + 3);
                if (lower) continue;
                if (cnt == (int)threadIdx.x) { my_bi = bi; my_bj = bj; break; }
                ++cnt;
            }
    }
    DD acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = DD{0.f, 0.f};
    const int64_t nchunks = (n + kWideRows - 1) / kWideRows;
    for (int64_t ci = b; ci < nchunks; ci += G) {
        const int64_t row0 = ci * kWideRows;
        __syncthreads();
        for (int e = threadIdx.x; e < (ccount + nb) * kWideRows; e += blockDim.x) {
            const int c = e / kWideRows, r = e % kWideRows;
            const int64_t row = row0 + r;
            float h = 0.f, l = 0.f;
            if (row < n) {
                const T* p = c < ccount ? col_ptr(Q, ldq, k, V, ldv, cg0 + c)
                                        : V + (int64_t)(c - ccount) * ldv;
                split_val(__ldg(p + row), h, l);
            }
            if (c < ccount) Xs[c * LD + r] = make_float2(h, l); else Ys[(c - ccount) * LD + r] = make_float2(h, l);
        }
        __syncthreads();
        if (my_bi >= 0) {
            const float2* xs = Xs + 4 * my_bi * LD;
            const float2* ys = Ys + 4 * my_bj * LD;
#pragma unroll 2
            for (int r = 0; r < kWideRows; ++r) {
                float2 a[4], c[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) { a[t] = xs[t * LD + r]; c[t] = ys[t * LD + r]; }
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        if (sizeof(T) == sizeof(float)) dd_mac1(acc[s][t], a[s].x, c[t].x, c[t].y);
                        else dd_mac(acc[s][t], a[s].x, a[s].y, c[t].x, c[t].y);
                    }
            }
        }
    }
    if (my_bi >= 0) {
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int cl = 4 * my_bi + s, j = 4 * my_bj + t;
                if (cl < ccount && j < nb) slot[cl * nb + j] = dd_value(acc[s][t]);
            }
    }
}

// W = [-P T^{-1}; T^{-1}] ((k+nb) x nb, FP64 from R), split into (hi, lo) pairs
// in shared memory at Ws[c * ldw + pos(j)]; with kPipNoTrsm, W = [-P; I].
// pos(j) = j, or, with interleave > 1, (j % grp) * interleave + j / grp where
// grp = 64 / interleave (conflict-free reads by `interleave` output groups).
// Tinv: nb x nb FP64 scratch in shared memory.
__device__ inline void stage_w_df(int k, int nb, const double* __restrict__ R, int ldr, int mode, float2* Ws,
                                  int ldw, int interleave, double* Tinv) {
    const bool notrsm = (mode & kPipNoTrsm) != 0;
    // T^{-1} one column per thread (upper triangular back substitution)
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        for (int i = 0; i < nb; ++i) Tinv[i * nb + j] = 0.0;
        if (notrsm) { Tinv[j * nb + j] = 1.0; continue; }
        Tinv[j * nb + j] = 1.0 / R[(k + j) + (size_t)j * ldr];
        for (int i = j - 1; i >= 0; --i) {
            double acc = 0.0;
            for (int l = i + 1; l <= j; ++l) acc = fma(R[(k + i) + (size_t)l * ldr], Tinv[l * nb + j], acc);
            Tinv[i * nb + j] = -acc / R[(k + i) + (size_t)i * ldr];
        }
    }
    __syncthreads();
    const int grp = interleave > 1 ? kMaxNB / interleave : 0;
    for (int e = threadIdx.x; e < (k + nb) * nb; e += blockDim.x) {
        const int c = e / nb, j = e % nb;
        double w;
        if (c < k) {
            double acc = 0.0;
            for (int i = 0; i <= j; ++i) acc = fma(R[c + (size_t)i * ldr], Tinv[i * nb + j], acc);
            w = -acc;
        } else {
            w = Tinv[(c - k) * nb + j];
        }
        float h, l;
        split_f64(w, h, l);
        const int pj = interleave > 1 ? (j % grp) * interleave + j / grp : j;
        Ws[c * ldw + pj] = make_float2(h, l);
    }
    __syncthreads();
}

// One row of the double-float update: v_j <- sum_c x_c W[c][j], x = [q, v].
template <typename T, int NB>
__device__ __forceinline__ void update_row_df(int64_t row, const T* __restrict__ Q, int64_t ldq, int k,
                                              T* __restrict__ V, int64_t ldv, const float2* Ws) {
    DD acc[NB];
#pragma unroll
    for (int j = 0; j < NB; ++j) acc[j] = DD{0.f, 0.f};
    for (int c = 0; c < k + NB; ++c) {
        const T xv = c < k ? __ldg(Q + (int64_t)c * ldq + row) : V[(int64_t)(c - k) * ldv + row];
        float xh, xl;
        split_val(xv, xh, xl);
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const float2 w = Ws[c * NB + j];
            if (sizeof(T) == sizeof(float)) dd_mac1(acc[j], xh, w.x, w.y);
            else dd_mac(acc[j], xh, xl, w.x, w.y);
        }
    }
#pragma unroll
    for (int j = 0; j < NB; ++j) V[(int64_t)j * ldv + row] = dd_store<T>(acc[j]);
}

// Wide double-float update of a 64-row tile (k + nb <= 64): 256 threads =
// 64 rows x 4 groups of 16 outputs; the tile staged pre-split in shared memory,
// W interleaved by group.  Rows beyond n are skipped.
template <typename T>
__device__ void update_tile_wide_df(int64_t row0, int64_t n, const T* __restrict__ Q, int64_t ldq, int k,
                                    T* __restrict__ V, int64_t ldv, int nb, const float2* Ws, float2* Xt) {
    constexpr int XLD = kMaxNB + 1;
    const int kx = k + nb;
    __syncthreads();
    for (int e = threadIdx.x; e < kx * kDfWideRows; e += blockDim.x) {
        const int c = e / kDfWideRows, r = e % kDfWideRows;
        const int64_t row = row0 + r;
        float h = 0.f, l = 0.f;
        if (row < n) split_val(c < k ? __ldg(Q + (int64_t)c * ldq + row) : V[(int64_t)(c - k) * ldv + row], h, l);
        Xt[r * XLD + c] = make_float2(h, l);
    }
    __syncthreads();
    const int r = threadIdx.x >> 2, gq = threadIdx.x & 3;
    const int64_t row = row0 + r;
    const int j0 = 16 * gq;
    if (j0 < nb && row < n) {
        DD acc[16];
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) acc[jj] = DD{0.f, 0.f};
        const int cmax = min(kx, k + j0 + 16);   // W[c][j] = 0 for c - k > j (upper triangular)
        for (int c = 0; c < cmax; ++c) {
            const float2 x = Xt[r * XLD + c];
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
                const float2 w = Ws[c * kMaxNB + jj * 4 + gq];
                if (sizeof(T) == sizeof(float)) dd_mac1(acc[jj], x.x, w.x, w.y);
                else dd_mac(acc[jj], x.x, x.y, w.x, w.y);
            }
        }
#pragma unroll
        for (int jj = 0; jj < 16; ++jj)
            if (j0 + jj < nb) V[(int64_t)(j0 + jj) * ldv + row] = dd_store<T>(acc[jj]);
    }
}

}  // namespace gm
