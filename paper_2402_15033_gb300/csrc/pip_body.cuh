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
// counter holds groups + 1 arrival counters; every counter is re-armed to zero.
__device__ inline void pip_finish(int k, int nb, int g, int groups, int G, double* R, int ldr,
                                  const double* partial0, size_t ps, unsigned* counter, double* gram,
                                  int32_t* d_status, int32_t* d_skip, double* smem, int mode) {
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
        double acc = __ldcg(gram + (k + i) + (size_t)j * kx);
        for (int l = 0; l < k; ++l)
            acc -= __ldcg(gram + l + (size_t)i * kx) * __ldcg(gram + l + (size_t)j * kx);
        S[i + j * kSLd] = acc;
    }
    if (tid == 0) s_info = 0;
    __syncthreads();

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

}  // namespace gm
