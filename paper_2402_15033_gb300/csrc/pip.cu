// BCGS-PIP on FP64 data (§IV-C, Fig. 4a of the paper), the primitive of both
// stages of the two-stage block orthogonalization (§V, Fig. 5).
//
//   [P; G] = [Q, V]^T V          single tall-skinny reduction over the n rows
//   T      = Chol(G - P^T P)     block Pythagorean theorem, T upper, T_ii > 0
//   V     <- (V - Q P) T^{-1}    fused block update + triangular solve
//
// Kernel (a), the Gram reduction, is split over n: every CTA reduces a fixed,
// interleaved set of 128-row (skinny) or 32-row (wide) chunks into registers,
// folds its warps' partial sums with shuffles and writes one partial block to
// a per-CTA slot.  The last CTA to arrive (atomic ticket) sums the slots in
// CTA order, so the result does not depend on scheduling, then factors
// G - P^T P in shared memory (kernel (d)) and writes R = [P; T].
// Kernel (b) applies V <- (V - Q P) T^{-1} row by row.
//
// The basis element type T is double (FP64 path) or float (the mixed-precision
// path: FP32 basis, every product and sum in FP64, the FP32 inputs widened
// exactly on load and the updated block rounded to FP32 on store).
//
// These kernels run on the FP64 pipe, which on GB300 issues about 2 FMA per
// SM per clock (1.19 TFLOP/s measured): the Gram and the update are bound by
// FP64 arithmetic, not by HBM, at the paper's block sizes.
#include <cstdio>
#include <cstdarg>
#include "common.cuh"

namespace gm {

namespace {

constexpr int kSkinnyRows = 128;   // rows per chunk, skinny path (nb <= 16)
constexpr int kWideRows = 32;      // rows per chunk, wide path
constexpr int kSLd = kMaxNB + 1;   // leading dimension of the factor in shared memory

template <typename T>
__device__ __forceinline__ const T* col_ptr(const T* Q, int64_t ldq, int k, const T* V, int64_t ldv, int c) {
    return c < k ? Q + (int64_t)c * ldq : V + (int64_t)(c - k) * ldv;
}

__device__ __forceinline__ double ld_d(const double* p) { return __ldg(p); }
__device__ __forceinline__ double ld_d(const float* p) { return (double)__ldg(p); }

// Entry (c, j) of the (k+nb) x nb block [P; G] is needed unless it lies strictly
// below the diagonal of the symmetric G block.
__device__ __forceinline__ bool needed(int c, int j, int k) { return c < k || (c - k) <= j; }

// Last-CTA epilogue, shared by both Gram paths.  Reduces the partial slots of
// column group g in CTA order; the last group to finish factors the Gram.
__device__ void pip_epilogue(int64_t n, int k, int nb, int kx, double* R, int ldr,
                             double* partial, unsigned* counter, double* gram,
                             int32_t* d_status, int32_t* d_skip, double* smem, int mode) {
    __shared__ unsigned s_ticket;
    __shared__ int s_info;
    __shared__ double s_inv;
    const int tid = threadIdx.x;
    const int g = blockIdx.y;
    const int G = gridDim.x;
    const int groups = gridDim.y;
    const int ccount = min(kMaxNB, kx - g * kMaxNB);
    const size_t ps = (size_t)kMaxNB * nb;

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
        const double* p = partial + ((size_t)g * G) * ps + e;
        double acc = 0.0;
#pragma unroll 8
        for (int b = 0; b < G; ++b) acc += __ldcg(p + (size_t)b * ps);
        gram[c + (size_t)j * kx] = acc;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        counter[g] = 0u;  // re-arm for the next call
        s_ticket = (groups == 1) ? 0u : atomicAdd(&counter[groups], 1u) - (unsigned)(groups - 1);
    }
    __syncthreads();
    if (s_ticket != 0u) return;   // another group's last CTA factors the Gram
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

// Skinny Gram: nb <= 12.  Warp w owns the group columns w, w+8, ...; lane l owns
// rows l, l+32, ... of each chunk; the V chunk is staged in shared memory.
template <typename T, int NB>
__global__ void __launch_bounds__(kGramThreads)
gram_skinny_kernel(int64_t n, const T* __restrict__ Q, int64_t ldq, int k,
                   const T* __restrict__ V, int64_t ldv, double* __restrict__ R, int ldr,
                   double* partial, unsigned* counter, double* gram, int32_t* d_status,
                   int32_t* d_skip, int mode) {
    extern __shared__ double smem[];
    if (d_skip && *d_skip) return;
    const int kx = k + NB;
    const int g = blockIdx.y;
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
    for (int64_t ci = blockIdx.x; ci < nchunks; ci += gridDim.x) {
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
    // warp fold (fixed butterfly order) and one partial block per CTA
    const size_t ps = (size_t)kMaxNB * NB;
    double* slot = partial + ((size_t)g * gridDim.x + blockIdx.x) * ps;
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
    pip_epilogue(n, k, NB, kx, R, ldr, partial, counter, gram, d_status, d_skip, smem, mode);
}

// Wide Gram: nb up to 64.  Each thread owns a 4 x 4 tile of the group's
// (<= 64) x nb block; tiles strictly below the diagonal of the symmetric G
// block are skipped and the remaining tiles are packed onto the first threads.
template <typename T>
__global__ void __launch_bounds__(kGramThreads)
gram_wide_kernel(int64_t n, const T* __restrict__ Q, int64_t ldq, int k,
                 const T* __restrict__ V, int64_t ldv, int nb, double* __restrict__ R, int ldr,
                 double* partial, unsigned* counter, double* gram, int32_t* d_status,
                 int32_t* d_skip, int mode) {
    extern __shared__ double smem[];
    if (d_skip && *d_skip) return;
    const int kx = k + nb;
    const int g = blockIdx.y;
    const int cg0 = g * kMaxNB;
    const int ccount = min(kMaxNB, kx - cg0);
    constexpr int LD = kWideRows + 1;
    double* Xs = smem;                   // [64][LD]
    double* Ys = smem + kMaxNB * LD;     // [64][LD]

    // find this thread's tile among the active ones
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
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

    const int64_t nchunks = (n + kWideRows - 1) / kWideRows;
    for (int64_t ci = blockIdx.x; ci < nchunks; ci += gridDim.x) {
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
                double a[4], b[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) { a[t] = xs[t * LD + r]; b[t] = ys[t * LD + r]; }
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int t = 0; t < 4; ++t) acc[s][t] = fma(a[s], b[t], acc[s][t]);
            }
        }
    }
    // entries outside [ccount) x [nb) multiply zero-filled shared rows; drop them
    const size_t ps = (size_t)kMaxNB * nb;
    double* slot = partial + ((size_t)g * gridDim.x + blockIdx.x) * ps;
    if (my_bi >= 0) {
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int cl = 4 * my_bi + s, j = 4 * my_bj + t;
                if (cl < ccount && j < nb) slot[cl * nb + j] = acc[s][t];
            }
    }
    pip_epilogue(n, k, nb, kx, R, ldr, partial, counter, gram, d_status, d_skip, smem, mode);
}

// Update, nb <= 16: one thread per row, P and T staged in shared memory.
template <typename T, int NB>
__global__ void __launch_bounds__(256)
update_skinny_kernel(int64_t n, const T* __restrict__ Q, int64_t ldq, int k,
                     T* __restrict__ V, int64_t ldv, const double* __restrict__ R, int ldr,
                     const int32_t* d_status, const int32_t* d_skip, int mode) {
    extern __shared__ double smem[];
    if ((d_skip && *d_skip) || *d_status) return;
    double* Ps = smem;                 // [k][NB]
    double* Ts = smem + (size_t)k * NB;  // [NB][NB] (i, j) at i*NB + j
    double* Dinv = Ts + NB * NB;
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
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n;
         row += (int64_t)gridDim.x * blockDim.x) {
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
}

// Update, 16 < nb <= 64: one thread per row, the row of V in registers, T in
// shared memory, P read through the read-only cache (uniform across a warp).
template <typename T>
__global__ void __launch_bounds__(128)
update_wide_kernel(int64_t n, const T* __restrict__ Q, int64_t ldq, int k,
                   T* __restrict__ V, int64_t ldv, int nb, const double* __restrict__ R, int ldr,
                   const int32_t* d_status, const int32_t* d_skip, int mode) {
    __shared__ double Ts[kMaxNB * kMaxNB];
    __shared__ double Dinv[kMaxNB];
    if ((d_skip && *d_skip) || *d_status) return;
    for (int e = threadIdx.x; e < kMaxNB * kMaxNB; e += blockDim.x) {
        const int i = e / kMaxNB, j = e % kMaxNB;
        Ts[e] = (i < nb && j < nb) ? ((mode & kPipNoTrsm) ? (i == j ? 1.0 : 0.0) : R[(k + i) + (size_t)j * ldr])
                                   : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < kMaxNB) Dinv[threadIdx.x] = threadIdx.x < nb ? 1.0 / Ts[threadIdx.x * (kMaxNB + 1)] : 0.0;
    __syncthreads();
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n;
         row += (int64_t)gridDim.x * blockDim.x) {
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
}

template <typename T, int NB>
cudaError_t launch_skinny(cudaStream_t st, int64_t n, const T* Q, int64_t ldq, int k,
                          const T* V, int64_t ldv, double* R, int ldr, const PipWork& w,
                          int32_t* d_status, int32_t* d_skip, int grid, int mode) {
    const int kx = k + NB;
    const dim3 g(grid, (kx + kMaxNB - 1) / kMaxNB);
    const size_t sm = (size_t)kMaxNB * kSLd * sizeof(double);  // >= NB * kSkinnyRows doubles
    gram_skinny_kernel<T, NB><<<g, kGramThreads, sm, st>>>(n, Q, ldq, k, V, ldv, R, ldr, w.partial,
                                                        w.counter, w.gram, d_status, d_skip, mode);
    return cudaGetLastError();
}

template <typename T, int NB>
cudaError_t launch_update_skinny(cudaStream_t st, int64_t n, const T* Q, int64_t ldq, int k,
                                 T* V, int64_t ldv, const double* R, int ldr,
                                 const int32_t* d_status, const int32_t* d_skip, int mode) {
    const size_t sm = ((size_t)k * NB + NB * NB + NB) * sizeof(double);
    const int64_t blocks = (n + 255) / 256;
    const int grid = (int)(blocks < 8 * (int64_t)num_sms() ? blocks : 8 * (int64_t)num_sms());
    update_skinny_kernel<T, NB><<<grid, 256, sm, st>>>(n, Q, ldq, k, V, ldv, R, ldr, d_status, d_skip, mode);
    return cudaGetLastError();
}

}  // namespace

static_assert(kMaxNB * kSLd >= 12 * kSkinnyRows, "skinny staging fits the epilogue buffer");
constexpr size_t kWideSmem = (2 * kMaxNB * (kWideRows + 1) > kMaxNB * kSLd ? 2 * kMaxNB * (kWideRows + 1)
                                                                            : kMaxNB * kSLd) * sizeof(double);

template <typename T>
cudaError_t pip_gram_chol_t(cudaStream_t st, int64_t n, const T* Q, int64_t ldq, int k,
                            const T* V, int64_t ldv, int nb, double* R, int ldr,
                            const PipWork& w, int32_t* d_status, int32_t* d_skip, int grid, int mode) {
    switch (nb) {
#define GM_CASE(NBV) case NBV: return launch_skinny<T, NBV>(st, n, Q, ldq, k, V, ldv, R, ldr, w, d_status, d_skip, grid, mode);
        GM_CASE(1) GM_CASE(2) GM_CASE(3) GM_CASE(4) GM_CASE(5) GM_CASE(6) GM_CASE(7) GM_CASE(8)
        GM_CASE(9) GM_CASE(10) GM_CASE(11) GM_CASE(12)
#undef GM_CASE
        default: break;  // wider blocks: 8 x nb accumulators per thread would spill
    }
    const int kx = k + nb;
    const dim3 g(grid, (kx + kMaxNB - 1) / kMaxNB);
    const size_t sm = kWideSmem;
    gram_wide_kernel<T><<<g, kGramThreads, sm, st>>>(n, Q, ldq, k, V, ldv, nb, R, ldr, w.partial,
                                                  w.counter, w.gram, d_status, d_skip, mode);
    return cudaGetLastError();
}

template <typename T>
cudaError_t pip_update_t(cudaStream_t st, int64_t n, const T* Q, int64_t ldq, int k,
                         T* V, int64_t ldv, int nb, const double* R, int ldr,
                         const int32_t* d_status, const int32_t* d_skip, int mode) {
    switch (nb) {
#define GM_CASE(NBV) case NBV: return launch_update_skinny<T, NBV>(st, n, Q, ldq, k, V, ldv, R, ldr, d_status, d_skip, mode);
        GM_CASE(1) GM_CASE(2) GM_CASE(3) GM_CASE(4) GM_CASE(5) GM_CASE(6) GM_CASE(7) GM_CASE(8)
        GM_CASE(9) GM_CASE(10) GM_CASE(11) GM_CASE(12) GM_CASE(13) GM_CASE(14) GM_CASE(15) GM_CASE(16)
#undef GM_CASE
        default: break;
    }
    const int64_t blocks = (n + 127) / 128;
    const int grid = (int)(blocks < 16 * (int64_t)num_sms() ? blocks : 16 * (int64_t)num_sms());
    update_wide_kernel<T><<<grid, 128, 0, st>>>(n, Q, ldq, k, V, ldv, nb, R, ldr, d_status, d_skip, mode);
    return cudaGetLastError();
}

cudaError_t launch_pip_gram_chol(cudaStream_t st, int64_t n, const double* Q, int64_t ldq, int k,
                                 const double* V, int64_t ldv, int nb, double* R, int ldr,
                                 const PipWork& w, int32_t* d_status, int32_t* d_skip, int grid, int mode) {
    return pip_gram_chol_t<double>(st, n, Q, ldq, k, V, ldv, nb, R, ldr, w, d_status, d_skip, grid, mode);
}
cudaError_t launch_pip_gram_chol(cudaStream_t st, int64_t n, const float* Q, int64_t ldq, int k,
                                 const float* V, int64_t ldv, int nb, double* R, int ldr,
                                 const PipWork& w, int32_t* d_status, int32_t* d_skip, int grid, int mode) {
    return pip_gram_chol_t<float>(st, n, Q, ldq, k, V, ldv, nb, R, ldr, w, d_status, d_skip, grid, mode);
}
cudaError_t launch_pip_update(cudaStream_t st, int64_t n, const double* Q, int64_t ldq, int k,
                              double* V, int64_t ldv, int nb, const double* R, int ldr,
                              const int32_t* d_status, const int32_t* d_skip, int mode) {
    return pip_update_t<double>(st, n, Q, ldq, k, V, ldv, nb, R, ldr, d_status, d_skip, mode);
}
cudaError_t launch_pip_update(cudaStream_t st, int64_t n, const float* Q, int64_t ldq, int k,
                              float* V, int64_t ldv, int nb, const double* R, int ldr,
                              const int32_t* d_status, const int32_t* d_skip, int mode) {
    return pip_update_t<float>(st, n, Q, ldq, k, V, ldv, nb, R, ldr, d_status, d_skip, mode);
}

PipWork pip_work_layout(void* base, int64_t n, int k, int nb) {
    // The arrival counters sit at a fixed offset so that calls of different
    // shapes sharing one workspace never overwrite each other's counters; the
    // Gram and partial regions are rewritten in full by every call.
    PipWork w{};
    const int grid = reduction_grid(n);
    const int kx = k + nb;
    const int groups = (kx + kMaxNB - 1) / kMaxNB;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_counter = 256;
    const size_t b_gram = up((size_t)kx * nb * sizeof(double));
    const size_t b_partial = up((size_t)grid * groups * kMaxNB * nb * sizeof(double));
    char* p = static_cast<char*>(base);
    w.counter = reinterpret_cast<unsigned*>(p);
    w.gram = reinterpret_cast<double*>(p + b_counter);
    w.partial = reinterpret_cast<double*>(p + b_counter + b_gram);
    w.bytes = b_counter + b_gram + b_partial;
    return w;
}

}  // namespace gm
