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
#include <algorithm>
#include <type_traits>
#include "pip_body.cuh"
#include "gram_tc.cuh"
#include "gram_tcq.cuh"
#include "gram_t5.cuh"
#include "gram_w5.cuh"
#include "update_tc.cuh"
#include "update_tcd.cuh"

namespace gm {

namespace {

template <typename T, int NB>
__global__ void __launch_bounds__(kGramThreads)
gram_skinny_kernel(int64_t n, const T* __restrict__ Q, int64_t ldq, int k,
                   const T* __restrict__ V, int64_t ldv, double* __restrict__ R, int ldr,
                   double* partial, unsigned* counter, double* gram, int32_t* d_status,
                   int32_t* d_skip, int mode) {
    extern __shared__ double smem[];
    if (d_skip && *d_skip) return;
    const int g = blockIdx.y, G = gridDim.x;
    const size_t ps = (size_t)kMaxNB * NB;
    double* partial0 = partial + (size_t)g * G * ps;
    gram_skinny_part<T, NB>(n, Q, ldq, k, V, ldv, g, blockIdx.x, G, partial0 + blockIdx.x * ps, smem);
    pip_finish(k, NB, g, gridDim.y, G, R, ldr, partial0, ps, counter, gram, d_status, d_skip, smem, mode, n);
}

template <typename T>
__global__ void __launch_bounds__(kGramThreads)
gram_wide_kernel(int64_t n, const T* __restrict__ Q, int64_t ldq, int k,
                 const T* __restrict__ V, int64_t ldv, int nb, double* __restrict__ R, int ldr,
                 double* partial, unsigned* counter, double* gram, int32_t* d_status,
                 int32_t* d_skip, int mode) {
    extern __shared__ double smem[];
    if (d_skip && *d_skip) return;
    const int g = blockIdx.y, G = gridDim.x;
    const size_t ps = (size_t)kMaxNB * nb;
    double* partial0 = partial + (size_t)g * G * ps;
    gram_wide_part<T>(n, Q, ldq, k, V, ldv, nb, g, blockIdx.x, G, partial0 + blockIdx.x * ps, smem);
    pip_finish(k, nb, g, gridDim.y, G, R, ldr, partial0, ps, counter, gram, d_status, d_skip, smem, mode, n);
}

// Exact-slice tensor-core Gram (gram_tc.cuh), k + nb <= 64: one column group.
// The first kc columns of [Q, V] come from the digit basis when kc > 0.
__global__ void __launch_bounds__(kGramThreads, 2)
gram_tc_kernel(int64_t n, const double* __restrict__ Q, int64_t ldq, int k,
               const double* __restrict__ V, int64_t ldv, int nb, double* __restrict__ R, int ldr,
               double* partial, unsigned* counter, double* gram, int32_t* d_status,
               int32_t* d_skip, int mode, const uint4* dig, const int* dex, int capc, int kc) {
    extern __shared__ double smem[];
    if (d_skip && *d_skip) return;
    const int G = gridDim.x;
    const size_t ps = (size_t)kMaxNB * nb;
    gram_tc_part(n, Q, ldq, k, V, ldv, nb, blockIdx.x, G, partial + blockIdx.x * ps, smem, dig, dex, capc, kc);
    pip_finish(k, nb, 0, 1, G, R, ldr, partial, ps, counter, gram, d_status, d_skip, smem, mode, n);
}

// Narrow Gram with every Q column from the digit basis (gram_tcq.cuh): one CTA
// per SM, a producer warp bulk-copying the chunks, slicer and MMA warps.
__global__ void __launch_bounds__(kGqThreads, 1)
gram_tcq_kernel(int64_t n, const double* __restrict__ V, int64_t ldv, int k, int nb, double* __restrict__ R, int ldr,
                double* partial, unsigned* counter, double* gram, int32_t* d_status, int32_t* d_skip, int mode,
                const uint4* dig, const int* dex, int capc) {
    extern __shared__ __align__(16) char gq_smem[];
    if (d_skip && *d_skip) return;
    const int G = gridDim.x;
    const size_t ps = (size_t)kMaxNB * nb;
    gram_tcq_part(n, V, ldv, k, nb, blockIdx.x, G, partial + blockIdx.x * ps, gq_smem, dig, dex, capc);
    pip_finish(k, nb, 0, 1, G, R, ldr, partial, ps, counter, gram, d_status, d_skip,
               reinterpret_cast<double*>(gq_smem), mode, n);
}

cudaError_t launch_gram_tcq(cudaStream_t st, int64_t n, int k, const double* V, int64_t ldv, int nb, double* R,
                            int ldr, const PipWork& w, int32_t* d_status, int32_t* d_skip, int grid, int mode,
                            const void* digits, int capc) {
    static const cudaError_t attr = smem_limit(gram_tcq_kernel, gram_tcq_smem(kGqMaxKX - 1));
    if (attr != cudaSuccess) return attr;
    const uint4* dig = static_cast<const uint4*>(digits);
    const int* dex = reinterpret_cast<const int*>(dig + tc_digits_units(n, capc));
    const int G = std::min(grid, num_sms());
    gram_tcq_kernel<<<G, kGqThreads, gram_tcq_smem(k), st>>>(n, V, ldv, k, nb, R, ldr, w.partial, w.counter,
                                                             w.gram, d_status, d_skip, mode, dig, dex, capc);
    return cudaGetLastError();
}

// Narrow Gram on the fifth-generation tensor cores (gram_t5.cuh): one
// warp-specialized CTA per SM.
__global__ void __launch_bounds__(kG5Threads, 1)
gram_t5_kernel(int64_t n, const double* __restrict__ V, int64_t ldv, int k, int nb, double* __restrict__ R, int ldr,
               double* partial, unsigned* counter, double* gram, int32_t* d_status, int32_t* d_skip, int mode,
               const uint4* dig, const int* dex, int capc) {
    extern __shared__ __align__(1024) char g5_smem[];
    if (d_skip && *d_skip) return;
    const int G = gridDim.x;
    const size_t ps = (size_t)kMaxNB * nb;
    gram_t5_part(n, V, ldv, k, nb, blockIdx.x, G, partial + blockIdx.x * ps, g5_smem, dig, dex, capc);
    pip_finish(k, nb, 0, 1, G, R, ldr, partial, ps, counter, gram, d_status, d_skip,
               reinterpret_cast<double*>(g5_smem), mode, n);
}

cudaError_t launch_gram_t5(cudaStream_t st, int64_t n, int k, const double* V, int64_t ldv, int nb, double* R,
                           int ldr, const PipWork& w, int32_t* d_status, int32_t* d_skip, int grid, int mode,
                           const void* digits, int capc) {
    static const cudaError_t attr = smem_limit(gram_t5_kernel, kG5Smem);
    if (attr != cudaSuccess) return attr;
    const uint4* dig = static_cast<const uint4*>(digits);
    const int* dex = reinterpret_cast<const int*>(dig + tc_digits_units(n, capc));
    const int G = std::min(grid, num_sms());
    gram_t5_kernel<<<G, kG5Threads, kG5Smem, st>>>(n, V, ldv, k, nb, R, ldr, w.partial, w.counter, w.gram, d_status,
                                                   d_skip, mode, dig, dex, capc);
    return cudaGetLastError();
}

// Wide Gram over columns all in the digit basis (the stage-2 panel) on the
// fifth-generation tensor cores (gram_w5.cuh): one warp-specialized CTA per SM.
__global__ void __launch_bounds__(kW5Threads, 1)
gram_w5_kernel(int64_t n, int k, int nb, double* __restrict__ R, int ldr, double* partial, unsigned* counter,
               double* gram, int32_t* d_status, int32_t* d_skip, int mode, const uint4* dig, const int* dex, int capc) {
    extern __shared__ __align__(1024) char w5_smem_buf[];
    if (d_skip && *d_skip) return;
    const int G = gridDim.x;
    const size_t ps = (size_t)kMaxNB * nb;
    gram_w5_part(n, k, nb, blockIdx.x, G, partial + blockIdx.x * ps, w5_smem_buf, dig, dex, capc);
    pip_finish(k, nb, 0, 1, G, R, ldr, partial, ps, counter, gram, d_status, d_skip,
               reinterpret_cast<double*>(w5_smem_buf), mode, n);
}

cudaError_t launch_gram_w5(cudaStream_t st, int64_t n, int k, int nb, double* R, int ldr, const PipWork& w,
                           int32_t* d_status, int32_t* d_skip, int grid, int mode, const void* digits, int capc) {
    static const cudaError_t attr = smem_limit(gram_w5_kernel, (int)w5_smem(kW5MaxKX));
    if (attr != cudaSuccess) return attr;
    const uint4* dig = static_cast<const uint4*>(digits);
    const int* dex = reinterpret_cast<const int*>(dig + tc_digits_units(n, capc));
    const int G = std::min(grid, num_sms());
    gram_w5_kernel<<<G, kW5Threads, w5_smem(k + nb), st>>>(n, k, nb, R, ldr, w.partial, w.counter, w.gram, d_status,
                                                          d_skip, mode, dig, dex, capc);
    return cudaGetLastError();
}

cudaError_t launch_gram_tc(cudaStream_t st, int64_t n, const double* Q, int64_t ldq, int k,
                           const double* V, int64_t ldv, int nb, double* R, int ldr, const PipWork& w,
                           int32_t* d_status, int32_t* d_skip, int grid, int mode,
                           const void* digits = nullptr, int capc = 0, int kc = 0) {
    static const cudaError_t attr = smem_limit(gram_tc_kernel, gram_tc_smem(kTcMaxKX));
    if (attr != cudaSuccess) return attr;
    const uint4* dig = static_cast<const uint4*>(digits);
    const int* dex = digits ? reinterpret_cast<const int*>(dig + tc_digits_units(n, capc)) : nullptr;
    // two CTAs per SM (the chunk tiles take most of the shared memory)
    const int G = std::min(grid, 2 * num_sms());
    gram_tc_kernel<<<G, kGramThreads, gram_tc_smem(k + nb), st>>>(n, Q, ldq, k, V, ldv, nb, R, ldr, w.partial,
                                                                   w.counter, w.gram, d_status, d_skip, mode, dig,
                                                                   dex, capc, digits ? kc : 0);
    return cudaGetLastError();
}

// Digit-basis fill: columns c0 .. c0+nc-1 of the digit basis from X(:, 0:nc).
// One (chunk, column) item per half warp; a half warp without an item of its
// own repeats its partner's (the same bytes to the same places) so that both
// halves reach the exponent shuffles together.
__global__ void __launch_bounds__(256)
digits_fill_kernel(int64_t n, const double* __restrict__ X, int64_t ldx, int c0, int nc, uint4* dig, int* dex,
                   int capc) {
    const int hw = threadIdx.x >> 4, h = threadIdx.x & 15, nhw = blockDim.x >> 4;
    const int w = h >> 2, g = h & 3;
    const int64_t items = (n + 63) / 64 * nc;
    for (int64_t base = (int64_t)blockIdx.x * nhw; base < items; base += (int64_t)gridDim.x * nhw) {
        const int64_t e0 = base + (hw & ~1);             // the warp's first item
        if (e0 >= items) continue;                        // warp-uniform
        const int64_t e = base + hw < items ? base + hw : e0;
        const int64_t ch = e / nc;
        const int c = (int)(e % nc);
        double x[4];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int64_t r0 = ch * 64 + 16 * w + 2 * g + 8 * hh;
            const double* p = X + (int64_t)c * ldx + r0;
            x[2 * hh] = 0.0;
            x[2 * hh + 1] = 0.0;
            if (r0 + 1 < n) {
                const double2 v = __ldg(reinterpret_cast<const double2*>(p));
                x[2 * hh] = v.x;
                x[2 * hh + 1] = v.y;
            } else if (r0 < n) {
                x[2 * hh] = __ldg(p);
            }
        }
        tc_b8_store(x, dig + ((size_t)ch * capc + c0 + c) * kTcB8Units,
                    dex + (size_t)ch * tc_dex_stride(capc) + c0 + c);
    }
}

cudaError_t launch_digits_fill(cudaStream_t st, int64_t n, const double* X, int64_t ldx, int c0, int nc,
                               void* digits, int capc) {
    uint4* dig = static_cast<uint4*>(digits);
    int* dex = reinterpret_cast<int*>(dig + tc_digits_units(n, capc));
    const int64_t items = (n + 63) / 64 * nc;
    const int grid = (int)std::min<int64_t>((items + 15) / 16, 8 * (int64_t)num_sms());
    digits_fill_kernel<<<grid, 256, 0, st>>>(n, X, ldx, c0, nc, dig, dex, capc);
    return cudaGetLastError();
}

// Exact-slice tensor-core update (update_tc.cuh), k + nb <= 64; with DIG it also
// writes the new columns into the digit basis.
template <bool DIG>
__global__ void __launch_bounds__(512, 1)
update_tc_kernel(int64_t n, const double* __restrict__ Q, int64_t ldq, int k, double* V, int64_t ldv, int nb,
                 const double* __restrict__ R, int ldr, const int32_t* d_status, const int32_t* d_skip, int mode,
                 uint4* dig, int* dex, int capc) {
    extern __shared__ __align__(16) char tu_smem[];
    if ((d_skip && *d_skip) || *d_status) return;
    update_tc_body<DIG>(n, Q, ldq, k, V, ldv, nb, R, ldr, mode, blockIdx.x, gridDim.x, tu_smem, dig, dex, capc);
}

cudaError_t launch_update_tc(cudaStream_t st, int64_t n, const double* Q, int64_t ldq, int k, double* V,
                             int64_t ldv, int nb, const double* R, int ldr, const int32_t* d_status,
                             const int32_t* d_skip, int mode, void* digits = nullptr, int capc = 0) {
    const bool dg = digits != nullptr;
    static const cudaError_t attr_dg = smem_limit(update_tc_kernel<true>, update_tc_smem(kTuMaxKX, kTuMaxKX, true));
    static const cudaError_t attr_fp =
        smem_limit(update_tc_kernel<false>, update_tc_smem(kTuMaxKX, kTuMaxKX, false));
    const cudaError_t attr = dg ? attr_dg : attr_fp;
    if (attr != cudaSuccess) return attr;
    // wide blocks: one 16-warp CTA per SM (the W slices take a third of the
    // shared memory); narrow ones: 8-warp CTAs, two per SM where they fit
    const int threads = nb > 32 ? 512 : 256;
    const size_t sm = update_tc_smem(k + nb, nb, dg);
    const int per_sm = nb > 32 ? 1 : (2 * (sm + 1024) <= 228 * 1024 ? 2 : 1);
    const int64_t chunks = (n + kTuRows - 1) / kTuRows;
    const int G = (int)std::min<int64_t>(chunks, (int64_t)per_sm * num_sms());
    uint4* dig = static_cast<uint4*>(digits);
    int* dex = dg ? reinterpret_cast<int*>(dig + tc_digits_units(n, capc)) : nullptr;
    if (dg)
        update_tc_kernel<true><<<G, threads, sm, st>>>(n, Q, ldq, k, V, ldv, nb, R, ldr, d_status, d_skip, mode, dig,
                                                       dex, capc);
    else
        update_tc_kernel<false><<<G, threads, sm, st>>>(n, Q, ldq, k, V, ldv, nb, R, ldr, d_status, d_skip, mode,
                                                        nullptr, nullptr, 0);
    return cudaGetLastError();
}

// Narrow update from the digit basis (update_tcd.cuh), nb <= 8, k + nb <= 64.
__global__ void __launch_bounds__(kUdThreads, 4)
update_tcd_kernel(int64_t n, int k, double* V, int64_t ldv, int nb, const double* __restrict__ R, int ldr,
                  const int32_t* d_status, const int32_t* d_skip, int mode, uint4* dig, int* dex, int capc) {
    extern __shared__ __align__(16) char td_smem[];
    if ((d_skip && *d_skip) || *d_status) return;
    update_tcd_body(n, k, V, ldv, nb, R, ldr, mode, blockIdx.x, gridDim.x, td_smem, dig, dex, capc);
}

cudaError_t launch_update_tcd(cudaStream_t st, int64_t n, int k, double* V, int64_t ldv, int nb, const double* R,
                              int ldr, const int32_t* d_status, const int32_t* d_skip, int mode, void* digits,
                              int capc) {
    static const cudaError_t attr = smem_limit(update_tcd_kernel, update_tcd_smem(kTuMaxKX, kUdMaxNB));
    if (attr != cudaSuccess) return attr;
    const int64_t chunks = (n + kUdRows - 1) / kUdRows;
    const int G = (int)std::min<int64_t>(chunks, 4 * (int64_t)num_sms());
    uint4* dig = static_cast<uint4*>(digits);
    int* dex = reinterpret_cast<int*>(dig + tc_digits_units(n, capc));
    update_tcd_kernel<<<G, kUdThreads, update_tcd_smem(k + nb, nb), st>>>(n, k, V, ldv, nb, R, ldr, d_status, d_skip,
                                                                          mode, dig, dex, capc);
    return cudaGetLastError();
}

// Update, nb <= 16: one thread per row, P and T staged in shared memory.
template <typename T, int NB>
__global__ void __launch_bounds__(256)
update_skinny_kernel(int64_t n, const T* __restrict__ Q, int64_t ldq, int k,
                     T* __restrict__ V, int64_t ldv, const double* __restrict__ R, int ldr,
                     const int32_t* d_status, const int32_t* d_skip, int mode) {
    extern __shared__ double smem[];
    if ((d_skip && *d_skip) || *d_status) return;
    double* Ps = smem;
    double* Ts = smem + (size_t)k * NB;
    double* Dinv = Ts + NB * NB;
    stage_pt<NB>(k, R, ldr, mode, Ps, Ts, Dinv);
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n;
         row += (int64_t)gridDim.x * blockDim.x)
        update_row<T, NB>(row, Q, ldq, k, V, ldv, Ps, Ts, Dinv);
}

// Update, 16 < nb <= 64.
template <typename T>
__global__ void __launch_bounds__(128)
update_wide_kernel(int64_t n, const T* __restrict__ Q, int64_t ldq, int k,
                   T* __restrict__ V, int64_t ldv, int nb, const double* __restrict__ R, int ldr,
                   const int32_t* d_status, const int32_t* d_skip, int mode) {
    __shared__ double Ts[kMaxNB * kMaxNB];
    __shared__ double Dinv[kMaxNB];
    if ((d_skip && *d_skip) || *d_status) return;
    stage_t_wide(k, nb, R, ldr, mode, Ts, Dinv);
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n;
         row += (int64_t)gridDim.x * blockDim.x)
        update_row_wide<T>(row, Q, ldq, k, V, ldv, nb, R, ldr, Ts, Dinv);
}

// ---------------------------------------------------------------- double-float kernels
template <typename T, int NB>
__global__ void __launch_bounds__(kGramThreads)
gram_skinny_df_kernel(int64_t n, const T* __restrict__ Q, int64_t ldq, int k,
                      const T* __restrict__ V, int64_t ldv, double* __restrict__ R, int ldr,
                      double* partial, unsigned* counter, double* gram, int32_t* d_status,
                      int32_t* d_skip, int mode) {
    extern __shared__ double smem[];
    if (d_skip && *d_skip) return;
    const int g = blockIdx.y, G = gridDim.x;
    const size_t ps = (size_t)kMaxNB * NB;
    double* partial0 = partial + (size_t)g * G * ps;
    gram_skinny_part_df<T, NB>(n, Q, ldq, k, V, ldv, g, blockIdx.x, G, partial0 + blockIdx.x * ps, smem);
    pip_finish(k, NB, g, gridDim.y, G, R, ldr, partial0, ps, counter, gram, d_status, d_skip, smem, mode, n);
}

template <typename T>
__global__ void __launch_bounds__(kGramThreads)
gram_wide_df_kernel(int64_t n, const T* __restrict__ Q, int64_t ldq, int k,
                    const T* __restrict__ V, int64_t ldv, int nb, double* __restrict__ R, int ldr,
                    double* partial, unsigned* counter, double* gram, int32_t* d_status,
                    int32_t* d_skip, int mode) {
    extern __shared__ double smem[];
    if (d_skip && *d_skip) return;
    const int g = blockIdx.y, G = gridDim.x;
    const size_t ps = (size_t)kMaxNB * nb;
    double* partial0 = partial + (size_t)g * G * ps;
    gram_wide_part_df<T>(n, Q, ldq, k, V, ldv, nb, g, blockIdx.x, G, partial0 + blockIdx.x * ps, smem);
    pip_finish(k, nb, g, gridDim.y, G, R, ldr, partial0, ps, counter, gram, d_status, d_skip, smem, mode, n);
}

// Double-float update, nb <= 16: W = [-P T^{-1}; T^{-1}] staged pre-split, one thread per row.
template <typename T, int NB>
__global__ void __launch_bounds__(256)
update_skinny_df_kernel(int64_t n, const T* __restrict__ Q, int64_t ldq, int k,
                        T* __restrict__ V, int64_t ldv, const double* __restrict__ R, int ldr,
                        const int32_t* d_status, const int32_t* d_skip, int mode) {
    extern __shared__ double smem[];
    if ((d_skip && *d_skip) || *d_status) return;
    double* Tinv = smem;                                          // [NB][NB]
    float2* Ws = reinterpret_cast<float2*>(smem + NB * NB);       // [(k+NB)][NB]
    stage_w_df(k, NB, R, ldr, mode, Ws, NB, 1, Tinv);
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < n;
         row += (int64_t)gridDim.x * blockDim.x)
        update_row_df<T, NB>(row, Q, ldq, k, V, ldv, Ws);
}

constexpr size_t kWideDfSmem = (size_t)kMaxNB * kMaxNB * sizeof(float2) +            // W
                               (size_t)kDfWideRows * (kMaxNB + 1) * sizeof(float2);  // row tile (and T^{-1})

// Double-float update, 16 < nb and k + nb <= 64: 64-row tiles, 4 output groups.
template <typename T>
__global__ void __launch_bounds__(256)
update_wide_df_kernel(int64_t n, const T* __restrict__ Q, int64_t ldq, int k,
                      T* __restrict__ V, int64_t ldv, int nb, const double* __restrict__ R, int ldr,
                      const int32_t* d_status, const int32_t* d_skip, int mode) {
    extern __shared__ double smem[];
    if ((d_skip && *d_skip) || *d_status) return;
    float2* Ws = reinterpret_cast<float2*>(smem);
    float2* Xt = Ws + kMaxNB * kMaxNB;
    stage_w_df(k, nb, R, ldr, mode, Ws, kMaxNB, 4, reinterpret_cast<double*>(Xt));
    const int64_t ntiles = (n + kDfWideRows - 1) / kDfWideRows;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x)
        update_tile_wide_df<T>(t * kDfWideRows, n, Q, ldq, k, V, ldv, nb, Ws, Xt);
}

template <typename T, int NB>
cudaError_t launch_skinny(cudaStream_t st, int64_t n, const T* Q, int64_t ldq, int k,
                          const T* V, int64_t ldv, double* R, int ldr, const PipWork& w,
                          int32_t* d_status, int32_t* d_skip, int grid, int mode) {
    const int kx = k + NB;
    const dim3 g(grid, (kx + kMaxNB - 1) / kMaxNB);
    gram_skinny_kernel<T, NB><<<g, kGramThreads, kGramSmem, st>>>(n, Q, ldq, k, V, ldv, R, ldr, w.partial,
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

template <typename T, int NB>
cudaError_t launch_skinny_df(cudaStream_t st, int64_t n, const T* Q, int64_t ldq, int k,
                             const T* V, int64_t ldv, double* R, int ldr, const PipWork& w,
                             int32_t* d_status, int32_t* d_skip, int grid, int mode) {
    const int kx = k + NB;
    const dim3 g(grid, (kx + kMaxNB - 1) / kMaxNB);
    const size_t sm = gram_skinny_df_smem(std::min(kx, kMaxNB) + NB);
    static const cudaError_t attr = smem_limit(gram_skinny_df_kernel<T, NB>, gram_skinny_df_smem(kMaxNB + NB));
    if (attr != cudaSuccess) return attr;
    gram_skinny_df_kernel<T, NB><<<g, kGramThreads, sm, st>>>(n, Q, ldq, k, V, ldv, R, ldr, w.partial,
                                                              w.counter, w.gram, d_status, d_skip, mode);
    return cudaGetLastError();
}

template <typename T, int NB>
cudaError_t launch_update_skinny_df(cudaStream_t st, int64_t n, const T* Q, int64_t ldq, int k,
                                    T* V, int64_t ldv, const double* R, int ldr,
                                    const int32_t* d_status, const int32_t* d_skip, int mode) {
    const size_t sm = (size_t)NB * NB * sizeof(double) + (size_t)(k + NB) * NB * sizeof(float2);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(update_skinny_df_kernel<T, NB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    const int64_t blocks = (n + 255) / 256;
    const int grid = (int)(blocks < 8 * (int64_t)num_sms() ? blocks : 8 * (int64_t)num_sms());
    update_skinny_df_kernel<T, NB><<<grid, 256, sm, st>>>(n, Q, ldq, k, V, ldv, R, ldr, d_status, d_skip, mode);
    return cudaGetLastError();
}

}  // namespace

// The tensor-core and double-float kernels stage column pieces with 16-byte
// asynchronous copies: every column of Q and V must start on a 16-byte
// boundary (base aligned and ld * sizeof(T) a multiple of 16).  Other layouts
// run the FP64-pipe kernels, which read element by element.
template <typename T>
static bool cols_aligned16(const T* Q, int64_t ldq, int k, const T* V, int64_t ldv) {
    auto ok = [](const T* p, int64_t ld) {
        return (reinterpret_cast<uintptr_t>(p) & 15) == 0 && ((uint64_t)ld * sizeof(T)) % 16 == 0;
    };
    return ok(V, ldv) && (k == 0 || ok(Q, ldq));
}

template <typename T>
cudaError_t pip_gram_chol_t(cudaStream_t st, int64_t n, const T* Q, int64_t ldq, int k,
                            const T* V, int64_t ldv, int nb, double* R, int ldr,
                            const PipWork& w, int32_t* d_status, int32_t* d_skip, int grid, int mode,
                            int arith) {
    if (arith != kArithFP64 && !cols_aligned16(Q, ldq, k, V, ldv)) arith = kArithFP64;
    if constexpr (std::is_same<T, double>::value) {
        if (arith == kArithTC && k + nb <= kTcMaxKX)
            return launch_gram_tc(st, n, Q, ldq, k, V, ldv, nb, R, ldr, w, d_status, d_skip, grid, mode);
    }
    if (arith == kArithDD) {
        switch (nb) {
#define GM_CASE(NBV) case NBV: return launch_skinny_df<T, NBV>(st, n, Q, ldq, k, V, ldv, R, ldr, w, d_status, d_skip, grid, mode);
            GM_CASE(1) GM_CASE(2) GM_CASE(3) GM_CASE(4) GM_CASE(5) GM_CASE(6) GM_CASE(7) GM_CASE(8)
#undef GM_CASE
            default: break;
        }
        const dim3 g(grid, (k + nb + kMaxNB - 1) / kMaxNB);
        gram_wide_df_kernel<T><<<g, kGramThreads, kGramSmem, st>>>(n, Q, ldq, k, V, ldv, nb, R, ldr, w.partial,
                                                                   w.counter, w.gram, d_status, d_skip, mode);
        return cudaGetLastError();
    }
    switch (nb) {
#define GM_CASE(NBV) case NBV: return launch_skinny<T, NBV>(st, n, Q, ldq, k, V, ldv, R, ldr, w, d_status, d_skip, grid, mode);
        GM_CASE(1) GM_CASE(2) GM_CASE(3) GM_CASE(4) GM_CASE(5) GM_CASE(6) GM_CASE(7) GM_CASE(8)
        GM_CASE(9) GM_CASE(10) GM_CASE(11) GM_CASE(12)
#undef GM_CASE
        default: break;  // wider blocks: 8 x nb accumulators per thread would spill
    }
    const int kx = k + nb;
    const dim3 g(grid, (kx + kMaxNB - 1) / kMaxNB);
    gram_wide_kernel<T><<<g, kGramThreads, kGramSmem, st>>>(n, Q, ldq, k, V, ldv, nb, R, ldr, w.partial,
                                                  w.counter, w.gram, d_status, d_skip, mode);
    return cudaGetLastError();
}

template <typename T>
cudaError_t pip_update_t(cudaStream_t st, int64_t n, const T* Q, int64_t ldq, int k,
                         T* V, int64_t ldv, int nb, const double* R, int ldr,
                         const int32_t* d_status, const int32_t* d_skip, int mode, int arith) {
    if (arith != kArithFP64 && !cols_aligned16<T>(Q, ldq, k, V, ldv)) arith = kArithFP64;
    if constexpr (std::is_same<T, double>::value) {
        if (arith == kArithTC && k + nb <= kTuMaxKX)
            return launch_update_tc(st, n, Q, ldq, k, V, ldv, nb, R, ldr, d_status, d_skip, mode);
    }
    if (arith == kArithDD) {
        switch (nb) {
#define GM_CASE(NBV) case NBV: return launch_update_skinny_df<T, NBV>(st, n, Q, ldq, k, V, ldv, R, ldr, d_status, d_skip, mode);
            GM_CASE(1) GM_CASE(2) GM_CASE(3) GM_CASE(4) GM_CASE(5) GM_CASE(6) GM_CASE(7) GM_CASE(8)
            GM_CASE(9) GM_CASE(10) GM_CASE(11) GM_CASE(12) GM_CASE(13) GM_CASE(14) GM_CASE(15) GM_CASE(16)
#undef GM_CASE
            default: break;
        }
        if (k + nb <= kMaxNB) {
            static const cudaError_t attr = smem_limit(update_wide_df_kernel<T>, kWideDfSmem);
            if (attr != cudaSuccess) return attr;
            const int64_t tiles = (n + kDfWideRows - 1) / kDfWideRows;
            const int grid = (int)(tiles < 4 * (int64_t)num_sms() ? tiles : 4 * (int64_t)num_sms());
            update_wide_df_kernel<T><<<grid, 256, kWideDfSmem, st>>>(n, Q, ldq, k, V, ldv, nb, R, ldr, d_status,
                                                                      d_skip, mode);
            return cudaGetLastError();
        }
        // wider than one 64-column tile: the FP64-pipe kernel below
    }
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
                                 const PipWork& w, int32_t* d_status, int32_t* d_skip, int grid, int mode,
                                 int arith) {
    return pip_gram_chol_t<double>(st, n, Q, ldq, k, V, ldv, nb, R, ldr, w, d_status, d_skip, grid, mode, arith);
}
cudaError_t launch_pip_gram_chol(cudaStream_t st, int64_t n, const float* Q, int64_t ldq, int k,
                                 const float* V, int64_t ldv, int nb, double* R, int ldr,
                                 const PipWork& w, int32_t* d_status, int32_t* d_skip, int grid, int mode,
                                 int arith) {
    return pip_gram_chol_t<float>(st, n, Q, ldq, k, V, ldv, nb, R, ldr, w, d_status, d_skip, grid, mode, arith);
}
cudaError_t launch_pip_update(cudaStream_t st, int64_t n, const double* Q, int64_t ldq, int k,
                              double* V, int64_t ldv, int nb, const double* R, int ldr,
                              const int32_t* d_status, const int32_t* d_skip, int mode, int arith) {
    return pip_update_t<double>(st, n, Q, ldq, k, V, ldv, nb, R, ldr, d_status, d_skip, mode, arith);
}
cudaError_t launch_pip_update(cudaStream_t st, int64_t n, const float* Q, int64_t ldq, int k,
                              float* V, int64_t ldv, int nb, const double* R, int ldr,
                              const int32_t* d_status, const int32_t* d_skip, int mode, int arith) {
    return pip_update_t<float>(st, n, Q, ldq, k, V, ldv, nb, R, ldr, d_status, d_skip, mode, arith);
}

// Tensor-core halves with a digit basis (entry points ortho_*_tcd, ortho_digits_fill).
cudaError_t launch_gram_tc_digits(cudaStream_t st, int64_t n, const double* Q, int64_t ldq, int k, const double* V,
                                  int64_t ldv, int nb, double* R, int ldr, const PipWork& w, int32_t* d_status,
                                  int grid, const void* digits, int capc, int kc, int32_t* d_skip, int mode) {
    // narrow blocks against a Q held entirely in the digit basis: wider than 32
    // columns on tcgen05 (gram_t5.cuh), narrower ones on mma.sync with per-warp
    // streaming (gram_tcq.cuh)
    if (nb <= kG5MaxNB && kc == k && k + nb >= kG5MinKX && k + nb <= kG5MaxKX)
        return launch_gram_t5(st, n, k, V, ldv, nb, R, ldr, w, d_status, d_skip, grid, mode, digits, capc);
    // every column in the digit basis (the stage-2 panel, wide blocks): tcgen05
    // with exact per-CTA accumulation (gram_w5.cuh)
    if (nb >= kW5MinNB && kc == k + nb && k + nb <= kW5MaxKX)
        return launch_gram_w5(st, n, k, nb, R, ldr, w, d_status, d_skip, grid, mode, digits, capc);
    if (nb <= kGqMaxNB && kc == k && k + nb <= kGqMaxKX)
        return launch_gram_tcq(st, n, k, V, ldv, nb, R, ldr, w, d_status, d_skip, grid, mode, digits, capc);
    return launch_gram_tc(st, n, Q, ldq, k, V, ldv, nb, R, ldr, w, d_status, d_skip, grid, mode, digits, capc, kc);
}
cudaError_t launch_update_tc_digits(cudaStream_t st, int64_t n, const double* Q, int64_t ldq, int k, double* V,
                                    int64_t ldv, int nb, const double* R, int ldr, const int32_t* d_status,
                                    void* digits, int capc, const int32_t* d_skip, int mode) {
    // narrow blocks read Q's digits instead of slicing its rows
    if (nb <= kUdMaxNB) return launch_update_tcd(st, n, k, V, ldv, nb, R, ldr, d_status, d_skip, mode, digits, capc);
    return launch_update_tc(st, n, Q, ldq, k, V, ldv, nb, R, ldr, d_status, d_skip, mode, digits, capc);
}
cudaError_t launch_digits_fill_cols(cudaStream_t st, int64_t n, const double* X, int64_t ldx, int c0, int nc,
                                    void* digits, int capc) {
    return launch_digits_fill(st, n, X, ldx, c0, nc, digits, capc);
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
