// Batched s-step GMRES: many independent systems of different sizes advanced
// together, one restart cycle per CUDA-graph launch.
//
// Layout.  The systems' rows are concatenated (each system padded to a
// multiple of 32 rows), so every vector and every basis column is one array
// over the concatenated row space and A is one block-diagonal CSR.  A device
// table maps row tiles (256 rows) and virtual reduction CTAs to systems.
//
// Kernels.  Each step of the cycle (MPK SpMV, the Gram reductions with their
// fused Cholesky, the block update, the Hessenberg/Givens work, the solution
// update, the restart residual) is one persistent launch over the work items
// of all systems.  A system's Gram reduction uses the same virtual-CTA split
// (function of its n only) and the same fixed-order second-level reduce as a
// single solve, so each system's arithmetic, and therefore its result, does
// not depend on which other systems share the batch.  Systems that converged,
// broke down or ran out of restarts stand down at the start of the cycle.
//
// Precision: FP64 or the mixed pattern (FP32 basis and MPK, FP64 Gram,
// Cholesky, Hessenberg and refinement), as in the single-system solver.
#include <cstring>
#include <cmath>
#include <vector>
#include <algorithm>
#include <chrono>
#include "pip_body.cuh"
#include "smallls_body.cuh"

namespace gm {

constexpr int kTile = 256;

struct BSys {
    int64_t n;      // rows of this system
    int64_t row0;   // first row in the concatenated space (multiple of 32)
    int32_t G;      // virtual CTAs of its reductions
    int32_t v0;     // first virtual CTA id
    int32_t t0;     // first row tile
    int32_t nt;     // row tiles
};

struct BatchDev {
    const BSys* sys;
    const int32_t* vsys;    // virtual CTA -> system
    const int32_t* tsys;    // row tile -> system
    int32_t nsys, vtot, ttot;
    int64_t ld;             // leading dimension of the concatenated basis
    DevState* st;           // [nsys]
    const int32_t* active;  // [nsys] 1 = keep iterating
    double* partial;        // [vtot][64 * nb_max]
    unsigned* counter;      // [nsys][8]
    double* gram;           // [nsys][64 * 64]
    double* tpart;          // [ttot] residual partial sums
    unsigned* tcount;       // [nsys]
};

namespace {

__device__ inline double block_sum256(double v) {
    __shared__ double s_w[kTile / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if (lane == 0) s_w[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < (int)(blockDim.x >> 5) ? s_w[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    }
    return t;
}

// which = 0: Rhat block of stage 1 at column k0; 1: Cm block of stage 2 at column k0
__device__ inline double* r_block(DevState* st, int which, int k0) {
    return (which == 0 ? st->Rhat : st->Cm) + (size_t)k0 * kMaxCols;
}

template <typename T, int NB, bool DDA>
__global__ void __launch_bounds__(kGramThreads)
bgram_skinny_kernel(BatchDev B, T* basis, int k, int vcol, int which, int rrow, int statidx, int mode) {
    extern __shared__ double smem[];
    const size_t ps = (size_t)kMaxNB * NB;
    for (int v = blockIdx.x; v < B.vtot; v += gridDim.x) {
        const int s = B.vsys[v];
        DevState* st = B.st + s;
        if (st->done) continue;
        const BSys S = B.sys[s];
        const int b = v - S.v0;
        double* partial0 = B.partial + (size_t)S.v0 * ps;
        const T* Q = basis + S.row0;
        const T* V = basis + S.row0 + (int64_t)vcol * B.ld;
        if (DDA) gram_skinny_part_df<T, NB>(S.n, Q, B.ld, k, V, B.ld, 0, b, S.G, partial0 + (size_t)b * ps, smem);
        else gram_skinny_part<T, NB>(S.n, Q, B.ld, k, V, B.ld, 0, b, S.G, partial0 + (size_t)b * ps, smem);
        pip_finish(k, NB, 0, 1, S.G, r_block(st, which, vcol) + rrow, kMaxCols, partial0, ps,
                   B.counter + 8 * s, B.gram + (size_t)s * kMaxNB * kMaxNB, &st->blkstat[statidx], &st->done, smem,
                   mode);
    }
}

template <typename T, bool DDA>
__global__ void __launch_bounds__(kGramThreads)
bgram_wide_kernel(BatchDev B, T* basis, int k, int nb, int vcol, int which, int rrow, int statidx, int mode) {
    extern __shared__ double smem[];
    const size_t ps = (size_t)kMaxNB * nb;
    for (int v = blockIdx.x; v < B.vtot; v += gridDim.x) {
        const int s = B.vsys[v];
        DevState* st = B.st + s;
        if (st->done) continue;
        const BSys S = B.sys[s];
        const int b = v - S.v0;
        double* partial0 = B.partial + (size_t)S.v0 * ps;
        const T* Q = basis + S.row0;
        const T* V = basis + S.row0 + (int64_t)vcol * B.ld;
        if (DDA) gram_wide_part_df<T>(S.n, Q, B.ld, k, V, B.ld, nb, 0, b, S.G, partial0 + (size_t)b * ps, smem);
        else gram_wide_part<T>(S.n, Q, B.ld, k, V, B.ld, nb, 0, b, S.G, partial0 + (size_t)b * ps, smem);
        pip_finish(k, nb, 0, 1, S.G, r_block(st, which, vcol) + rrow, kMaxCols, partial0, ps,
                   B.counter + 8 * s, B.gram + (size_t)s * kMaxNB * kMaxNB, &st->blkstat[statidx], &st->done, smem,
                   mode);
    }
}

template <typename T, int NB, bool DDA>
__global__ void __launch_bounds__(kTile)
bupdate_skinny_kernel(BatchDev B, T* basis, int k, int vcol, int which, int rrow, int statidx, int mode) {
    __shared__ double Tinv[16 * 16];
    __shared__ float2 Ws[kMaxCols * 16];
    __shared__ double Ps[kMaxCols * 16];
    __shared__ double Ts[16 * 16];
    __shared__ double Dinv[16];
    int cur = -1;
    for (int t = blockIdx.x; t < B.ttot; t += gridDim.x) {
        const int s = B.tsys[t];
        DevState* st = B.st + s;
        if (st->done || st->blkstat[statidx]) continue;
        const BSys S = B.sys[s];
        const double* R = r_block(st, which, vcol) + rrow;
        if (s != cur) {
            __syncthreads();
            if (DDA) stage_w_df(k, NB, R, kMaxCols, mode, Ws, NB, 1, Tinv);
            else stage_pt<NB>(k, R, kMaxCols, mode, Ps, Ts, Dinv);
            cur = s;
        }
        const int64_t row = (int64_t)(t - S.t0) * kTile + threadIdx.x;
        if (row < S.n) {
            T* V = basis + S.row0 + (int64_t)vcol * B.ld;
            if (DDA) update_row_df<T, NB>(row, basis + S.row0, B.ld, k, V, B.ld, Ws);
            else update_row<T, NB>(row, basis + S.row0, B.ld, k, V, B.ld, Ps, Ts, Dinv);
        }
    }
}

constexpr size_t kBWideSmem = (size_t)kMaxNB * kMaxNB * sizeof(float2) + (size_t)kDfWideRows * (kMaxNB + 1) * sizeof(float2);

template <typename T, bool DDA>
__global__ void __launch_bounds__(256)
bupdate_wide_kernel(BatchDev B, T* basis, int k, int nb, int vcol, int which, int rrow, int statidx, int mode) {
    extern __shared__ double smem[];
    float2* Ws = reinterpret_cast<float2*>(smem);
    float2* Xt = Ws + kMaxNB * kMaxNB;
    double* Ts = smem;                       // FP64 path: T and 1/T_jj
    double* Dinv = smem + kMaxNB * kMaxNB;
    int cur = -1;
    for (int t = blockIdx.x; t < B.ttot; t += gridDim.x) {
        const int s = B.tsys[t];
        DevState* st = B.st + s;
        if (st->done || st->blkstat[statidx]) continue;
        const BSys S = B.sys[s];
        const double* R = r_block(st, which, vcol) + rrow;
        if (s != cur) {
            __syncthreads();
            if (DDA) stage_w_df(k, nb, R, kMaxCols, mode, Ws, kMaxNB, 4, reinterpret_cast<double*>(Xt));
            else stage_t_wide(k, nb, R, kMaxCols, mode, Ts, Dinv);
            cur = s;
        }
        const int64_t r0 = (int64_t)(t - S.t0) * kTile;
        T* V = basis + S.row0 + (int64_t)vcol * B.ld;
        if (DDA) {
            for (int q = 0; q < kTile / kDfWideRows; ++q)
                update_tile_wide_df<T>(r0 + q * kDfWideRows, S.n, basis + S.row0, B.ld, k, V, B.ld, nb, Ws, Xt);
        } else {
            for (int r = threadIdx.x; r < kTile; r += blockDim.x)
                if (r0 + r < S.n)
                    update_row_wide<T>(r0 + r, basis + S.row0, B.ld, k, V, B.ld, nb, R, kMaxCols, Ts, Dinv);
        }
    }
}

// y = (A x - theta x) / sigma on the block-diagonal matrix, per-system skip
template <typename T>
__global__ void __launch_bounds__(kTile)
bspmv_kernel(BatchDev B, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
             const T* __restrict__ vals, T* basis, int xcol, int ycol, int step) {
    for (int t = blockIdx.x; t < B.ttot; t += gridDim.x) {
        const int s = B.tsys[t];
        const DevState* st = B.st + s;
        if (st->done) continue;
        const BSys S = B.sys[s];
        const int64_t loc = (int64_t)(t - S.t0) * kTile + threadIdx.x;
        if (loc >= S.n) continue;
        const int64_t i = S.row0 + loc;
        const T* x = basis + (int64_t)xcol * B.ld;
        const int32_t p0 = __ldg(rowptr + i), p1 = __ldg(rowptr + i + 1);
        T acc = T(0);
        for (int32_t p = p0; p < p1; ++p) acc = fma(__ldg(vals + p), __ldg(x + __ldg(colind + p)), acc);
        const T th = (T)st->theta[step];
        if (th != T(0)) acc = fma(-th, x[i], acc);
        basis[(int64_t)ycol * B.ld + i] = acc * (T)(1.0 / st->sigma);
    }
}

// r = b - A x per system (x null: r = b), FP64; per-system norm reduced in tile order.
__global__ void __launch_bounds__(kTile)
bresidual_kernel(BatchDev B, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                 const double* __restrict__ vals, const double* __restrict__ b, const double* __restrict__ x,
                 double* out, int which) {
    __shared__ bool s_last;
    for (int t = blockIdx.x; t < B.ttot; t += gridDim.x) {
        const int s = B.tsys[t];
        if (!B.active[s]) continue;
        const BSys S = B.sys[s];
        const int64_t loc = (int64_t)(t - S.t0) * kTile + threadIdx.x;
        double ss = 0.0;
        if (loc < S.n) {
            const int64_t i = S.row0 + loc;
            double r = b[i];
            if (x) {
                const int32_t p0 = __ldg(rowptr + i), p1 = __ldg(rowptr + i + 1);
                double acc = 0.0;
                for (int32_t p = p0; p < p1; ++p) acc = fma(__ldg(vals + p), __ldg(x + __ldg(colind + p)), acc);
                r -= acc;
            }
            if (out) out[i] = r;
            ss = r * r;
        }
        const double tsum = block_sum256(ss);
        if (threadIdx.x == 0) {
            B.tpart[t] = tsum;
            __threadfence();
            s_last = atomicAdd(&B.tcount[s], 1u) == (unsigned)(S.nt - 1);
        }
        __syncthreads();
        if (s_last && threadIdx.x == 0) {
            __threadfence();
            double acc = 0.0;
            for (int q = 0; q < S.nt; ++q) acc += __ldcg(B.tpart + S.t0 + q);
            const double nrm = sqrt(acc);
            DevState* st = B.st + s;
            if (which == 0) {
                st->beta = nrm;
                st->inv_beta = nrm > 0.0 ? 1.0 / nrm : 0.0;
            } else {
                st->bnorm = nrm;
            }
            B.tcount[s] = 0u;
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(kTile) bscale_kernel(BatchDev B, const double* r, T* basis) {
    for (int t = blockIdx.x; t < B.ttot; t += gridDim.x) {
        const int s = B.tsys[t];
        const DevState* st = B.st + s;
        if (st->done) continue;
        const BSys S = B.sys[s];
        const int64_t loc = (int64_t)(t - S.t0) * kTile + threadIdx.x;
        if (loc < S.n) basis[S.row0 + loc] = (T)(r[S.row0 + loc] * st->inv_beta);
    }
}

template <typename T>
__global__ void __launch_bounds__(kTile) bxupdate_kernel(BatchDev B, const T* basis, double* x) {
    for (int t = blockIdx.x; t < B.ttot; t += gridDim.x) {
        const int s = B.tsys[t];
        DevState* st = B.st + s;
        if (!B.active[s]) continue;
        const int k = st->k_used;
        if (k == 0) continue;
        const BSys S = B.sys[s];
        const int64_t loc = (int64_t)(t - S.t0) * kTile + threadIdx.x;
        if (loc < S.n) {
            const int64_t i = S.row0 + loc;
            double acc = x[i];
            for (int c = 0; c < k; ++c) acc = fma((double)__ldg(basis + (int64_t)c * B.ld + i), st->y[c], acc);
            x[i] = acc;
        }
        if (t == S.t0 && threadIdx.x == 0) st->iters += k;
    }
}

__global__ void bcycle_begin_kernel(BatchDev B) {
    const int s = blockIdx.x;
    cycle_begin_body(B.st + s, B.active[s] ? 0 : 1);
}

__global__ void __launch_bounds__(kLsThreads) bhess_kernel(BatchDev B, int lo, int t) {
    extern __shared__ __align__(16) double bh_dyn[];
    hessenberg_ls_body(B.st + blockIdx.x, lo, t, bh_dyn);
}

}  // namespace
}  // namespace gm

using namespace gm;

struct gmres_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    gmres_opts opts{};
    int32_t nsys = 0;
    std::vector<BSys> hsys;
    std::vector<int32_t> hvsys, htsys;
    int64_t ntot = 0;           // concatenated (padded) rows
    BatchDev B{};
    BSys* d_sys = nullptr;
    int32_t* d_vsys = nullptr;
    int32_t* d_tsys = nullptr;
    int32_t* d_active = nullptr;
    DevState* d_st = nullptr;
    std::vector<DevState> hst_init;
    DevState* h_st = nullptr;   // pinned mirror
    int32_t* d_rowptr = nullptr;
    int32_t* d_colind = nullptr;
    double* d_vals = nullptr;
    float* d_vals32 = nullptr;
    void* basis = nullptr;
    double *d_b = nullptr, *d_x = nullptr, *d_r = nullptr;
    double* d_partial = nullptr;
    unsigned* d_counter = nullptr;
    double* d_gram = nullptr;
    double* d_tpart = nullptr;
    unsigned* d_tcount = nullptr;
    int grid_gram = 0, grid_rows = 0;   // persistent grid sizes (autotuned)
    cudaGraphExec_t graph = nullptr;
    double tune_ms[4] = {0, 0, 0, 0};
};

namespace {

int cuda_rc_b(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return GMRES_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? GMRES_ERR_OOM : GMRES_ERR_CUDA;
}

template <typename T, bool DDA>
cudaError_t launch_bgram_t(gmres_batch* c, T* basis, int k, int nb, int vcol, int which, int rrow, int statidx,
                           int mode) {
    const BatchDev& B = c->B;
    if (!DDA || nb > kDfSkinnyMaxNB) {
        if (nb <= kSkinnyMaxNB && !DDA) {
            switch (nb) {
#define GM_CASE(NBV)                                                                                       \
    case NBV:                                                                                              \
        bgram_skinny_kernel<T, NBV, false><<<c->grid_gram, kGramThreads, kGramSmem, c->stream>>>(          \
            B, basis, k, vcol, which, rrow, statidx, mode);                                                \
        return cudaGetLastError();
                GM_CASE(1) GM_CASE(2) GM_CASE(3) GM_CASE(4) GM_CASE(5) GM_CASE(6) GM_CASE(7) GM_CASE(8)
                GM_CASE(9) GM_CASE(10) GM_CASE(11) GM_CASE(12)
#undef GM_CASE
                default: break;
            }
        }
        bgram_wide_kernel<T, DDA><<<c->grid_gram, kGramThreads, kGramSmem, c->stream>>>(B, basis, k, nb, vcol, which,
                                                                                         rrow, statidx, mode);
        return cudaGetLastError();
    }
    switch (nb) {
#define GM_CASE(NBV)                                                                                       \
    case NBV: {                                                                                            \
        static const cudaError_t attr =                                                                    \
            smem_limit(bgram_skinny_kernel<T, NBV, true>, gram_skinny_df_smem(kMaxNB + NBV));              \
        if (attr != cudaSuccess) return attr;                                                              \
        bgram_skinny_kernel<T, NBV, true><<<c->grid_gram, kGramThreads, gram_skinny_df_smem(k + NBV + NBV), \
                                            c->stream>>>(B, basis, k, vcol, which, rrow, statidx, mode);   \
        return cudaGetLastError();                                                                         \
    }
        GM_CASE(1) GM_CASE(2) GM_CASE(3) GM_CASE(4) GM_CASE(5) GM_CASE(6) GM_CASE(7) GM_CASE(8)
#undef GM_CASE
        default: break;
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_bgram(gmres_batch* c, T* basis, int k, int nb, int vcol, int which, int rrow, int statidx,
                         int mode) {
    return c->opts.arith == GMRES_ARITH_DD ? launch_bgram_t<T, true>(c, basis, k, nb, vcol, which, rrow, statidx, mode)
                                           : launch_bgram_t<T, false>(c, basis, k, nb, vcol, which, rrow, statidx, mode);
}

template <typename T, bool DDA>
cudaError_t launch_bupdate_t(gmres_batch* c, T* basis, int k, int nb, int vcol, int which, int rrow, int statidx,
                             int mode) {
    const BatchDev& B = c->B;
    switch (nb) {
#define GM_CASE(NBV)                                                                                          \
    case NBV:                                                                                                 \
        bupdate_skinny_kernel<T, NBV, DDA><<<c->grid_rows, kTile, 0, c->stream>>>(B, basis, k, vcol, which,   \
                                                                                   rrow, statidx, mode);      \
        return cudaGetLastError();
        GM_CASE(1) GM_CASE(2) GM_CASE(3) GM_CASE(4) GM_CASE(5) GM_CASE(6) GM_CASE(7) GM_CASE(8)
        GM_CASE(9) GM_CASE(10) GM_CASE(11) GM_CASE(12) GM_CASE(13) GM_CASE(14) GM_CASE(15) GM_CASE(16)
#undef GM_CASE
        default: break;
    }
    static const cudaError_t attr = smem_limit(bupdate_wide_kernel<T, DDA>, kBWideSmem);
    if (attr != cudaSuccess) return attr;
    bupdate_wide_kernel<T, DDA><<<c->grid_rows, DDA ? 256 : 128, kBWideSmem, c->stream>>>(B, basis, k, nb, vcol, which,
                                                                                        rrow, statidx, mode);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bupdate(gmres_batch* c, T* basis, int k, int nb, int vcol, int which, int rrow, int statidx,
                           int mode) {
    return c->opts.arith == GMRES_ARITH_DD
               ? launch_bupdate_t<T, true>(c, basis, k, nb, vcol, which, rrow, statidx, mode)
               : launch_bupdate_t<T, false>(c, basis, k, nb, vcol, which, rrow, statidx, mode);
}

// One restart cycle for every active system (the sequence captured in the graph).
template <typename T>
cudaError_t enqueue_cycle(gmres_batch* c) {
    const gmres_opts& o = c->opts;
    const BatchDev& B = c->B;
    cudaStream_t s = c->stream;
    T* basis = static_cast<T*>(c->basis);
    const T* vals = sizeof(T) == sizeof(double) ? reinterpret_cast<const T*>(c->d_vals)
                                                : reinterpret_cast<const T*>(c->d_vals32);
    const int nblk = o.m / o.s;
    int panel_idx = 0;
    bcycle_begin_kernel<<<c->nsys, 64, 0, s>>>(B);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        bscale_kernel<T><<<c->grid_rows, kTile, 0, s>>>(B, c->d_r, basis);
        e = cudaGetLastError();
    }
    for (int j = 0; j < nblk && e == cudaSuccess; ++j) {
        const int st0 = j * o.s;
        for (int i = 0; i < o.s && e == cudaSuccess; ++i) {
            bspmv_kernel<T><<<c->grid_rows, kTile, 0, s>>>(B, c->d_rowptr, c->d_colind, vals, basis, st0 + i,
                                                            st0 + i + 1, i);
            e = cudaGetLastError();
        }
        const int k = st0 + 1;
        if (e != cudaSuccess) break;
        if (sizeof(T) == sizeof(double)) {
            e = launch_bgram<T>(c, basis, k, o.s, k, 0, 0, j, 0);
            if (e == cudaSuccess) e = launch_bupdate<T>(c, basis, k, o.s, k, 0, 0, j, 0);
        } else {
            e = launch_bgram<T>(c, basis, k, o.s, k, 0, 0, j, kPipGramOnly);
            if (e == cudaSuccess) e = launch_bupdate<T>(c, basis, k, o.s, k, 0, 0, j, kPipNoTrsm);
            if (e == cudaSuccess) e = launch_bgram<T>(c, basis, 0, o.s, k, 0, k, j, 0);
            if (e == cudaSuccess) e = launch_bupdate<T>(c, basis, 0, o.s, k, 0, k, j, 0);
        }
        const int t = st0 + o.s;
        if (e == cudaSuccess && t % o.panel == 0) {
            const int lo = (t == o.panel) ? 0 : t - o.panel + 1;
            const int np = t - lo + 1;
            const int sidx = nblk + panel_idx;
            e = launch_bgram<T>(c, basis, lo, np, lo, 1, 0, sidx, 0);
            if (e == cudaSuccess) e = launch_bupdate<T>(c, basis, lo, np, lo, 1, 0, sidx, 0);
            if (e == cudaSuccess) {
                bhess_kernel<<<c->nsys, kLsThreads, hessenberg_ls_smem(), s>>>(B, lo, t);
                e = cudaGetLastError();
            }
            ++panel_idx;
        }
    }
    if (e == cudaSuccess) {
        bxupdate_kernel<T><<<c->grid_rows, kTile, 0, s>>>(B, basis, c->d_x);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t enqueue_cycle_any(gmres_batch* c) {
    return c->opts.precision == GMRES_PREC_MIXED ? enqueue_cycle<float>(c) : enqueue_cycle<double>(c);
}

}  // namespace

extern "C" {

int gmres_batch_destroy(gmres_batch* c) {
    if (!c) return GMRES_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    void* ptrs[] = {c->d_sys, c->d_vsys, c->d_tsys, c->d_active, c->d_st, c->d_rowptr, c->d_colind, c->d_vals,
                    c->d_vals32, c->basis, c->d_b, c->d_x, c->d_r, c->d_partial, c->d_counter, c->d_gram,
                    c->d_tpart, c->d_tcount};
    for (void* p : ptrs) cudaFree(p);
    cudaFreeHost(c->h_st);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return GMRES_OK;
}

// The options a batch accepts (GMRES_ERR_ARG with the reason otherwise).
static int check_batch_opts(const gmres_opts& o) {
    GM_ARG(o.m >= 1 && o.m + 1 <= kMaxCols && o.s >= 1 && o.s <= 16 && o.panel % o.s == 0 && o.m % o.panel == 0,
           "need s | panel | m, m + 1 <= 64, s <= 16");
    GM_ARG(o.precision == GMRES_PREC_FP64 || o.precision == GMRES_PREC_MIXED, "unknown precision");
    GM_ARG(o.tol > 0.0 && o.max_restarts >= 1, "bad tol / max_restarts");
    GM_ARG(o.arith == GMRES_ARITH_FP64 || o.arith == GMRES_ARITH_DD,
           "arith must be GMRES_ARITH_FP64 or GMRES_ARITH_DD for batches");
    GM_ARG(o.ortho == GMRES_ORTHO_TWO_STAGE || o.ortho == GMRES_ORTHO_BCGS_PIP2,
           "ortho must be GMRES_ORTHO_TWO_STAGE or GMRES_ORTHO_BCGS_PIP2 for batches");
    GM_ARG(o.shift == GMRES_SHIFT_NONE, "shifted CholQR (opts.shift) is not available in the batched engine");
    GM_ARG(o.precond == GMRES_PRECOND_NONE, "the Gauss-Seidel preconditioner is not available in the batched engine");
    GM_ARG(o.basis == GMRES_BASIS_MONOMIAL || o.basis == GMRES_BASIS_NEWTON,
           "basis must be GMRES_BASIS_MONOMIAL or GMRES_BASIS_NEWTON for batches (pass the shifts in opts.theta)");
    return GMRES_OK;
}

size_t gmres_batch_footprint(int32_t nsys, const int64_t* n, const int64_t* nnz, const gmres_opts* opts) {
    if (nsys <= 0 || !n || !nnz) return 0;
    gmres_opts o;
    if (opts) o = *opts; else gmres_default_opts(&o);
    if (o.ortho == GMRES_ORTHO_BCGS_PIP2) o.panel = o.s;
    if (check_batch_opts(o)) return 0;
    const size_t esz = o.precision == GMRES_PREC_MIXED ? 4 : 8;
    size_t rows = 0, nz = 0, vt = 0;
    for (int i = 0; i < nsys; ++i) {
        if (n[i] < 1 || nnz[i] < 0) return 0;
        rows += (size_t)((n[i] + 31) / 32 * 32);
        nz += (size_t)nnz[i];
        vt += (size_t)reduction_grid(n[i]);
    }
    size_t b = rows * (size_t)(o.m + 1) * esz;                 // basis
    b += rows * 8 * (o.precision == GMRES_PREC_MIXED ? 3 : 2);  // b, x (, r)
    b += (rows + nsys) * 4 + nz * (4 + 8 + (o.precision == GMRES_PREC_MIXED ? 4 : 0));  // CSR
    const size_t nbmax = (size_t)std::max(o.s, o.panel + 1);
    b += vt * kMaxNB * nbmax * 8 + (size_t)nsys * (sizeof(DevState) + kMaxNB * kMaxNB * 8 + 64);
    b += rows / kTile * 12 + (size_t)nsys * 64;
    return b;
}

int gmres_batch_create(gmres_batch** out, int32_t nsys, const int64_t* n, const int64_t* const* rowptr,
                       const int32_t* const* colind, const double* const* vals, const gmres_opts* opts,
                       void* stream) {
    clear_error();
    GM_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    GM_ARG(nsys >= 1 && n && rowptr && colind && vals, "need nsys >= 1 and non-NULL arrays");
    gmres_opts o;
    if (opts) o = *opts; else gmres_default_opts(&o);
    if (o.ortho == GMRES_ORTHO_BCGS_PIP2) o.panel = o.s;
    {
        const int rc = check_batch_opts(o);
        if (rc) return rc;
    }
    gmres_batch* c = new gmres_batch();
    c->opts = o;
    c->nsys = nsys;
    auto fail = [&](int rc) { gmres_batch_destroy(c); return rc; };
    if (cudaGetDevice(&c->device) != cudaSuccess) return fail(cuda_rc_b(cudaGetLastError(), "cudaGetDevice"));
    // the least-squares kernel stages its matrices in dynamic shared memory (set
    // here, before any cycle is captured into a graph)
    if (cudaFuncSetAttribute(bhess_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hessenberg_ls_smem()) !=
        cudaSuccess)
        return fail(cuda_rc_b(cudaGetLastError(), "cudaFuncSetAttribute"));
    if (stream) {
        c->stream = static_cast<cudaStream_t>(stream);
    } else {
        // graph capture needs a stream other than the legacy default stream
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(cuda_rc_b(cudaGetLastError(), "cudaStreamCreate"));
        c->own_stream = true;
    }
    cudaStream_t s = c->stream;
    // system table, tiles, virtual CTAs, concatenated block-diagonal CSR
    int64_t row0 = 0, nnz_tot = 0;
    int32_t v0 = 0, t0 = 0;
    // argument errors from here on release the context (and its stream)
#define BARG(cond, ...)                        \
    do {                                       \
        if (!(cond)) {                         \
            set_error(__VA_ARGS__);            \
            return fail(GMRES_ERR_ARG);        \
        }                                      \
    } while (0)
    for (int i = 0; i < nsys; ++i) {
        BARG(n[i] >= 1, "system %d: n must be >= 1", i);
        const int64_t nz = rowptr[i][n[i]];
        BARG(rowptr[i][0] == 0 && nz >= 0, "system %d: rowptr must start at 0", i);
        BSys S;
        S.n = n[i];
        S.row0 = row0;
        S.G = reduction_grid(n[i]);
        S.v0 = v0;
        S.nt = (int32_t)((n[i] + kTile - 1) / kTile);
        S.t0 = t0;
        c->hsys.push_back(S);
        for (int q = 0; q < S.G; ++q) c->hvsys.push_back(i);
        for (int q = 0; q < S.nt; ++q) c->htsys.push_back(i);
        v0 += S.G;
        t0 += S.nt;
        row0 += (n[i] + 31) / 32 * 32;
        nnz_tot += nz;
    }
    BARG(nnz_tot < (int64_t(1) << 31) && row0 < (int64_t(1) << 31), "batch too large for 32-bit CSR indices");
#undef BARG
    c->ntot = row0;
    std::vector<int32_t> rp(row0 + 1), ci(nnz_tot > 0 ? nnz_tot : 1);
    std::vector<double> vv(nnz_tot > 0 ? nnz_tot : 1);
    {
        int64_t p = 0;
        for (int i = 0; i < nsys; ++i) {
            const BSys& S = c->hsys[i];
            const int64_t rows_pad = (S.n + 31) / 32 * 32;
            for (int64_t r = 0; r < rows_pad; ++r) {
                rp[S.row0 + r] = (int32_t)p;
                if (r < S.n) {
                    for (int64_t q = rowptr[i][r]; q < rowptr[i][r + 1]; ++q) {
                        const int32_t col = colind[i][q];
                        if (col < 0 || col >= S.n || rowptr[i][r + 1] < rowptr[i][r]) {
                            set_error("system %d: invalid CSR (row %lld)", i, (long long)r);
                            return fail(GMRES_ERR_ARG);
                        }
                        ci[p] = (int32_t)(S.row0 + col);
                        vv[p] = vals[i][q];
                        ++p;
                    }
                }
            }
        }
        rp[row0] = (int32_t)p;
    }
    const size_t esz = o.precision == GMRES_PREC_MIXED ? sizeof(float) : sizeof(double);
    const int vtot = v0, ttot = t0;
#define BK(call, what) do { int rc_ = cuda_rc_b((call), what); if (rc_) return fail(rc_); } while (0)
    BK(cudaMalloc(&c->d_sys, nsys * sizeof(BSys)), "cudaMalloc");
    BK(cudaMalloc(&c->d_vsys, vtot * sizeof(int32_t)), "cudaMalloc");
    BK(cudaMalloc(&c->d_tsys, ttot * sizeof(int32_t)), "cudaMalloc");
    BK(cudaMalloc(&c->d_active, nsys * sizeof(int32_t)), "cudaMalloc");
    BK(cudaMalloc(&c->d_st, nsys * sizeof(DevState)), "cudaMalloc state");
    BK(cudaMalloc(&c->d_rowptr, (row0 + 1) * sizeof(int32_t)), "cudaMalloc rowptr");
    BK(cudaMalloc(&c->d_colind, ci.size() * sizeof(int32_t)), "cudaMalloc colind");
    BK(cudaMalloc(&c->d_vals, vv.size() * sizeof(double)), "cudaMalloc vals");
    BK(cudaMalloc(&c->basis, (size_t)(o.m + 1) * row0 * esz), "cudaMalloc basis");
    BK(cudaMalloc(&c->d_b, row0 * sizeof(double)), "cudaMalloc b");
    BK(cudaMalloc(&c->d_x, row0 * sizeof(double)), "cudaMalloc x");
    BK(cudaMalloc(&c->d_r, row0 * sizeof(double)), "cudaMalloc r");
    const int nbmax = std::max(o.s, o.panel + 1);   // widest Gram block of a cycle
    BK(cudaMalloc(&c->d_partial, (size_t)vtot * kMaxNB * nbmax * sizeof(double)), "cudaMalloc partial");
    BK(cudaMalloc(&c->d_counter, (size_t)nsys * 8 * sizeof(unsigned)), "cudaMalloc counter");
    BK(cudaMalloc(&c->d_gram, (size_t)nsys * kMaxNB * kMaxNB * sizeof(double)), "cudaMalloc gram");
    BK(cudaMalloc(&c->d_tpart, ttot * sizeof(double)), "cudaMalloc tpart");
    BK(cudaMalloc(&c->d_tcount, nsys * sizeof(unsigned)), "cudaMalloc tcount");
    BK(cudaMallocHost(&c->h_st, nsys * sizeof(DevState)), "cudaMallocHost");
    if (o.precision == GMRES_PREC_MIXED) BK(cudaMalloc(&c->d_vals32, vv.size() * sizeof(float)), "cudaMalloc vals32");
    BK(cudaMemcpyAsync(c->d_sys, c->hsys.data(), nsys * sizeof(BSys), cudaMemcpyHostToDevice, s), "copy");
    BK(cudaMemcpyAsync(c->d_vsys, c->hvsys.data(), vtot * sizeof(int32_t), cudaMemcpyHostToDevice, s), "copy");
    BK(cudaMemcpyAsync(c->d_tsys, c->htsys.data(), ttot * sizeof(int32_t), cudaMemcpyHostToDevice, s), "copy");
    BK(cudaMemcpyAsync(c->d_rowptr, rp.data(), rp.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s), "copy");
    BK(cudaMemcpyAsync(c->d_colind, ci.data(), ci.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s), "copy");
    BK(cudaMemcpyAsync(c->d_vals, vv.data(), vv.size() * sizeof(double), cudaMemcpyHostToDevice, s), "copy");
    if (o.precision == GMRES_PREC_MIXED)
        BK(launch_narrow_vals(s, (int64_t)vv.size(), c->d_vals, c->d_vals32), "narrow vals");
    BK(cudaMemsetAsync(c->basis, 0, (size_t)(o.m + 1) * row0 * esz, s), "memset");
    BK(cudaMemsetAsync(c->d_x, 0, row0 * sizeof(double), s), "memset");
    BK(cudaMemsetAsync(c->d_b, 0, row0 * sizeof(double), s), "memset");
    BK(cudaMemsetAsync(c->d_r, 0, row0 * sizeof(double), s), "memset");
    BK(cudaMemsetAsync(c->d_counter, 0, (size_t)nsys * 8 * sizeof(unsigned), s), "memset");
    BK(cudaMemsetAsync(c->d_tcount, 0, nsys * sizeof(unsigned), s), "memset");
    // per-system state: MPK scale (power of two of the row-sum norm, or opts.sigma)
    c->hst_init.assign(nsys, DevState{});
    for (int i = 0; i < nsys; ++i) {
        DevState& d = c->hst_init[i];
        std::memset(&d, 0, sizeof(DevState));
        d.m = o.m;
        d.s = o.s;
        d.panel = o.panel;
        double rmax = 0.0;
        for (int64_t r = 0; r < n[i]; ++r) {
            double acc = 0.0;
            for (int64_t q = rowptr[i][r]; q < rowptr[i][r + 1]; ++q) acc += std::fabs(vals[i][q]);
            rmax = std::max(rmax, acc);
        }
        d.sigma = o.sigma > 0.0 ? o.sigma
                                : ((rmax > 0.0 && std::isfinite(rmax)) ? std::ldexp(1.0, (int)std::floor(std::log2(rmax)))
                                                                       : 1.0);
        for (int q = 0; q < 16; ++q) d.theta[q] = o.basis == GMRES_BASIS_NEWTON ? o.theta[q] : 0.0;
    }
    BK(cudaMemcpyAsync(c->d_st, c->hst_init.data(), nsys * sizeof(DevState), cudaMemcpyHostToDevice, s), "copy");
    BK(cudaStreamSynchronize(s), "sync");
    c->B.sys = c->d_sys;
    c->B.vsys = c->d_vsys;
    c->B.tsys = c->d_tsys;
    c->B.nsys = nsys;
    c->B.vtot = vtot;
    c->B.ttot = ttot;
    c->B.ld = row0;
    c->B.st = c->d_st;
    c->B.active = c->d_active;
    c->B.partial = c->d_partial;
    c->B.counter = c->d_counter;
    c->B.gram = c->d_gram;
    c->B.tpart = c->d_tpart;
    c->B.tcount = c->d_tcount;
    c->grid_gram = std::min(vtot, 2 * num_sms());
    c->grid_rows = std::min(ttot, 8 * num_sms());
#undef BK
    *out = c;
    return GMRES_OK;
}

// Autotune the persistent grid sizes of the batched Gram and row kernels on
// the batch's own shapes: each candidate runs the stage-1 Gram of the widest
// block (and the matching update) on the current basis contents; the fastest
// is kept.  The per-system reduction split is a function of n alone, so the
// choice changes speed, never results.  Results are written to res_ms[4]
// (best Gram ms, best update ms, Gram grid, row grid) when non-NULL.
int gmres_batch_autotune(gmres_batch* c, double* res_ms) {
    clear_error();
    GM_ARG(c != nullptr, "NULL batch");
    const gmres_opts& o = c->opts;
    cudaStream_t s = c->stream;
    const int k = o.m - o.s + 1;   // the widest stage-1 block of a cycle
    // all systems active, nothing converged: a benign state for timing
    std::vector<int32_t> ones(c->nsys, 1);
    int rc = cuda_rc_b(cudaMemcpyAsync(c->d_active, ones.data(), c->nsys * 4, cudaMemcpyHostToDevice, s), "copy");
    if (rc) return rc;
    bcycle_begin_kernel<<<c->nsys, 64, 0, s>>>(c->B);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int sms = num_sms();
    float best_g = 1e30f, best_u = 1e30f;
    int pick_g = c->grid_gram, pick_u = c->grid_rows;
    const int gmult[] = {1, 2, 3, 4};
    const int umult[] = {2, 4, 8, 16};
    for (int q = 0; q < 4; ++q) {
        c->grid_gram = std::max(1, std::min(c->B.vtot, gmult[q] * sms));
        c->grid_rows = std::max(1, std::min(c->B.ttot, umult[q] * sms));
        float tg = 0.f, tu = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(a, s);
            cudaError_t e = o.precision == GMRES_PREC_MIXED
                                ? launch_bgram<float>(c, static_cast<float*>(c->basis), k, o.s, k, 0, 0, 0, kPipGramOnly)
                                : launch_bgram<double>(c, static_cast<double*>(c->basis), k, o.s, k, 0, 0, 0,
                                                       kPipGramOnly);
            cudaEventRecord(b, s);
            if (e != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) {
                cudaEventDestroy(a);
                cudaEventDestroy(b);
                return cuda_rc_b(e != cudaSuccess ? e : cudaGetLastError(), "autotune gram");
            }
            cudaEventElapsedTime(&tg, a, b);
            cudaEventRecord(a, s);
            e = o.precision == GMRES_PREC_MIXED
                    ? launch_bupdate<float>(c, static_cast<float*>(c->basis), k, o.s, k, 0, 0, 0, kPipNoTrsm)
                    : launch_bupdate<double>(c, static_cast<double*>(c->basis), k, o.s, k, 0, 0, 0, kPipNoTrsm);
            cudaEventRecord(b, s);
            if (e != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) {
                cudaEventDestroy(a);
                cudaEventDestroy(b);
                return cuda_rc_b(e != cudaSuccess ? e : cudaGetLastError(), "autotune update");
            }
            cudaEventElapsedTime(&tu, a, b);
        }
        if (tg < best_g) { best_g = tg; pick_g = c->grid_gram; }
        if (tu < best_u) { best_u = tu; pick_u = c->grid_rows; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    c->grid_gram = pick_g;
    c->grid_rows = pick_u;
    if (c->graph) {   // the captured cycle used the old grid sizes
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    // leave the basis and state as a fresh solve expects them
    rc = cuda_rc_b(cudaMemsetAsync(c->basis, 0, (size_t)(o.m + 1) * c->ntot *
                                                    (o.precision == GMRES_PREC_MIXED ? 4 : 8), s), "memset");
    if (!rc) rc = cuda_rc_b(cudaMemsetAsync(c->d_counter, 0, (size_t)c->nsys * 8 * sizeof(unsigned), s), "memset");
    if (!rc) rc = cuda_rc_b(cudaStreamSynchronize(s), "sync");
    if (res_ms) {
        res_ms[0] = best_g;
        res_ms[1] = best_u;
        res_ms[2] = pick_g;
        res_ms[3] = pick_u;
    }
    return rc;
}

int gmres_batch_solve(gmres_batch* c, const double* const* b, double* const* x, gmres_result* res) {
    clear_error();
    GM_ARG(c != nullptr && b != nullptr && x != nullptr, "NULL argument");
    for (int i = 0; i < c->nsys; ++i) GM_ARG(b[i] != nullptr && x[i] != nullptr, "system %d: NULL b or x", i);
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_rc_b(cudaGetLastError(), "cudaSetDevice");
    const gmres_opts& o = c->opts;
    cudaStream_t s = c->stream;
    const int ns = c->nsys;
    int rc = GMRES_OK;
    // inputs: b, x0 into the concatenated vectors
    for (int i = 0; i < ns && !rc; ++i) {
        const BSys& S = c->hsys[i];
        rc = cuda_rc_b(cudaMemcpyAsync(c->d_b + S.row0, b[i], S.n * sizeof(double), cudaMemcpyHostToDevice, s), "copy b");
        if (!rc) rc = cuda_rc_b(cudaMemcpyAsync(c->d_x + S.row0, x[i], S.n * sizeof(double), cudaMemcpyHostToDevice, s),
                                "copy x");
    }
    if (rc) return rc;
    std::vector<int32_t> active(ns, 1);
    std::vector<gmres_result> out(ns);
    std::vector<double> bnorm(ns);
    for (int i = 0; i < ns; ++i) {
        out[i] = gmres_result{};
        out[i].breakdown_block = -1;
        out[i].status = GMRES_WARN_MAXIT;
    }
    // fresh per-system state and ||b||
    rc = cuda_rc_b(cudaMemcpyAsync(c->d_st, c->hst_init.data(), ns * sizeof(DevState), cudaMemcpyHostToDevice, s),
                   "state");
    if (!rc) rc = cuda_rc_b(cudaMemcpyAsync(c->d_active, active.data(), ns * 4, cudaMemcpyHostToDevice, s), "copy");
    if (!rc) {
        bresidual_kernel<<<c->grid_rows, kTile, 0, s>>>(c->B, c->d_rowptr, c->d_colind, c->d_vals, c->d_b, nullptr,
                                                         nullptr, 1);
        rc = cuda_rc_b(cudaGetLastError(), "norm b");
    }
    if (!rc) rc = cuda_rc_b(cudaMemcpyAsync(c->h_st, c->d_st, ns * sizeof(DevState), cudaMemcpyDeviceToHost, s), "read");
    if (!rc) rc = cuda_rc_b(cudaStreamSynchronize(s), "sync");
    if (rc) return rc;
    for (int i = 0; i < ns; ++i) {
        bnorm[i] = c->h_st[i].bnorm;
        c->hst_init[i].bnorm = bnorm[i];
        c->hst_init[i].tol_abs = o.tol * bnorm[i];
        if (!std::isfinite(bnorm[i])) { active[i] = 0; out[i].status = GMRES_ERR_NAN; }
        else if (bnorm[i] == 0.0) { active[i] = 0; out[i].status = GMRES_OK; }
    }
    rc = cuda_rc_b(cudaMemcpyAsync(c->d_st, c->hst_init.data(), ns * sizeof(DevState), cudaMemcpyHostToDevice, s),
                   "state");
    const int nstat = o.m / o.s + o.m / o.panel;
    for (int cyc = 0; !rc; ++cyc) {
        rc = cuda_rc_b(cudaMemcpyAsync(c->d_active, active.data(), ns * 4, cudaMemcpyHostToDevice, s), "copy");
        if (rc) break;
        bresidual_kernel<<<c->grid_rows, kTile, 0, s>>>(c->B, c->d_rowptr, c->d_colind, c->d_vals, c->d_b, c->d_x,
                                                         c->d_r, 0);
        rc = cuda_rc_b(cudaGetLastError(), "residual");
        if (!rc) rc = cuda_rc_b(cudaMemcpyAsync(c->h_st, c->d_st, ns * sizeof(DevState), cudaMemcpyDeviceToHost, s),
                                "read");
        if (!rc) rc = cuda_rc_b(cudaStreamSynchronize(s), "sync");
        if (rc) break;
        int nact = 0;
        for (int i = 0; i < ns; ++i) {
            if (!active[i]) continue;
            const DevState& h = c->h_st[i];
            gmres_result& r = out[i];
            r.iters = h.iters;
            r.restarts = cyc;
            r.relres_true = h.beta / bnorm[i];
            if (cyc > 0) r.relres_implicit = h.resid / bnorm[i];
            if (o.precision == GMRES_PREC_MIXED) r.ir_steps = cyc;
            bool stop = false;
            for (int q = 0; q < nstat; ++q)
                if (h.blkstat[q]) {
                    r.breakdown_block = q;
                    r.breakdown_pivot = h.blkstat[q];
                    r.status = GMRES_ERR_BREAKDOWN;
                    stop = true;
                    break;
                }
            if (!stop && !std::isfinite(h.beta)) { r.status = GMRES_ERR_NAN; stop = true; }
            if (!stop && h.beta <= o.tol * bnorm[i]) { r.status = GMRES_OK; stop = true; }
            if (!stop && cyc >= o.max_restarts) { r.status = GMRES_WARN_MAXIT; stop = true; }
            if (stop) active[i] = 0; else ++nact;
        }
        if (nact == 0) break;
        rc = cuda_rc_b(cudaMemcpyAsync(c->d_active, active.data(), ns * 4, cudaMemcpyHostToDevice, s), "copy");
        if (rc) break;
        if (!c->graph) {
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e2 = enqueue_cycle_any(c);
                e = cudaStreamEndCapture(s, &g);
                if (e2 != cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, g, 0);
            if (g) cudaGraphDestroy(g);
            rc = cuda_rc_b(e, "cycle graph");
            if (rc) break;
        }
        rc = cuda_rc_b(cudaGraphLaunch(c->graph, s), "graph launch");
    }
    if (rc) return rc;
    for (int i = 0; i < ns && !rc; ++i) {
        const BSys& S = c->hsys[i];
        rc = cuda_rc_b(cudaMemcpyAsync(x[i], c->d_x + S.row0, S.n * sizeof(double), cudaMemcpyDeviceToHost, s), "copy x");
    }
    if (!rc) rc = cuda_rc_b(cudaStreamSynchronize(s), "sync");
    if (rc) return rc;
    int worst = GMRES_OK;
    for (int i = 0; i < ns; ++i) {
        if (res) res[i] = out[i];
        if (out[i].status < 0) worst = out[i].status;
        else if (out[i].status > worst && worst >= 0) worst = out[i].status;
    }
    return worst;
}

}  // extern "C"
