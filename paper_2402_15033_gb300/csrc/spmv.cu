// Sparse and vector kernels of the s-step GMRES cycle (§III):
//   (c) the matrix powers kernel step y = (A x - theta x) / sigma (CSR SpMV),
//   the restart residual r = b - A x with a deterministic norm reduction,
//   the start-vector scaling q_1 = r / ||r||, and the solution update x += Q y.
#include "common.cuh"
#include "solver_state.cuh"

namespace gm {

namespace {

constexpr int kVecThreads = 256;

// Block-wide sum in a fixed order (warp butterflies, then warp 0 over warps).
__device__ double block_sum(double v) {
    __shared__ double s_w[kVecThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) s_w[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < (int)(blockDim.x >> 5) ? s_w[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    }
    return t;  // valid in thread 0
}

// y = (A x - theta w - nu z) * sinv in the basis precision T (FP64, or FP32
// for the mixed-precision MPK with an FP32 copy of the values); w = x, or,
// with a right preconditioner, the unpreconditioned vector x = M^{-1} w came
// from; z the basis vector before w (the three-term term of the Chebyshev
// basis, nu = 0 otherwise).
template <typename T>
__global__ void __launch_bounds__(kVecThreads)
spmv_kernel(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
            const T* __restrict__ vals, const T* __restrict__ x, T* __restrict__ y,
            T theta, T sinv, const int32_t* d_skip, const T* __restrict__ w, const T* __restrict__ z, T nu) {
    if (d_skip && *d_skip) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p0 = __ldg(rowptr + i), p1 = __ldg(rowptr + i + 1);
        T acc = T(0);
        for (int32_t p = p0; p < p1; ++p) acc = fma(__ldg(vals + p), __ldg(x + __ldg(colind + p)), acc);
        if (theta != T(0)) acc = fma(-theta, w[i], acc);
        if (nu != T(0)) acc = fma(-nu, z[i], acc);
        y[i] = acc * sinv;
    }
}

// One color of a forward multicolor Gauss-Seidel sweep (the local
// Gauss-Seidel preconditioner of §VIII, Fig. 9): every row i of the color,
// z_i = (r_i - sum_j a_ij z_j) / a_ii, the sum over the row in CSR order with
// z_i itself still zero (rows of one color are not coupled, so they update at
// once; colors already swept hold their values, later ones zero).
__global__ void __launch_bounds__(kVecThreads)
gs_color_kernel(int64_t cnt, const int32_t* __restrict__ rows, const int32_t* __restrict__ rowptr,
                const int32_t* __restrict__ colind, const double* __restrict__ vals,
                const double* __restrict__ diag, const double* __restrict__ r, double* z, const int32_t* d_skip) {
    if (d_skip && *d_skip) return;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < cnt;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = __ldg(rows + q);
        const int32_t p0 = __ldg(rowptr + i), p1 = __ldg(rowptr + i + 1);
        double acc = 0.0;
        for (int32_t p = p0; p < p1; ++p) acc = fma(__ldg(vals + p), z[__ldg(colind + p)], acc);
        z[i] = (r[i] - acc) / __ldg(diag + i);
    }
}

// a_ii of every row (0 where the row holds no diagonal entry; any zero or
// non-finite diagonal sets *bad).
__global__ void __launch_bounds__(kVecThreads)
diag_kernel(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
            const double* __restrict__ vals, double* diag, int32_t* bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            if (colind[p] == (int32_t)i) d += vals[p];
        diag[i] = d;
        if (!(d != 0.0) || !isfinite(d)) atomicOr(bad, 1);
    }
}

// x += z
__global__ void __launch_bounds__(kVecThreads)
axpy1_kernel(int64_t n, const double* __restrict__ z, double* __restrict__ x, const DevState* st) {
    if (st->k_used == 0) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] += z[i];
}

// r = b - A x (x may be null: r = b); r written to out; ||r||^2 reduced in a
// fixed order by the last CTA into st->beta / st->inv_beta (or st->bnorm).
__global__ void __launch_bounds__(kVecThreads)
residual_kernel(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                const double* __restrict__ vals, const double* __restrict__ b,
                const double* __restrict__ x, double* __restrict__ out, double* partial,
                unsigned* counter, DevState* st, int which) {
    double ss = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double r = b[i];
        if (x) {
            const int32_t p0 = __ldg(rowptr + i), p1 = __ldg(rowptr + i + 1);
            double acc = 0.0;
            for (int32_t p = p0; p < p1; ++p) acc = fma(__ldg(vals + p), __ldg(x + __ldg(colind + p)), acc);
            r -= acc;
        }
        if (out) out[i] = r;
        ss = fma(r, r, ss);
    }
    const double t = block_sum(ss);
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = t;
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    if (threadIdx.x == 0) {
        __threadfence();
        double acc = 0.0;
        for (unsigned bI = 0; bI < gridDim.x; ++bI) acc += __ldcg(partial + bI);
        const double nrm = sqrt(acc);
        if (which == 0) {
            st->beta = nrm;
            st->inv_beta = nrm > 0.0 ? 1.0 / nrm : 0.0;
        } else {
            st->bnorm = nrm;
        }
        *counter = 0u;
    }
}

// out = (T)(v * (1/||r||)): the start vector q_1 of a cycle in the basis precision.
template <typename T>
__global__ void __launch_bounds__(kVecThreads)
scale_kernel(int64_t n, const double* v, T* out, const DevState* st) {
    const double s = st->inv_beta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (T)(v[i] * s);
}

// x += Q[:, 0:k] y with k = st->k_used, y = st->y (FP64 accumulation); with
// assign, x = Q y (the correction a right preconditioner then maps); also
// counts iterations.
template <typename T>
__global__ void __launch_bounds__(kVecThreads)
xupdate_kernel(int64_t n, const T* __restrict__ Q, int64_t ldq, double* __restrict__ x, DevState* st, bool assign) {
    __shared__ double ys[kMaxCols];
    const int k = st->k_used;
    for (int c = threadIdx.x; c < k; c += blockDim.x) ys[c] = st->y[c];
    __syncthreads();
    if (k == 0) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double acc = assign ? 0.0 : x[i];
        for (int c = 0; c < k; ++c) acc = fma((double)__ldg(Q + (int64_t)c * ldq + i), ys[c], acc);
        x[i] = acc;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) st->iters += k;
}

__global__ void narrow_vals_kernel(int64_t m, const double* in, float* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

// CSR sanity check: rowptr[0] = 0, nondecreasing, rowptr[n] = nnz, columns in [0, n).
__global__ void validate_csr_kernel(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* colind,
                                    int32_t* bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p0 = rowptr[i], p1 = rowptr[i + 1];
        if (p1 < p0 || p0 < 0 || (int64_t)p1 > nnz) { atomicOr(bad, 1); continue; }
        for (int32_t p = p0; p < p1; ++p) {
            const int32_t c = colind[p];
            if (c < 0 || (int64_t)c >= n) { atomicOr(bad, 2); break; }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (rowptr[0] != 0 || (int64_t)rowptr[n] != nnz) atomicOr(bad, 4);
    }
}

// max_i sum_j |a_ij| (non-negative doubles compare like their bit patterns)
__global__ void rowabs_kernel(int64_t n, const int32_t* __restrict__ rowptr, const double* __restrict__ vals,
                              unsigned long long* out) {
    double mx = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int32_t p = rowptr[i]; p < rowptr[i + 1]; ++p) acc += fabs(vals[p]);
        mx = fmax(mx, acc);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

// Entries outside [0, nnz] become -1, which the CSR validation rejects (a plain
// narrowing could wrap one into a valid-looking offset).
__global__ void rowptr_narrow_kernel(int64_t m, const int64_t* in, int32_t* out, int64_t nnz) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = in[i];
        out[i] = (v < 0 || v > nnz) ? -1 : (int32_t)v;
    }
}

int vec_grid(int64_t n) {
    const int64_t b = (n + kVecThreads - 1) / kVecThreads;
    const int64_t cap = 8 * (int64_t)num_sms();
    return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

int norm_grid(int64_t n) { return vec_grid(n); }

cudaError_t launch_spmv(cudaStream_t st, const DevCSR& A, const double* x, double* y, double theta,
                        double sinv, const int32_t* d_skip, const double* w, const double* z, double nu) {
    spmv_kernel<double><<<vec_grid(A.n), kVecThreads, 0, st>>>(A.n, A.rowptr, A.colind, A.vals, x, y, theta, sinv,
                                                               d_skip, w ? w : x, z ? z : x, z ? nu : 0.0);
    return cudaGetLastError();
}

cudaError_t launch_spmv(cudaStream_t st, const DevCSR& A, const float* x, float* y, double theta,
                        double sinv, const int32_t* d_skip, const float* z, double nu) {
    spmv_kernel<float><<<vec_grid(A.n), kVecThreads, 0, st>>>(A.n, A.rowptr, A.colind, A.vals32, x, y, (float)theta,
                                                              (float)sinv, d_skip, x, z ? z : x,
                                                              z ? (float)nu : 0.0f);
    return cudaGetLastError();
}

cudaError_t launch_gs_sweep(cudaStream_t st, const DevCSR& A, const McGs& gs, const double* r, double* z,
                            const int32_t* d_skip) {
    cudaError_t e = cudaMemsetAsync(z, 0, A.n * sizeof(double), st);
    for (size_t c = 0; c + 1 < gs.off.size() && e == cudaSuccess; ++c) {
        const int64_t cnt = gs.off[c + 1] - gs.off[c];
        gs_color_kernel<<<vec_grid(cnt), kVecThreads, 0, st>>>(cnt, gs.perm + gs.off[c], A.rowptr, A.colind, A.vals,
                                                               gs.diag, r, z, d_skip);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_diag(cudaStream_t st, const DevCSR& A, double* diag, int32_t* bad) {
    diag_kernel<<<vec_grid(A.n), kVecThreads, 0, st>>>(A.n, A.rowptr, A.colind, A.vals, diag, bad);
    return cudaGetLastError();
}

cudaError_t launch_axpy1(cudaStream_t st, int64_t n, const double* z, double* x, const DevState* ds) {
    axpy1_kernel<<<vec_grid(n), kVecThreads, 0, st>>>(n, z, x, ds);
    return cudaGetLastError();
}

cudaError_t launch_residual(cudaStream_t st, const DevCSR& A, const double* b, const double* x, double* out,
                            double* partial, unsigned* counter, DevState* ds, int which) {
    residual_kernel<<<vec_grid(A.n), kVecThreads, 0, st>>>(A.n, A.rowptr, A.colind, A.vals, b, x, out, partial,
                                                           counter, ds, which);
    return cudaGetLastError();
}

cudaError_t launch_scale(cudaStream_t st, int64_t n, const double* v, double* out, const DevState* ds) {
    scale_kernel<double><<<vec_grid(n), kVecThreads, 0, st>>>(n, v, out, ds);
    return cudaGetLastError();
}

cudaError_t launch_scale(cudaStream_t st, int64_t n, const double* v, float* out, const DevState* ds) {
    scale_kernel<float><<<vec_grid(n), kVecThreads, 0, st>>>(n, v, out, ds);
    return cudaGetLastError();
}

cudaError_t launch_xupdate(cudaStream_t st, int64_t n, const double* Q, int64_t ldq, double* x, DevState* ds,
                           bool assign) {
    xupdate_kernel<double><<<vec_grid(n), kVecThreads, 0, st>>>(n, Q, ldq, x, ds, assign);
    return cudaGetLastError();
}

cudaError_t launch_xupdate(cudaStream_t st, int64_t n, const float* Q, int64_t ldq, double* x, DevState* ds,
                           bool assign) {
    xupdate_kernel<float><<<vec_grid(n), kVecThreads, 0, st>>>(n, Q, ldq, x, ds, assign);
    return cudaGetLastError();
}

cudaError_t launch_narrow_vals(cudaStream_t st, int64_t m, const double* in, float* out) {
    narrow_vals_kernel<<<vec_grid(m), kVecThreads, 0, st>>>(m, in, out);
    return cudaGetLastError();
}

cudaError_t launch_validate_csr(cudaStream_t st, int64_t n, int64_t nnz, const int32_t* rowptr,
                                const int32_t* colind, int32_t* bad) {
    validate_csr_kernel<<<vec_grid(n), kVecThreads, 0, st>>>(n, nnz, rowptr, colind, bad);
    return cudaGetLastError();
}

cudaError_t launch_rowabs(cudaStream_t st, const DevCSR& A, unsigned long long* out) {
    rowabs_kernel<<<vec_grid(A.n), kVecThreads, 0, st>>>(A.n, A.rowptr, A.vals, out);
    return cudaGetLastError();
}

cudaError_t launch_rowptr_narrow(cudaStream_t st, int64_t m, const int64_t* in, int32_t* out, int64_t nnz) {
    rowptr_narrow_kernel<<<vec_grid(m), kVecThreads, 0, st>>>(m, in, out, nnz);
    return cudaGetLastError();
}

}  // namespace gm
