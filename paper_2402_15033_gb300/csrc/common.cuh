// Shared helpers of the GB300 s-step GMRES library (host + device).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include "../../include/gmres.h"

namespace gm {

// Thread-local last-error message (gmres_last_error).
void set_error(const char* fmt, ...);
void clear_error();

constexpr int kMaxNB = 64;        // widest block handled by one Gram column group
constexpr int kMaxKX = 256;       // k + nb limit of the standalone ortho calls
constexpr int kGramThreads = 256;

// Number of CTAs of the split-n reductions: enough to fill every SM twice,
// never more CTAs than 64-row chunks.
int reduction_grid(int64_t n);
int num_sms();

// Raises kernel f's dynamic shared-memory limit to `bytes`.  Callers keep the
// result in a function-local static, whose initialization C++ runs once even
// when several host threads launch.
template <class F>
inline cudaError_t smem_limit(F* f, size_t bytes) {
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Layout of the scratch space of one BCGS-PIP call (bytes, 256-aligned pieces).
struct PipWork {
    double* partial;     // [grid][groups][64*64] per-CTA partial Gram blocks
    unsigned* counter;   // [groups] arrival counters of the last-CTA reduce
    double* gram;        // [kx * nb] reduced Gram (column-major, ld = kx)
    size_t bytes;
};
PipWork pip_work_layout(void* base, int64_t n, int k, int nb);

// Device-side status block of one BCGS-PIP (also used by the solver).
struct PipStatus {
    int32_t* status;     // 0 or 1-based bad pivot
};

// Mode bits of the BCGS-PIP launchers.
constexpr int kPipGramOnly = 1;   // Gram kernel: write [P; G] (upper G), no Cholesky, status 0
constexpr int kPipNoTrsm = 2;     // update kernel: V <- V - Q P only (T taken as the identity)
constexpr int kPipShift = 4;      // Gram kernel: factor G - P^T P + sigma I (shifted CholQR, see pip_finish)

// Arithmetic of the Gram and update kernels (gmres_opts.arith).
constexpr int kArithFP64 = 0;     // native FP64 pipe (default)
constexpr int kArithDD = 1;       // double-float on the FP32 pipe (df.cuh), ~2^-48 relative
constexpr int kArithTC = 2;       // Gram and update on the f16 tensor cores by exact slicing (tc_common.cuh)

// ---------------------------------------------------------------- launchers
// BCGS-PIP step 1+2: [P; G] = [Q, V]^T V split over n rows; the last CTA to
// finish reduces the partial blocks in a fixed order, forms G - P^T P, factors
// it, and writes R = [P; T].  Q may be null when k == 0.
cudaError_t launch_pip_gram_chol(cudaStream_t st, int64_t n,
                                 const double* Q, int64_t ldq, int k,
                                 const double* V, int64_t ldv, int nb,
                                 double* R, int ldr, const PipWork& w, int32_t* d_status,
                                 int32_t* d_skip, int grid, int mode = 0, int arith = kArithFP64);
cudaError_t launch_pip_gram_chol(cudaStream_t st, int64_t n,
                                 const float* Q, int64_t ldq, int k,
                                 const float* V, int64_t ldv, int nb,
                                 double* R, int ldr, const PipWork& w, int32_t* d_status,
                                 int32_t* d_skip, int grid, int mode = 0, int arith = kArithFP64);
// BCGS-PIP step 3: V <- (V - Q P) T^{-1}, P and T read from R.
cudaError_t launch_pip_update(cudaStream_t st, int64_t n,
                              const double* Q, int64_t ldq, int k,
                              double* V, int64_t ldv, int nb,
                              const double* R, int ldr, const int32_t* d_status,
                              const int32_t* d_skip, int mode = 0, int arith = kArithFP64);
cudaError_t launch_pip_update(cudaStream_t st, int64_t n,
                              const float* Q, int64_t ldq, int k,
                              float* V, int64_t ldv, int nb,
                              const double* R, int ldr, const int32_t* d_status,
                              const int32_t* d_skip, int mode = 0, int arith = kArithFP64);

// Tensor-core halves with a digit basis (the seven digit slices of basis
// columns kept in HBM, tc_common.cuh): the Gram reads the first kc columns of
// [Q, V] from it; the update writes the new columns' digits into columns
// k .. k+nb-1; the fill slices X(:, 0:nc) into columns c0 ...  Columns of Q, V
// and X must start on 16-byte boundaries; k + nb <= 64.
cudaError_t launch_gram_tc_digits(cudaStream_t st, int64_t n, const double* Q, int64_t ldq, int k, const double* V,
                                  int64_t ldv, int nb, double* R, int ldr, const PipWork& w, int32_t* d_status,
                                  int grid, const void* digits, int capc, int kc, int32_t* d_skip = nullptr,
                                  int mode = 0);
cudaError_t launch_update_tc_digits(cudaStream_t st, int64_t n, const double* Q, int64_t ldq, int k, double* V,
                                    int64_t ldv, int nb, const double* R, int ldr, const int32_t* d_status,
                                    void* digits, int capc, const int32_t* d_skip = nullptr, int mode = 0);
cudaError_t launch_digits_fill_cols(cudaStream_t st, int64_t n, const double* X, int64_t ldx, int c0, int nc,
                                    void* digits, int capc);

}  // namespace gm

#define GM_CUDA_RET(call)                                                              \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            gm::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),       \
                          __FILE__, __LINE__);                                         \
            return e_ == cudaErrorMemoryAllocation ? GMRES_ERR_OOM : GMRES_ERR_CUDA;   \
        }                                                                              \
    } while (0)

#define GM_ARG(cond, ...)                                                              \
    do {                                                                               \
        if (!(cond)) {                                                                 \
            gm::set_error(__VA_ARGS__);                                                \
            return GMRES_ERR_ARG;                                                      \
        }                                                                              \
    } while (0)
