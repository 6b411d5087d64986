// ortho_plan: the two-stage block orthogonalization of one panel (§V, Fig. 5)
// as one library call on host or device buffers.
//
// The panel is X = [x_0, V_0, V_1, ..., V_{B-1}]: a unit first column and B
// blocks of s columns.  Stage 1 runs one BCGS-PIP of every block against all
// accumulated columns (k = 1 + s j), stage 2 one BCGS-PIP (= CholQR, k = 0) of
// the whole big panel.  The plan owns the device basis, the digit basis of
// the tensor-core arithmetic, the reduction workspace and the factors, all
// allocated once by ortho_plan_create, so a run allocates nothing.
//
// With host buffers the copies overlap the kernels inside one call: the
// columns travel to the device block by block on a copy stream while the
// earlier blocks' stage 1 runs (each block waits only for its own columns),
// and the stage-2 update runs in row ranges, each range's rows of Q travelling
// back on a second copy stream while the next range is updated.
#include <algorithm>
#include <vector>
#include "common.cuh"
#include "tc_common.cuh"

namespace gm {
namespace {
constexpr int kPlanRanges = 4;        // row ranges of the stage-2 update (host output overlap)
}
}  // namespace gm

using namespace gm;

struct ortho_plan {
    int device = 0;
    int64_t n = 0, ld = 0;
    int s = 0, nblk = 0, ncol = 0, arith = 0;
    cudaStream_t st = nullptr;             // the caller's stream: every kernel
    cudaStream_t h2d = nullptr, d2h = nullptr;
    double* basis = nullptr;               // ncol columns, ld rows
    double* Rh = nullptr;                  // ncol x ncol stage-1 factors (column blocks)
    double* R2 = nullptr;                  // ncol x ncol stage-2 factor
    int32_t* stat = nullptr;               // nblk + 1 statuses
    void* work = nullptr;
    size_t work_bytes = 0;
    void* digits = nullptr;
    std::vector<cudaEvent_t> ev_in, ev_out;
    cudaEvent_t ev_start = nullptr, ev_done = nullptr;
};

extern "C" {

int ortho_plan_destroy(ortho_plan* p) {
    if (!p) return GMRES_OK;
    cudaSetDevice(p->device);
    if (p->st) cudaStreamSynchronize(p->st);
    if (p->h2d) cudaStreamSynchronize(p->h2d);
    if (p->d2h) cudaStreamSynchronize(p->d2h);
    for (auto e : p->ev_in) cudaEventDestroy(e);
    for (auto e : p->ev_out) cudaEventDestroy(e);
    if (p->ev_start) cudaEventDestroy(p->ev_start);
    if (p->ev_done) cudaEventDestroy(p->ev_done);
    if (p->h2d) cudaStreamDestroy(p->h2d);
    if (p->d2h) cudaStreamDestroy(p->d2h);
    cudaFree(p->basis);
    cudaFree(p->Rh);
    cudaFree(p->R2);
    cudaFree(p->stat);
    cudaFree(p->work);
    cudaFree(p->digits);
    delete p;
    return GMRES_OK;
}

int ortho_plan_create(ortho_plan** out, int64_t n, int32_t s, int32_t nblk, int32_t arith, void* stream) {
    clear_error();
    GM_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    GM_ARG(n >= 64, "n must be >= 64");
    GM_ARG(s >= 1 && s <= 16 && nblk >= 1 && 1 + (int64_t)s * nblk <= 64,
           "need 1 <= s <= 16, nblk >= 1 and 1 + s nblk <= 64 columns");
    GM_ARG(arith == GMRES_ARITH_FP64 || arith == GMRES_ARITH_TC, "arith must be GMRES_ARITH_FP64 or _TC");
    ortho_plan* p = new ortho_plan();
    p->n = n;
    p->ld = (n + 31) / 32 * 32;
    p->s = s;
    p->nblk = nblk;
    p->ncol = 1 + s * nblk;
    p->arith = arith;
    p->st = static_cast<cudaStream_t>(stream);
    auto fail = [&](cudaError_t e, const char* what) {
        set_error("ortho_plan_create: %s: %s", what, cudaGetErrorString(e));
        ortho_plan_destroy(p);
        return e == cudaErrorMemoryAllocation ? GMRES_ERR_OOM : GMRES_ERR_CUDA;
    };
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) return fail(e, "cudaGetDevice");
    const int nc = p->ncol;
    p->work_bytes = ortho_workspace_bytes(n, nc, nc);
    if ((e = cudaMalloc(&p->basis, (size_t)nc * p->ld * sizeof(double))) != cudaSuccess) return fail(e, "basis");
    if ((e = cudaMalloc(&p->Rh, (size_t)nc * nc * sizeof(double))) != cudaSuccess) return fail(e, "factors");
    if ((e = cudaMalloc(&p->R2, (size_t)nc * nc * sizeof(double))) != cudaSuccess) return fail(e, "factors");
    if ((e = cudaMalloc(&p->stat, (size_t)(nblk + 1) * sizeof(int32_t))) != cudaSuccess) return fail(e, "status");
    if ((e = cudaMalloc(&p->work, p->work_bytes)) != cudaSuccess) return fail(e, "workspace");
    if (arith == GMRES_ARITH_TC &&
        (e = cudaMalloc(&p->digits, tc_digits_bytes(n, nc))) != cudaSuccess) return fail(e, "digit basis");
    if ((e = cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking)) != cudaSuccess) return fail(e, "stream");
    if ((e = cudaStreamCreateWithFlags(&p->d2h, cudaStreamNonBlocking)) != cudaSuccess) return fail(e, "stream");
    p->ev_in.resize(nblk);
    p->ev_out.resize(kPlanRanges);
    for (auto& x : p->ev_in)
        if ((e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
    for (auto& x : p->ev_out)
        if ((e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
    if ((e = cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
    if ((e = cudaEventCreateWithFlags(&p->ev_done, cudaEventDisableTiming)) != cudaSuccess) return fail(e, "event");
    if ((e = cudaMemsetAsync(p->work, 0, p->work_bytes, p->st)) != cudaSuccess) return fail(e, "memset");
    if (p->digits && (e = cudaMemsetAsync(p->digits, 0, tc_digits_bytes(n, nc), p->st)) != cudaSuccess)
        return fail(e, "memset");
    if ((e = cudaMemsetAsync(p->Rh, 0, (size_t)nc * nc * sizeof(double), p->st)) != cudaSuccess) return fail(e, "memset");
    if ((e = cudaStreamSynchronize(p->st)) != cudaSuccess) return fail(e, "sync");
    *out = p;
    return GMRES_OK;
}

int ortho_plan_run(ortho_plan* p, const double* X, int64_t ldx, double* Q, int64_t ldqo, double* Rhat, double* R2,
                   int32_t ldr, int32_t ptr_on_device, int32_t* block_status) {
    clear_error();
    GM_ARG(p != nullptr && X != nullptr && Q != nullptr, "NULL argument");
    GM_ARG(ldx >= p->n && ldqo >= p->n, "need ldx >= n and ldq >= n");
    GM_ARG((Rhat == nullptr && R2 == nullptr) || ldr >= p->ncol, "need ldr >= 1 + s nblk");
    const int64_t n = p->n, ld = p->ld;
    const int nc = p->ncol, s = p->s;
    const int kind_in = ptr_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const int kind_out = ptr_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    cudaError_t e = cudaSetDevice(p->device);
    double* B = p->basis;
    PipWork w = pip_work_layout(p->work, n, nc, nc);
    const bool tc = p->arith == GMRES_ARITH_TC;
    // the copy streams start after everything already on the caller's stream
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_start, p->st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->h2d, p->ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->d2h, p->ev_start, 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->stat, 0, (size_t)(p->nblk + 1) * sizeof(int32_t), p->st);
    // columns in, block by block (block 0 with column 0)
    for (int j = 0; j < p->nblk && e == cudaSuccess; ++j) {
        const int c0 = j == 0 ? 0 : 1 + s * j, c1 = 1 + s * (j + 1);
        e = cudaMemcpy2DAsync(B + (size_t)c0 * ld, ld * sizeof(double), X + (size_t)c0 * ldx, ldx * sizeof(double),
                              n * sizeof(double), c1 - c0, (cudaMemcpyKind)kind_in, p->h2d);
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_in[j], p->h2d);
    }
    // stage 1: one BCGS-PIP per block against every accumulated column
    for (int j = 0; j < p->nblk && e == cudaSuccess; ++j) {
        const int k = 1 + s * j;
        e = cudaStreamWaitEvent(p->st, p->ev_in[j], 0);
        double* V = B + (size_t)k * ld;
        double* R = p->Rh + (size_t)k * nc;
        if (e == cudaSuccess && tc && j == 0) e = launch_digits_fill_cols(p->st, n, B, ld, 0, 1, p->digits, nc);
        if (e != cudaSuccess) break;
        if (tc) {
            e = launch_gram_tc_digits(p->st, n, B, ld, k, V, ld, s, R, nc, w, p->stat + j, reduction_grid(n), p->digits,
                                      nc, k);
            if (e == cudaSuccess)
                e = launch_update_tc_digits(p->st, n, B, ld, k, V, ld, s, R, nc, p->stat + j, p->digits, nc);
        } else {
            e = launch_pip_gram_chol(p->st, n, B, ld, k, V, ld, s, R, nc, w, p->stat + j, nullptr, reduction_grid(n), 0,
                                     kArithFP64);
            if (e == cudaSuccess)
                e = launch_pip_update(p->st, n, B, ld, k, V, ld, s, R, nc, p->stat + j, nullptr, 0, kArithFP64);
        }
    }
    // stage 2 on the whole panel: the Gram, then the update in row ranges whose
    // rows leave as soon as they are final
    int32_t* st2 = p->stat + p->nblk;
    if (e == cudaSuccess) {
        e = tc ? launch_gram_tc_digits(p->st, n, nullptr, ld, 0, B, ld, nc, p->R2, nc, w, st2, reduction_grid(n),
                                       p->digits, nc, nc)
               : launch_pip_gram_chol(p->st, n, (const double*)nullptr, ld, 0, B, ld, nc, p->R2, nc, w, st2, nullptr,
                                      reduction_grid(n), 0, kArithFP64);
    }
    const int64_t chunk = ((n + kPlanRanges - 1) / kPlanRanges + 63) / 64 * 64;
    int nr = 0;
    for (int64_t r0 = 0; r0 < n && e == cudaSuccess; r0 += chunk, ++nr) {
        const int64_t rows = std::min(chunk, n - r0);
        e = launch_pip_update(p->st, rows, (const double*)nullptr, ld, 0, B + r0, ld, nc, p->R2, nc, st2, nullptr, 0,
                              tc ? kArithTC : kArithFP64);
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_out[nr], p->st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->d2h, p->ev_out[nr], 0);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(Q + r0, ldqo * sizeof(double), B + r0, ld * sizeof(double), rows * sizeof(double), nc,
                                  (cudaMemcpyKind)kind_out, p->d2h);
    }
    if (e == cudaSuccess && Rhat)
        e = cudaMemcpy2DAsync(Rhat, ldr * sizeof(double), p->Rh, nc * sizeof(double), nc * sizeof(double), nc,
                              (cudaMemcpyKind)kind_out, p->d2h);
    if (e == cudaSuccess && R2)
        e = cudaMemcpy2DAsync(R2, ldr * sizeof(double), p->R2, nc * sizeof(double), nc * sizeof(double), nc,
                              (cudaMemcpyKind)kind_out, p->d2h);
    std::vector<int32_t> hs(p->nblk + 1, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hs.data(), p->stat, hs.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, p->d2h);
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_done, p->d2h);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->st, p->ev_done, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
    if (e != cudaSuccess) {
        set_error("ortho_plan_run: %s", cudaGetErrorString(e));
        return GMRES_ERR_CUDA;
    }
    if (block_status) std::copy(hs.begin(), hs.end(), block_status);
    for (int32_t v : hs)
        if (v) {
            set_error("Cholesky breakdown in the two-stage step (block statuses in block_status)");
            return GMRES_ERR_BREAKDOWN;
        }
    return GMRES_OK;
}

}  // extern "C"
