// ortho_stage1_noalloc: the stage-1 block orthogonalization (one BCGS-PIP) for
// callers that cannot allocate device memory.
//
// Some callers have no way to hand this library a scratch buffer: code that
// runs inside another framework's memory arena (the arena owns all device
// memory and forbids cudaMalloc), plug-ins called from a host program that
// never exposes an allocator, and latency-critical loops that cannot afford
// the device-wide synchronization that cudaMalloc/cudaFree imply.  This entry
// point keeps the reduction scratch of the Gram kernel in a fixed array that
// the library itself owns, so the caller passes only inputs and outputs.
//
// The array is file-scope device memory: every GPU that loads the library
// holds kNoAllocScratchBytes of it until the process exits.  Host code never
// dereferences the array's name (on the host it is only a stand-in); the
// device address is looked up once per device with cudaGetSymbolAddress, with
// that device current, on the first call made on that device.
#include <mutex>
#include "common.cuh"

namespace gm {
namespace {

// Enough for k + nb <= 64 and nb <= 16 at any n: 256 B of arrival counters,
// the 64 x 16 reduced Gram and 304 per-CTA partial blocks of 64 x 16 doubles.
constexpr size_t kNoAllocScratchBytes = 2621440;   // 2.5 MiB
constexpr int kNoAllocMaxKX = 64;
constexpr int kNoAllocMaxNB = 16;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
cudaError_t scratch_address(int dev, void** out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch_ptr[dev] == nullptr) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace gm

using namespace gm;

extern "C" int ortho_stage1_noalloc(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k,
                                    double* V, int64_t ldv, int32_t nb, double* R, int32_t ldr,
                                    int32_t* d_status) {
    clear_error();
    GM_ARG(n >= 1, "n must be >= 1");
    GM_ARG(k >= 0 && nb >= 1, "need k >= 0 and nb >= 1");
    GM_ARG(nb <= kNoAllocMaxNB && k + nb <= kNoAllocMaxKX,
           "ortho_stage1_noalloc handles nb <= %d and k + nb <= %d (got k=%d, nb=%d); use ortho_stage1 "
           "with a caller workspace for larger blocks", kNoAllocMaxNB, kNoAllocMaxKX, (int)k, (int)nb);
    GM_ARG(k == 0 || (Q != nullptr && ldq >= n), "Q must be non-NULL with ldq >= n when k > 0");
    GM_ARG(V != nullptr && ldv >= n, "V must be non-NULL with ldv >= n");
    GM_ARG(R != nullptr && ldr >= k + nb, "R must be non-NULL with ldr >= k + nb");
    GM_ARG(d_status != nullptr, "d_status is NULL");
    GM_ARG((reinterpret_cast<uintptr_t>(V) & 15) == 0 && (k == 0 || (reinterpret_cast<uintptr_t>(Q) & 15) == 0),
           "Q and V must be 16-byte aligned");
    const size_t need = ortho_workspace_bytes(n, k, nb);
    GM_ARG(need <= kNoAllocScratchBytes, "scratch of %zu bytes exceeds the %zu-byte static array", need,
           kNoAllocScratchBytes);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess && (dev < 0 || dev >= kMaxDevices)) {
        set_error("device ordinal %d is beyond the %d devices this entry point tracks", dev, kMaxDevices);
        return GMRES_ERR_ARG;
    }
    void* scratch = nullptr;
    if (e == cudaSuccess) e = scratch_address(dev, &scratch);
    if (e != cudaSuccess) {
        set_error("ortho_stage1_noalloc set-up: %s", cudaGetErrorString(e));
        return GMRES_ERR_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PipWork w = pip_work_layout(scratch, n, k, nb);
    // the arrival counters must start at zero; the Gram and partial regions are
    // rewritten in full by the kernel before they are read
    e = cudaMemsetAsync(w.counter, 0, 256, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(int32_t), s);
    if (e == cudaSuccess)
        e = launch_pip_gram_chol(s, n, Q, ldq, k, V, ldv, nb, R, ldr, w, d_status, nullptr, reduction_grid(n));
    if (e == cudaSuccess) e = launch_pip_update(s, n, Q, ldq, k, V, ldv, nb, R, ldr, d_status, nullptr);
    if (e != cudaSuccess) {
        set_error("ortho_stage1_noalloc launch: %s", cudaGetErrorString(e));
        return GMRES_ERR_CUDA;
    }
    return GMRES_OK;
}
