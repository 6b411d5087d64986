// s-step GMRES solver loop (Fig. 1, §III) with two-stage block orthogonalization
// (§V, Fig. 5) and the C ABI of include/gmres.h.
//
// One restart cycle, all on the device, in stream order:
//   r = b - A x, q_1 = r/||r||                       (host reads ||r|| once per cycle)
//   for each s-step block j:
//     MPK: s SpMVs from the block's start column      (kernel (c))
//     stage 1: BCGS-PIP of the s new columns against every accumulated column
//              [Q_{1:l-1}, Q^_{l:j-1}]                (kernels (a)+(d), (b))
//     at the end of a big panel [l, t]:
//       stage 2: BCGS-PIP of Q^_{l:t} against Q_{1:l-1} (CholQR when l = 1)
//       Hessenberg recovery + Givens least squares  (kernel (d), one CTA)
//   x += Q_{1:k} y
// A device flag ("done") makes every later kernel of the cycle return at once
// after convergence at a big-panel end or after a Cholesky breakdown, so a
// cycle is a fixed launch sequence without host round trips.
//
// Mixed precision (GMRES_PREC_MIXED): the basis and the MPK are FP32 (an FP32
// copy of A's values), the Gram products and sums, the Cholesky factors, the
// Hessenberg/Givens work and x stay FP64.  Every restart cycle starts from the
// FP64 residual r = b - A x and ends with x += d, d = Q y: one step of FP64
// iterative refinement whose correction is solved with the FP32 basis.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <vector>
#include <algorithm>
#include <type_traits>
#include "solver_run.cuh"
#include "tc_common.cuh"

namespace gm {

static thread_local char g_err[512];

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }

int num_sms() {
    static const int cached = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            return v;
        return 152;
    }();
    return cached;
}

// A fixed cap (two CTAs on each of GB300's 152 SMs) keeps the reduction tree,
// and therefore the rounding, identical on every device.
int reduction_grid(int64_t n) {
    const int64_t chunks = (n + 127) / 128;
    return (int)(chunks < 304 ? (chunks > 0 ? chunks : 1) : 304);
}

}  // namespace gm

using namespace gm;

struct gmres_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    gmres_opts opts{};
    DevCSR A;
    int64_t n = 0, ldq = 0;
    double sigma = 1.0;
    void* basis = nullptr;       // (m+1) columns, ld = ldq, FP64 or FP32 (opts.precision)
    double* r = nullptr;         // FP64 residual (mixed precision only)
    double* b = nullptr;
    double* x = nullptr;
    double* red_partial = nullptr;
    unsigned* red_counter = nullptr;
    void* pip_work = nullptr;
    size_t pip_bytes = 0;
    double* bscr = nullptr;      // BCGS2-CholQR2: the five reductions' factors (5 x kMaxCols^2)
    void* digits = nullptr;      // tensor-core arithmetic: digit basis of the m+1 columns (tc_common.cuh)
    McGs gs;                     // multicolor Gauss-Seidel preconditioner (opts.precond)
    DevState* st = nullptr;      // device
    DevState* hst = nullptr;     // pinned host mirror
    std::vector<cudaEvent_t> ev;
    // restart cycles as CUDA graphs, one per cycle basis in use (captured on a
    // private stream, launched on `stream`); a basis runs eagerly once first
    struct CycleGraph {
        gm::CycleBasis cb{};
        int runs = 0;
        unsigned long long last = 0;
        cudaGraphExec_t exec = nullptr;
    };
    cudaStream_t cap = nullptr;
    CycleGraph graphs[2];
    // serving: device buffers from the server's memory pool (stream-ordered,
    // no device-wide synchronization), and the slot's capture stream and
    // page-locked state mirror, all owned by the server
    cudaMemPool_t pool = nullptr;
    bool external_slot = false;
    unsigned long long graph_tick = 0;
    bool no_graphs = false;
};

namespace gm {

enum { PH_MPK = 0, PH_S1 = 1, PH_S2 = 2, PH_LS = 3 };

CycleBasis first_cycle_basis(const gmres_opts& o, double sigma);
size_t pip_bytes_for(int64_t n, const gmres_opts& o);
size_t ctx_bytes(int64_t n, int64_t nnz, const gmres_opts& o);
bool uses_digits(const gmres_opts& o);

}  // namespace gm

extern "C" {

const char* gmres_last_error(void) { return g_err; }

int gmres_default_opts(gmres_opts* o) {
    if (!o) return GMRES_ERR_ARG;
    std::memset(o, 0, sizeof(*o));
    o->m = 60;
    o->s = 5;
    o->panel = 60;
    o->max_restarts = 10000;
    o->tol = 1e-8;
    o->sigma = 0.0;
    o->ortho = GMRES_ORTHO_TWO_STAGE;
    o->precision = GMRES_PREC_FP64;
    o->basis = GMRES_BASIS_MONOMIAL;
    o->timing = 0;
    o->inner_tol = 1e-5;
    o->max_ir = 20;
    return GMRES_OK;
}

size_t ortho_workspace_bytes(int64_t n, int32_t k, int32_t nb) {
    if (n <= 0 || k < 0 || nb <= 0) return 0;
    return pip_work_layout(nullptr, n, k, nb).bytes;
}

}  // extern "C"

namespace gm {

// Basis of a solve's first restart cycle: the options' own, or for
// GMRES_BASIS_NEWTON_AUTO standard GMRES, s = 1 with the two-stage panel also
// 1 (each vector re-orthogonalized at once; a single Pythagorean pass over a
// wide panel of s = 1 blocks loses orthogonality as the residual falls).
CycleBasis first_cycle_basis(const gmres_opts& o, double sigma) {
    CycleBasis cb;
    const bool aut = o.basis == GMRES_BASIS_NEWTON_AUTO || o.basis == GMRES_BASIS_CHEBYSHEV_AUTO;
    cb.s = aut ? 1 : o.s;
    cb.panel = (o.ortho == GMRES_ORTHO_TWO_STAGE && !aut) ? o.panel : cb.s;
    cb.sigma = sigma;
    for (int i = 0; i < 16; ++i) cb.theta[i] = (o.basis == GMRES_BASIS_NEWTON && i < o.s) ? o.theta[i] : 0.0;
    if (o.basis == GMRES_BASIS_CHEBYSHEV) {
        // the interval [c - delta, c + delta]: shift c, scale delta / 2 (cheb_coeffs)
        cb.cheb = 1;
        cb.sigma = 0.5 * o.theta[1];
        for (int i = 0; i < 16; ++i) cb.theta[i] = i < o.s ? o.theta[0] : 0.0;
    }
    return cb;
}

// Big panels of a restart cycle: stage 2 runs at every multiple of the panel
// width and at the restart (t = m), so that when the width does not divide m
// the last panel holds the remaining m mod width columns.  The first panel
// starts at column 0 (it holds s^ + 1 vectors), later ones after the previous
// panel's last column.
static bool panel_end(int t, int panel, int m) { return t % panel == 0 || t == m; }
static int panel_start(int t, int panel) {
    const int prev = (t - 1) / panel * panel;
    return prev == 0 ? 0 : prev + 1;
}

size_t pip_bytes_for(int64_t n, const gmres_opts& o) {
    size_t wb = 0;
    auto cover = [&](int s, int panel) {
        for (int st0 = 0; st0 < o.m; st0 += s) {
            wb = std::max(wb, ortho_workspace_bytes(n, st0 + 1, s));
            const int t = st0 + s;
            if (panel_end(t, panel, o.m)) {
                const int lo = panel_start(t, panel);
                wb = std::max(wb, ortho_workspace_bytes(n, lo, t - lo + 1));
            }
        }
    };
    cover(o.s, o.panel);
    const CycleBasis f = first_cycle_basis(o, 1.0);
    if (f.s != o.s) cover(f.s, f.panel);
    return wb;
}

// Device bytes gmres_create allocates for a host-CSR context (each piece
// rounded up to the 256-byte allocation granule).
// The tensor-core arithmetic keeps a digit basis of the FP64 basis (every column
// sliced once; stage 1 reads the accumulated columns' digits).
bool uses_digits(const gmres_opts& o) {
    return o.arith == GMRES_ARITH_TC && o.precision == GMRES_PREC_FP64 && o.m + 1 <= kMaxNB;
}

size_t ctx_bytes(int64_t n, int64_t nnz, const gmres_opts& o) {
    auto up = [](size_t b) { return (b + 511) & ~(size_t)511; };
    const int64_t ldq = (n + 31) / 32 * 32;
    const bool mixed = o.precision == GMRES_PREC_MIXED;
    const size_t esz = mixed ? 4 : 8;
    const size_t nz = (size_t)(nnz > 0 ? nnz : 1);
    size_t b = up((n + 1) * 4) + up(nz * 4) + up(nz * 8);
    if (mixed) b += up(nz * 4) + up(ldq * 8);
    b += up((size_t)(o.m + 1) * ldq * esz) + 2 * up(ldq * 8);
    b += up(norm_grid(n) * 8) + up(256) + up(pip_bytes_for(n, o)) + up(sizeof(DevState)) + up(16);
    if (o.ortho == GMRES_ORTHO_BCGS2_CHOLQR2 || o.shift != GMRES_SHIFT_NONE)
        b += up(5 * (size_t)kMaxCols * kMaxCols * sizeof(double));
    if (uses_digits(o)) b += up(tc_digits_bytes(n, o.m + 1));
    if (o.precond == GMRES_PRECOND_MCGS) b += up(n * 4) + 3 * up(ldq * 8);   // order, diagonal, two vectors
    return b;
}

}  // namespace gm

namespace gm {

// Device memory of a context: cudaMalloc, or the server's pool (stream
// ordered on the context's stream).
static cudaError_t dev_malloc(gmres_ctx* c, void** p, size_t bytes) {
    if (c->pool) return cudaMallocFromPoolAsync(p, bytes, c->pool, c->stream);
    return cudaMalloc(p, bytes);
}
template <typename P>
static cudaError_t dev_malloc(gmres_ctx* c, P** p, size_t bytes) {
    return dev_malloc(c, reinterpret_cast<void**>(p), bytes);
}
static void dev_free(gmres_ctx* c, void* p) {
    if (!p) return;
    if (c->pool) cudaFreeAsync(p, c->stream);
    else cudaFree(p);
}

}  // namespace gm

extern "C" {
static int check_opts(const gmres_opts* o) {
    GM_ARG(o->m >= 1 && o->m + 1 <= kMaxCols, "m must be in [1, %d]", kMaxCols - 1);
    GM_ARG(o->s >= 1 && o->s <= 16, "s must be in [1, 16]");
    GM_ARG(o->tol > 0.0, "tol must be positive");
    GM_ARG(o->max_restarts >= 1, "max_restarts must be >= 1");
    GM_ARG(o->ortho == GMRES_ORTHO_TWO_STAGE || o->ortho == GMRES_ORTHO_BCGS_PIP2 ||
               o->ortho == GMRES_ORTHO_BCGS2_CHOLQR2,
           "unknown ortho");
    GM_ARG(o->precision == GMRES_PREC_FP64 || o->precision == GMRES_PREC_MIXED, "unknown precision");
    GM_ARG(o->basis == GMRES_BASIS_MONOMIAL || o->basis == GMRES_BASIS_NEWTON || o->basis == GMRES_BASIS_NEWTON_AUTO ||
               o->basis == GMRES_BASIS_CHEBYSHEV || o->basis == GMRES_BASIS_CHEBYSHEV_AUTO,
           "unknown basis");
    GM_ARG(o->basis != GMRES_BASIS_CHEBYSHEV ||
               (std::isfinite(o->theta[0]) && o->theta[1] > 0.0 && std::isfinite(o->theta[1])),
           "the Chebyshev basis needs a finite center theta[0] and half-width theta[1] > 0");
    const int panel = o->ortho != GMRES_ORTHO_TWO_STAGE ? o->s : o->panel;
    GM_ARG(panel >= o->s && panel % o->s == 0 && o->m % o->s == 0 && panel <= o->m,
           "need s | panel, s | m and panel <= m");
    GM_ARG(o->sigma >= 0.0 && std::isfinite(o->sigma), "sigma must be >= 0");
    GM_ARG(o->arith == GMRES_ARITH_DD || o->arith == GMRES_ARITH_FP64 || o->arith == GMRES_ARITH_TC,
           "unknown arith");
    GM_ARG(o->shift == GMRES_SHIFT_NONE || o->shift == GMRES_SHIFT_CHOLQR3, "unknown shift");
    GM_ARG(o->precond == GMRES_PRECOND_NONE || o->precond == GMRES_PRECOND_MCGS, "unknown precond");
    GM_ARG(o->precond == GMRES_PRECOND_NONE || o->precision == GMRES_PREC_FP64,
           "the Gauss-Seidel preconditioner needs an FP64 basis (precision = GMRES_PREC_FP64)");
    GM_ARG(o->shift == GMRES_SHIFT_NONE || (o->precision == GMRES_PREC_FP64 && o->ortho != GMRES_ORTHO_BCGS2_CHOLQR2),
           "shifted CholQR needs an FP64 basis and the two-stage or BCGS-PIP2 scheme");
    return GMRES_OK;
}

int gmres_destroy(gmres_ctx* c) {
    if (!c) return GMRES_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (auto e : c->ev) cudaEventDestroy(e);
    for (auto& g : c->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (void* p : {(void*)c->A.rowptr, (void*)c->A.colind, (void*)c->A.vals, (void*)c->A.vals32, (void*)c->r,
                    c->basis, (void*)c->b, (void*)c->x, (void*)c->red_partial, (void*)c->red_counter, c->pip_work,
                    (void*)c->bscr, c->digits, (void*)c->gs.perm, (void*)c->gs.diag, (void*)c->gs.z, (void*)c->gs.t,
                    (void*)c->st})
        dev_free(c, p);
    if (!c->external_slot) {
        cudaFreeHost(c->hst);
        if (c->cap) cudaStreamDestroy(c->cap);
    }
    delete c;
    return GMRES_OK;
}

#define CK(call)                                    \
    do {                                            \
        int rc_ = (call);                           \
        if (rc_ != GMRES_OK) { gmres_destroy(c); return rc_; } \
    } while (0)

static int cuda_rc(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return GMRES_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? GMRES_ERR_OOM : GMRES_ERR_CUDA;
}

// Multicolor Gauss-Seidel set-up (host): greedy distance-1 coloring of the
// symmetrized pattern in natural row order (row i takes the smallest color no
// neighbor j < i holds, a_ij != 0 or a_ji != 0), rows sorted by color (row
// order within a color), the diagonal and two work vectors on the device.
static int setup_mcgs(gmres_ctx* c) {
    const int64_t n = c->n, nnz = c->A.nnz;
    cudaStream_t s = c->stream;
    std::vector<int32_t> rp(n + 1), ci(nnz > 0 ? nnz : 1);
    cudaError_t e = cudaMemcpyAsync(rp.data(), c->A.rowptr, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && nnz > 0)
        e = cudaMemcpyAsync(ci.data(), c->A.colind, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_rc(e, "Gauss-Seidel set-up copy");
    // transpose pattern (rows of A^T), so that both triangles count as neighbors
    std::vector<int64_t> tp(n + 1, 0);
    for (int64_t p = 0; p < nnz; ++p) ++tp[ci[p] + 1];
    for (int64_t i = 0; i < n; ++i) tp[i + 1] += tp[i];
    std::vector<int32_t> tr(nnz > 0 ? nnz : 1);
    {
        std::vector<int64_t> fill(tp.begin(), tp.end() - 1);
        for (int64_t i = 0; i < n; ++i)
            for (int32_t p = rp[i]; p < rp[i + 1]; ++p) tr[fill[ci[p]]++] = (int32_t)i;
    }
    std::vector<int32_t> color(n);
    std::vector<int64_t> mark;
    int ncol = 0;
    for (int64_t i = 0; i < n; ++i) {
        const size_t need = (size_t)(rp[i + 1] - rp[i]) + (size_t)(tp[i + 1] - tp[i]) + 1;
        if (mark.size() < need) mark.resize(need, -1);
        auto take = [&](int32_t j) {
            if (j < i && (size_t)color[j] < mark.size()) mark[color[j]] = i;
        };
        for (int32_t p = rp[i]; p < rp[i + 1]; ++p) take(ci[p]);
        for (int64_t p = tp[i]; p < tp[i + 1]; ++p) take(tr[p]);
        int cc = 0;
        while (mark[cc] == i) ++cc;
        color[i] = cc;
        ncol = std::max(ncol, cc + 1);
    }
    c->gs.off.assign(ncol + 1, 0);
    for (int64_t i = 0; i < n; ++i) ++c->gs.off[color[i] + 1];
    for (int q = 0; q < ncol; ++q) c->gs.off[q + 1] += c->gs.off[q];
    std::vector<int32_t> perm(n);
    {
        std::vector<int64_t> fill(c->gs.off.begin(), c->gs.off.end() - 1);
        for (int64_t i = 0; i < n; ++i) perm[fill[color[i]]++] = (int32_t)i;
    }
    int rc = cuda_rc(dev_malloc(c, &c->gs.perm, n * sizeof(int32_t)), "cudaMalloc Gauss-Seidel order");
    if (!rc) rc = cuda_rc(dev_malloc(c, &c->gs.diag, c->ldq * sizeof(double)), "cudaMalloc diagonal");
    if (!rc) rc = cuda_rc(dev_malloc(c, &c->gs.z, c->ldq * sizeof(double)), "cudaMalloc Gauss-Seidel vector");
    if (!rc) rc = cuda_rc(dev_malloc(c, &c->gs.t, c->ldq * sizeof(double)), "cudaMalloc Gauss-Seidel vector");
    if (rc) return rc;
    int32_t* bad = nullptr;
    e = cudaMemcpyAsync(c->gs.perm, perm.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = dev_malloc(c, &bad, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = launch_diag(s, c->A, c->gs.diag, bad);
    int32_t hb = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(c, bad);
    if (e != cudaSuccess) return cuda_rc(e, "Gauss-Seidel set-up");
    if (hb) {
        set_error("the Gauss-Seidel preconditioner needs a nonzero, finite diagonal in every row");
        return GMRES_ERR_ARG;
    }
    return GMRES_OK;
}

int gmres_create(gmres_ctx** out, int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colind,
                 const double* vals, int32_t ptr_on_device, const gmres_opts* opts, void* stream) {
    return create_ctx(out, n, nnz, rowptr, colind, vals, ptr_on_device, opts, stream, nullptr);
}

}  // extern "C"

namespace gm {

int create_ctx(gmres_ctx** out, int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colind,
               const double* vals, int32_t ptr_on_device, const gmres_opts* opts, void* stream,
               const CtxSlot* slot) {
    clear_error();
    GM_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    GM_ARG(n >= 1, "n must be >= 1");
    GM_ARG(nnz >= 0 && nnz < (int64_t(1) << 31), "nnz must be in [0, 2^31)");
    GM_ARG(rowptr != nullptr && (nnz == 0 || (colind != nullptr && vals != nullptr)), "NULL CSR array");
    gmres_opts o;
    if (opts) o = *opts; else gmres_default_opts(&o);
    if (o.ortho != GMRES_ORTHO_TWO_STAGE) o.panel = o.s;
    {
        int rc = check_opts(&o);
        if (rc) return rc;
    }
    gmres_ctx* c = new gmres_ctx();
    c->opts = o;
    c->n = n;
    c->stream = static_cast<cudaStream_t>(stream);
    if (slot) {
        c->pool = slot->pool;
        c->cap = slot->capture;
        c->hst = slot->host_state;
        c->external_slot = true;
    }
    CK(cuda_rc(cudaGetDevice(&c->device), "cudaGetDevice"));
    cudaStream_t s = c->stream;
    c->ldq = (n + 31) / 32 * 32;
    const int mp1 = o.m + 1;

    c->A.n = n;
    c->A.nnz = nnz;
    CK(cuda_rc(dev_malloc(c, &c->A.rowptr, (n + 1) * sizeof(int32_t)), "cudaMalloc rowptr"));
    CK(cuda_rc(dev_malloc(c, &c->A.colind, (nnz > 0 ? nnz : 1) * sizeof(int32_t)), "cudaMalloc colind"));
    CK(cuda_rc(dev_malloc(c, &c->A.vals, (nnz > 0 ? nnz : 1) * sizeof(double)), "cudaMalloc vals"));
    if (ptr_on_device) {
        int64_t* tmp = nullptr;
        CK(cuda_rc(dev_malloc(c, &tmp, (n + 1) * sizeof(int64_t)), "cudaMalloc tmp"));
        cudaError_t e = cudaMemcpyAsync(tmp, rowptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = launch_rowptr_narrow(s, n + 1, tmp, c->A.rowptr, nnz);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        dev_free(c, tmp);
        CK(cuda_rc(e, "rowptr copy"));
        if (nnz > 0) {
            CK(cuda_rc(cudaMemcpyAsync(c->A.colind, colind, nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, s), "colind copy"));
            CK(cuda_rc(cudaMemcpyAsync(c->A.vals, vals, nnz * sizeof(double), cudaMemcpyDeviceToDevice, s), "vals copy"));
        }
    } else {
        std::vector<int32_t> rp(n + 1);
        for (int64_t i = 0; i <= n; ++i) {
            if (rowptr[i] < 0 || rowptr[i] > nnz) {
                set_error("rowptr[%lld] out of range", (long long)i);
                gmres_destroy(c);
                return GMRES_ERR_ARG;
            }
            rp[i] = (int32_t)rowptr[i];
        }
        CK(cuda_rc(cudaMemcpyAsync(c->A.rowptr, rp.data(), (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s), "rowptr copy"));
        if (nnz > 0) {
            CK(cuda_rc(cudaMemcpyAsync(c->A.colind, colind, nnz * sizeof(int32_t), cudaMemcpyHostToDevice, s), "colind copy"));
            CK(cuda_rc(cudaMemcpyAsync(c->A.vals, vals, nnz * sizeof(double), cudaMemcpyHostToDevice, s), "vals copy"));
        }
        CK(cuda_rc(cudaStreamSynchronize(s), "sync"));
    }
    // validation and the power-of-two MPK scale
    {
        int32_t* bad = nullptr;
        unsigned long long* mx = nullptr;
        CK(cuda_rc(dev_malloc(c, &bad, 16), "cudaMalloc"));
        mx = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(bad) + 8);
        cudaError_t e = cudaMemsetAsync(bad, 0, 16, s);
        if (e == cudaSuccess) e = launch_validate_csr(s, n, nnz, c->A.rowptr, c->A.colind, bad);
        int32_t hb = 0;
        unsigned long long hm = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, bad, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess || hb) dev_free(c, bad);
        CK(cuda_rc(e, "CSR validation"));
        if (hb) {
            set_error("invalid CSR (code %d): rowptr must start at 0, be nondecreasing and end at nnz; "
                      "columns must lie in [0, n)", hb);
            gmres_destroy(c);
            return GMRES_ERR_ARG;
        }
        // only a validated CSR is read row by row
        e = launch_rowabs(s, c->A, mx);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hm, mx, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        dev_free(c, bad);
        CK(cuda_rc(e, "row sums"));
        double rmax;
        std::memcpy(&rmax, &hm, 8);
        if (o.sigma > 0.0) c->sigma = o.sigma;
        else if (o.precond != GMRES_PRECOND_NONE) c->sigma = 1.0;   // A M^{-1} is O(1) for a Gauss-Seidel M
        else c->sigma = (rmax > 0.0 && std::isfinite(rmax)) ? std::ldexp(1.0, (int)std::floor(std::log2(rmax))) : 1.0;
    }
    if (o.precond == GMRES_PRECOND_MCGS) CK(setup_mcgs(c));
    const size_t esz = o.precision == GMRES_PREC_MIXED ? sizeof(float) : sizeof(double);
    CK(cuda_rc(dev_malloc(c, &c->basis, (size_t)mp1 * c->ldq * esz), "cudaMalloc basis"));
    CK(cuda_rc(cudaMemsetAsync(c->basis, 0, (size_t)mp1 * c->ldq * esz, s), "memset basis"));
    if (o.precision == GMRES_PREC_MIXED) {
        CK(cuda_rc(dev_malloc(c, &c->A.vals32, (nnz > 0 ? nnz : 1) * sizeof(float)), "cudaMalloc vals32"));
        if (nnz > 0) CK(cuda_rc(launch_narrow_vals(s, nnz, c->A.vals, c->A.vals32), "narrow vals"));
        CK(cuda_rc(dev_malloc(c, &c->r, c->ldq * sizeof(double)), "cudaMalloc r"));
    }
    CK(cuda_rc(dev_malloc(c, &c->b, c->ldq * sizeof(double)), "cudaMalloc b"));
    CK(cuda_rc(dev_malloc(c, &c->x, c->ldq * sizeof(double)), "cudaMalloc x"));
    const int ng = norm_grid(n);
    CK(cuda_rc(dev_malloc(c, &c->red_partial, ng * sizeof(double)), "cudaMalloc partial"));
    CK(cuda_rc(dev_malloc(c, &c->red_counter, 256), "cudaMalloc counter"));
    CK(cuda_rc(cudaMemsetAsync(c->red_counter, 0, 256, s), "memset counter"));
    // PIP workspace: the largest of the cycle's calls
    const size_t wb = pip_bytes_for(n, o);
    c->pip_bytes = wb;
    CK(cuda_rc(dev_malloc(c, &c->pip_work, wb), "cudaMalloc workspace"));
    CK(cuda_rc(cudaMemsetAsync(c->pip_work, 0, wb, s), "memset workspace"));
    if (uses_digits(o)) {
        const size_t db = tc_digits_bytes(n, o.m + 1);
        CK(cuda_rc(dev_malloc(c, &c->digits, db), "cudaMalloc digit basis"));
        CK(cuda_rc(cudaMemsetAsync(c->digits, 0, db, s), "memset digit basis"));
    }
    if (o.ortho == GMRES_ORTHO_BCGS2_CHOLQR2 || o.shift != GMRES_SHIFT_NONE) {
        // BCGS2-CholQR2: the five reductions' factors; shifted CholQR3: the
        // second and third stage-2 passes' factors and two combine blocks
        const size_t sb = 5 * (size_t)kMaxCols * kMaxCols * sizeof(double);
        CK(cuda_rc(dev_malloc(c, &c->bscr, sb), "cudaMalloc bcgs2 scratch"));
        CK(cuda_rc(cudaMemsetAsync(c->bscr, 0, sb, s), "memset bcgs2 scratch"));
    }
    CK(cuda_rc(dev_malloc(c, &c->st, sizeof(DevState)), "cudaMalloc state"));
    if (!slot) CK(cuda_rc(cudaMallocHost(&c->hst, sizeof(DevState)), "cudaMallocHost state"));
    std::memset(c->hst, 0, sizeof(DevState));
    c->hst->m = o.m;
    c->hst->s = o.s;
    c->hst->panel = o.panel;
    c->hst->sigma = c->sigma;
    for (int i = 0; i < 16; ++i) c->hst->theta[i] = (o.basis == GMRES_BASIS_NEWTON) ? o.theta[i] : 0.0;
    CK(cuda_rc(cudaMemcpyAsync(c->st, c->hst, sizeof(DevState), cudaMemcpyHostToDevice, s), "state upload"));
    CK(cuda_rc(cudaStreamSynchronize(s), "sync"));
    if (o.timing) {
        const CycleBasis f = first_cycle_basis(o, c->sigma);
        const int per_cycle =
            2 * (2 * (o.m / std::min(o.s, f.s)) + 2 * ((o.m + std::min(o.panel, f.panel) - 1) / std::min(o.panel, f.panel))) + 2;
        c->ev.resize(per_cycle);
        for (auto& e : c->ev) CK(cuda_rc(cudaEventCreate(&e), "cudaEventCreate"));
    }
    *out = c;
    return GMRES_OK;
}

}  // namespace gm

extern "C" {


}  // extern "C"

template <typename T>
static int run_cycle(gmres_ctx* c, const CycleBasis& cb, std::vector<std::pair<int, int>>* marks, cudaStream_t s) {
    const gmres_opts& o = c->opts;
    DevState* ds = c->st;
    int32_t* done = &ds->done;
    T* basis = static_cast<T*>(c->basis);
    PipWork w{};
    int evi = 0;
    auto mark = [&](int phase) -> cudaError_t {
        if (!marks) return cudaSuccess;
        marks->push_back({phase, evi});
        return cudaEventRecord(c->ev[evi++], s);
    };
    const int nblk = o.m / cb.s;
    int panel_idx = 0;
    const bool shifted = o.shift != GMRES_SHIFT_NONE;
    const int s1mode = shifted ? kPipShift : 0;   // stage 1: shifted Cholesky (§II)
    cudaError_t e = launch_cycle_begin(s, ds, cb);
    if (e == cudaSuccess) e = launch_scale(s, c->n, c->r ? c->r : static_cast<double*>(c->basis), basis, ds);
    const int capc = o.m + 1;
    void* dig = (sizeof(T) == sizeof(double)) ? c->digits : nullptr;   // the digit basis (tensor-core arithmetic)
    if (e == cudaSuccess && dig)
        e = launch_digits_fill_cols(s, c->n, reinterpret_cast<const double*>(basis), c->ldq, 0, 1, dig, capc);
    for (int j = 0; j < nblk && e == cudaSuccess; ++j) {
        const int st0 = j * cb.s;
        e = mark(PH_MPK);
        for (int i = 0; i < cb.s && e == cudaSuccess; ++i) {
            const double th = cb.theta[i];
            double sig_i, nu_i;
            cheb_coeffs(cb.cheb, i, cb.sigma, &sig_i, &nu_i);
            const double sinv = 1.0 / sig_i;
            T* wi = basis + (size_t)(st0 + i) * c->ldq;
            T* zi = i > 0 ? basis + (size_t)(st0 + i - 1) * c->ldq : nullptr;   // Chebyshev: y_{i-1}
            if constexpr (std::is_same<T, double>::value) {
                if (c->gs.perm) {
                    // right preconditioning: w_{i+1} = (A M^{-1} w_i - theta w_i - nu w_{i-1}) / sigma_i,
                    // M^{-1} one multicolor Gauss-Seidel sweep (§VIII, Fig. 9)
                    e = launch_gs_sweep(s, c->A, c->gs, wi, c->gs.z, done);
                    if (e == cudaSuccess)
                        e = launch_spmv(s, c->A, c->gs.z, basis + (size_t)(st0 + i + 1) * c->ldq, th, sinv, done, wi,
                                        zi, nu_i);
                    continue;
                }
                e = launch_spmv(s, c->A, wi, basis + (size_t)(st0 + i + 1) * c->ldq, th, sinv, done, nullptr, zi,
                                nu_i);
            } else {
                e = launch_spmv(s, c->A, wi, basis + (size_t)(st0 + i + 1) * c->ldq, th, sinv, done, zi, nu_i);
            }
        }
        if (e == cudaSuccess) e = mark(PH_MPK);
        if (e == cudaSuccess) e = mark(PH_S1);
        if (e == cudaSuccess) {
            const int k = st0 + 1;
            w = pip_work_layout(c->pip_work, c->n, k, cb.s);
            T* V = basis + (size_t)k * c->ldq;
            double* R = ds->Rhat + (size_t)k * kMaxCols;
            int32_t* stat = &ds->blkstat[j];
            if (o.ortho == GMRES_ORTHO_BCGS2_CHOLQR2) {
                // BCGS2-CholQR2 (§IV-B, Fig. 2b): BCGS, CholQR2, BCGS, CholQR, five
                // reductions; the factors go to scratch blocks, their product to R
                const int grid = reduction_grid(c->n);
                const size_t SB = (size_t)kMaxCols * kMaxCols;
                double* S = c->bscr;
                PipWork w0 = pip_work_layout(c->pip_work, c->n, 0, cb.s);
                struct Step { int kk; double* R; int gmode; int umode; };
                const Step steps[5] = {{k, S, kPipGramOnly, kPipNoTrsm},     // P1, V <- V - Q P1
                                       {0, S + SB, 0, 0},                    // T1a, V <- V T1a^{-1}
                                       {0, S + 2 * SB, 0, 0},                // T1b, V <- V T1b^{-1}
                                       {k, S + 3 * SB, kPipGramOnly, kPipNoTrsm},   // P2
                                       {0, S + 4 * SB, 0, 0}};               // T2
                for (int q = 0; q < 5 && e == cudaSuccess; ++q) {
                    const Step& st_ = steps[q];
                    const PipWork& wq = st_.kk ? w : w0;
                    if (dig && st_.kk) {
                        // the projections on the tensor cores read the accumulated
                        // columns' digits from the digit basis
                        const double* Bd = reinterpret_cast<const double*>(basis);
                        double* Vd = reinterpret_cast<double*>(V);
                        e = launch_gram_tc_digits(s, c->n, Bd, c->ldq, k, Vd, c->ldq, cb.s, st_.R, kMaxCols, wq, stat,
                                                  grid, dig, capc, k, done, st_.gmode);
                        if (e == cudaSuccess)
                            e = launch_update_tc_digits(s, c->n, Bd, c->ldq, k, Vd, c->ldq, cb.s, st_.R, kMaxCols,
                                                        stat, dig, capc, done, st_.umode);
                        continue;
                    }
                    e = launch_pip_gram_chol(s, c->n, basis, c->ldq, st_.kk, V, c->ldq, cb.s, st_.R, kMaxCols, wq, stat,
                                             done, grid, st_.gmode, o.arith);
                    if (e == cudaSuccess)
                        e = launch_pip_update(s, c->n, basis, c->ldq, st_.kk, V, c->ldq, cb.s, st_.R, kMaxCols, stat,
                                              done, st_.umode, o.arith);
                }
                // the block's final columns into the digit basis for the blocks after it
                if (e == cudaSuccess && dig && st0 + cb.s < o.m)
                    e = launch_digits_fill_cols(s, c->n, reinterpret_cast<const double*>(V), c->ldq, k, cb.s, dig,
                                                capc);
                if (e == cudaSuccess) e = launch_bcgs2_combine(s, ds, k, cb.s, S, R);
            } else if (sizeof(T) == sizeof(double) && dig) {
                // BCGS-PIP (Fig. 4a) on the tensor cores, the accumulated columns'
                // digits read from the digit basis, the block's written back
                const double* Bd = reinterpret_cast<const double*>(basis);
                e = launch_gram_tc_digits(s, c->n, Bd, c->ldq, k, reinterpret_cast<const double*>(V), c->ldq, cb.s, R,
                                          kMaxCols, w, stat, reduction_grid(c->n), dig, capc, k, done, s1mode);
                if (e == cudaSuccess)
                    e = launch_update_tc_digits(s, c->n, Bd, c->ldq, k, reinterpret_cast<double*>(V), c->ldq, cb.s, R,
                                                kMaxCols, stat, dig, capc, done);
            } else if (sizeof(T) == sizeof(double)) {
                // BCGS-PIP (Fig. 4a): one reduction, Pythagorean Gram
                e = launch_pip_gram_chol(s, c->n, basis, c->ldq, k, V, c->ldq, cb.s, R, kMaxCols, w, stat, done,
                                         reduction_grid(c->n), s1mode, o.arith);
                if (e == cudaSuccess)
                    e = launch_pip_update(s, c->n, basis, c->ldq, k, V, c->ldq, cb.s, R, kMaxCols, stat, done, 0,
                                          o.arith);
            } else {
                // FP32 basis: project, then CholQR of the projected block with an
                // explicit FP64 Gram (the Pythagorean identity needs an
                // orthonormal stored basis, which FP32 storage is only to ~1e-7)
                e = launch_pip_gram_chol(s, c->n, basis, c->ldq, k, V, c->ldq, cb.s, R, kMaxCols, w, stat, done,
                                         reduction_grid(c->n), kPipGramOnly, o.arith);
                if (e == cudaSuccess)
                    e = launch_pip_update(s, c->n, basis, c->ldq, k, V, c->ldq, cb.s, R, kMaxCols, stat, done,
                                          kPipNoTrsm, o.arith);
                if (e == cudaSuccess) {
                    PipWork w0 = pip_work_layout(c->pip_work, c->n, 0, cb.s);
                    e = launch_pip_gram_chol(s, c->n, basis, c->ldq, 0, V, c->ldq, cb.s, R + k, kMaxCols, w0, stat,
                                             done, reduction_grid(c->n), 0, o.arith);
                }
                if (e == cudaSuccess)
                    e = launch_pip_update(s, c->n, basis, c->ldq, 0, V, c->ldq, cb.s, R + k, kMaxCols, stat, done, 0,
                                          o.arith);
            }
        }
        if (e == cudaSuccess) e = mark(PH_S1);
        const int t = st0 + cb.s;
        if (e == cudaSuccess && panel_end(t, cb.panel, o.m)) {
            const int lo = panel_start(t, cb.panel);
            const int np = t - lo + 1;
            e = mark(PH_S2);
            w = pip_work_layout(c->pip_work, c->n, lo, np);
            T* V = basis + (size_t)lo * c->ldq;
            double* R = ds->Cm + (size_t)lo * kMaxCols;
            int32_t* stat = &ds->blkstat[nblk + panel_idx];
            if (o.ortho == GMRES_ORTHO_BCGS2_CHOLQR2) {
                // the block is final after its five reductions: identity stage-2 factor
                if (e == cudaSuccess) e = launch_eye_panel(s, ds, lo, t);
            } else if (shifted) {
                // shifted CholQR3 of the big panel (§II): a shifted BCGS-PIP into Cm,
                // then two plain ones into scratch, and the product of the factors.
                // The passes read the basis itself; the final panel's digits are
                // refilled for the blocks after it
                const size_t SB = (size_t)kMaxCols * kMaxCols;
                double* Rq[3] = {R, c->bscr + lo * kMaxCols, c->bscr + SB + lo * kMaxCols};
                for (int q = 0; q < 3 && e == cudaSuccess; ++q) {
                    e = launch_pip_gram_chol(s, c->n, basis, c->ldq, lo, V, c->ldq, np, Rq[q], kMaxCols, w, stat, done,
                                             reduction_grid(c->n), q == 0 ? kPipShift : 0, o.arith);
                    if (e == cudaSuccess)
                        e = launch_pip_update(s, c->n, basis, c->ldq, lo, V, c->ldq, np, Rq[q], kMaxCols, stat, done, 0,
                                              o.arith);
                }
                if (e == cudaSuccess) e = launch_pip3_combine(s, ds, lo, t, c->bscr);
                if (e == cudaSuccess && dig && t < o.m)
                    e = launch_digits_fill_cols(s, c->n, reinterpret_cast<const double*>(V), c->ldq, lo, np, dig, capc);
            } else if (dig) {
                // every column 0 .. t is in the digit basis; the panel's final
                // columns are written back for the panels and blocks after it
                const double* Bd = reinterpret_cast<const double*>(basis);
                if (e == cudaSuccess)
                    e = launch_gram_tc_digits(s, c->n, Bd, c->ldq, lo, reinterpret_cast<const double*>(V), c->ldq, np,
                                              R, kMaxCols, w, stat, reduction_grid(c->n), dig, capc, lo + np, done);
                // the cycle's last panel: no later block reads its digits
                if (e == cudaSuccess)
                    e = t < o.m ? launch_update_tc_digits(s, c->n, Bd, c->ldq, lo, reinterpret_cast<double*>(V),
                                                          c->ldq, np, R, kMaxCols, stat, dig, capc, done)
                                : launch_pip_update(s, c->n, basis, c->ldq, lo, V, c->ldq, np, R, kMaxCols, stat, done,
                                                    0, o.arith);
            } else {
                if (e == cudaSuccess)
                    e = launch_pip_gram_chol(s, c->n, basis, c->ldq, lo, V, c->ldq, np, R, kMaxCols, w, stat, done,
                                             reduction_grid(c->n), 0, o.arith);
                if (e == cudaSuccess)
                    e = launch_pip_update(s, c->n, basis, c->ldq, lo, V, c->ldq, np, R, kMaxCols, stat, done, 0,
                                          o.arith);
            }
            if (e == cudaSuccess) e = mark(PH_S2);
            if (e == cudaSuccess) e = mark(PH_LS);
            if (e == cudaSuccess) e = launch_hessenberg_ls(s, ds, lo, t);
            if (e == cudaSuccess) e = mark(PH_LS);
            ++panel_idx;
        }
    }
    if (e == cudaSuccess) {
        if (c->gs.perm) {
            // x += M^{-1} (Q y)
            e = launch_xupdate(s, c->n, basis, c->ldq, c->gs.t, ds, true);
            if (e == cudaSuccess) e = launch_gs_sweep(s, c->A, c->gs, c->gs.t, c->gs.z, nullptr);
            if (e == cudaSuccess) e = launch_axpy1(s, c->n, c->gs.z, c->x, ds);
        } else {
            e = launch_xupdate(s, c->n, basis, c->ldq, c->x, ds);
        }
    }
    return cuda_rc(e, "cycle launch");
}

extern "C" {

}  // extern "C"

namespace gm {

// ---------------------------------------------------------------- step-wise solve
// gmres_solve is begin, then {enqueue_check, synchronize, decide, enqueue_cycle}
// until decide says stop, then finish.  The serving loop drives the same steps
// for many contexts on their own streams.

cudaStream_t run_stream(const SolveRun* R) { return R->c->stream; }

int run_begin(gmres_ctx* c, SolveRun* R, const double* b, const double* x, int on_device) {
    *R = SolveRun{};
    R->c = c;
    R->r.breakdown_block = -1;
    R->status = GMRES_WARN_MAXIT;
    R->on_device = on_device;
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_rc(cudaGetLastError(), "cudaSetDevice");
    cudaStream_t s = c->stream;
    const gmres_opts& o = c->opts;
    R->cb = R->ran = first_cycle_basis(o, c->sigma);
    R->auto_pending = o.basis == GMRES_BASIS_NEWTON_AUTO || o.basis == GMRES_BASIS_CHEBYSHEV_AUTO;
    R->r.sigma = R->cb.sigma;
    for (int i = 0; i < 16; ++i) R->r.theta[i] = R->cb.theta[i];
    const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t vb = c->n * sizeof(double);
    if (o.timing) {
        cudaEventCreate(&R->t0);
        cudaEventCreate(&R->t1);
        cudaEventRecord(R->t0, s);
    }
    int rc = cuda_rc(cudaMemcpyAsync(c->b, b, vb, kin, s), "copy b");
    if (!rc) rc = cuda_rc(cudaMemcpyAsync(c->x, x, vb, kin, s), "copy x");
    if (!rc) rc = cuda_rc(launch_residual(s, c->A, c->b, nullptr, nullptr, c->red_partial, c->red_counter, c->st, 1),
                          "norm b");
    if (!rc) rc = cuda_rc(cudaMemcpyAsync(c->hst, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, s), "state read");
    if (!rc) rc = cuda_rc(cudaStreamSynchronize(s), "sync");
    if (rc) return rc;
    R->bnorm = c->hst->bnorm;
    if (!std::isfinite(R->bnorm)) {
        set_error("b has non-finite entries");
        R->status = GMRES_ERR_NAN;
        R->finished = true;
        return GMRES_OK;
    }
    if (R->bnorm == 0.0) {
        // the solution of A x = 0 is x = 0
        rc = cuda_rc(cudaMemsetAsync(c->x, 0, vb, s), "zero x");
        R->status = GMRES_OK;
        R->finished = true;
        return rc;
    }
    double tol_abs = o.tol * R->bnorm;
    rc = cuda_rc(cudaMemcpyAsync(&c->st->tol_abs, &tol_abs, sizeof(double), cudaMemcpyHostToDevice, s), "tol");
    int32_t zero = 0;
    if (!rc) rc = cuda_rc(cudaMemcpyAsync(&c->st->iters, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, s), "iters");
    if (!rc) rc = cuda_rc(cudaStreamSynchronize(s), "sync");   // tol_abs is a stack value
    return rc;
}

int run_enqueue_check(SolveRun* R) {
    gmres_ctx* c = R->c;
    cudaStream_t s = c->stream;
    double* rout = c->r ? c->r : static_cast<double*>(c->basis);
    int rc = cuda_rc(launch_residual(s, c->A, c->b, c->x, rout, c->red_partial, c->red_counter, c->st, 0), "residual");
    if (!rc) rc = cuda_rc(cudaMemcpyAsync(c->hst, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, s), "state read");
    return rc;
}

int run_decide(SolveRun* R) {
    gmres_ctx* c = R->c;
    const gmres_opts& o = c->opts;
    const DevState& h = *c->hst;
    gmres_result& r = R->r;
    const int cyc = R->cyc;
    if (cyc > 0 && o.timing) {
        // accumulate the previous cycle's phase times
        for (size_t i = 0; i + 1 < R->marks.size(); i += 2) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, c->ev[R->marks[i].second], c->ev[R->marks[i + 1].second]);
            double* dst = R->marks[i].first == PH_MPK ? &r.t_mpk_ms : R->marks[i].first == PH_S1 ? &r.t_stage1_ms
                        : R->marks[i].first == PH_S2 ? &r.t_stage2_ms : &r.t_ls_ms;
            *dst += ms;
        }
    }
    r.iters = h.iters;
    r.restarts = cyc;
    r.relres_true = h.beta / R->bnorm;
    if (cyc > 0) r.relres_implicit = h.resid / R->bnorm;
    const int nb1 = o.m / R->ran.s;
    const int nstat = nb1 + (o.m + R->ran.panel - 1) / R->ran.panel;
    for (int i = 0; i < nstat; ++i) {
        if (h.blkstat[i]) {
            r.breakdown_block = i;
            r.breakdown_pivot = h.blkstat[i];
            set_error("Cholesky breakdown in %s %d at pivot %d (restart cycle %d)",
                      i < nb1 ? "stage-1 block" : "stage-2 panel", i < nb1 ? i : i - nb1, h.blkstat[i], cyc - 1);
            R->status = GMRES_ERR_BREAKDOWN;
            return (R->finished = true), 1;
        }
    }
    if (!std::isfinite(h.beta)) {
        set_error("non-finite residual norm");
        R->status = GMRES_ERR_NAN;
        return (R->finished = true), 1;
    }
    if (cyc > 0 && R->auto_pending) {
        // the first cycle was standard GMRES: its k x k Hessenberg matrix gives
        // the Ritz values; from now on the Newton basis takes them as shifts, or
        // the Chebyshev basis the interval of their real parts
        CycleBasis& nb = R->cb;
        nb.s = o.s;
        nb.panel = o.ortho == GMRES_ORTHO_TWO_STAGE ? o.panel : o.s;
        for (int i = 0; i < 16; ++i) nb.theta[i] = 0.0;
        if (o.basis == GMRES_BASIS_CHEBYSHEV_AUTO) {
            // the Chebyshev basis on the interval of the Ritz values' real parts
            double cc = 0.0, dl = 1.0;
            const int rc = chebyshev_interval(h.H, kMaxCols, h.k_used, &cc, &dl);
            if (rc) {
                R->status = rc;
                return (R->finished = true), 1;
            }
            for (int i = 0; i < o.s; ++i) nb.theta[i] = cc;
            nb.sigma = 0.5 * dl;
            nb.cheb = 1;
        } else {
            const int rc = newton_shifts(h.H, kMaxCols, h.k_used, o.s, nb.theta);
            if (rc) {
                R->status = rc;
                return (R->finished = true), 1;
            }
            nb.sigma = o.sigma > 0.0 ? c->sigma : newton_sigma(nb.theta, o.s, c->sigma);
        }
        R->auto_pending = false;
        r.sigma = nb.sigma;
        for (int i = 0; i < 16; ++i) r.theta[i] = nb.theta[i];
    }
    if (h.beta <= o.tol * R->bnorm) { R->status = GMRES_OK; return (R->finished = true), 1; }
    if (cyc >= o.max_restarts) { R->status = GMRES_WARN_MAXIT; return (R->finished = true), 1; }
    return 0;
}

static bool same_basis(const CycleBasis& a, const CycleBasis& b) {
    return a.s == b.s && a.panel == b.panel && a.cheb == b.cheb &&
           std::memcmp(&a.sigma, &b.sigma, sizeof(double)) == 0 && std::memcmp(a.theta, b.theta, sizeof(a.theta)) == 0;
}

static int enqueue_eager(gmres_ctx* c, const CycleBasis& cb, std::vector<std::pair<int, int>>* marks,
                         cudaStream_t s) {
    return c->opts.precision == GMRES_PREC_MIXED ? run_cycle<float>(c, cb, marks, s)
                                                 : run_cycle<double>(c, cb, marks, s);
}

// One restart cycle: replayed from its CUDA graph when the context has run this
// basis before (a cycle is some 50 kernel launches, so small systems are bound
// by launch latency), else enqueued kernel by kernel.  Timed runs stay eager
// (their phase events sit between the kernels).
static int enqueue_cycle(gmres_ctx* c, const CycleBasis& cb, std::vector<std::pair<int, int>>* marks) {
    if (marks || c->no_graphs) return enqueue_eager(c, cb, marks, c->stream);
    gmres_ctx::CycleGraph* g = nullptr;
    for (auto& x : c->graphs)
        if (x.runs > 0 && same_basis(x.cb, cb)) g = &x;
    if (!g) {
        // a free slot, else the least recently used one
        g = &c->graphs[0];
        for (auto& x : c->graphs)
            if (x.runs == 0 || x.last < g->last) g = &x;
        if (g->exec) {
            cudaStreamSynchronize(c->stream);   // no replay of it is still running
            cudaGraphExecDestroy(g->exec);
        }
        *g = gmres_ctx::CycleGraph{};
        g->cb = cb;
    }
    g->last = ++c->graph_tick;
    if (!g->exec && g->runs > 0) {
        // second use of this basis: capture the cycle on the private stream
        cudaError_t e = c->cap ? cudaSuccess : cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
        cudaGraph_t graph = nullptr;
        if (e == cudaSuccess) e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const int rc = enqueue_eager(c, cb, nullptr, c->cap);
            const cudaError_t e2 = cudaStreamEndCapture(c->cap, &graph);
            e = rc ? cudaErrorUnknown : e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            // capture is not available here: stay eager for this context
            cudaGetLastError();
            clear_error();
            g->exec = nullptr;
            c->no_graphs = true;
            return enqueue_eager(c, cb, nullptr, c->stream);
        }
    }
    ++g->runs;
    if (g->exec) return cuda_rc(cudaGraphLaunch(g->exec, c->stream), "cycle graph launch");
    return enqueue_eager(c, cb, nullptr, c->stream);
}

int run_enqueue_cycle(SolveRun* R) {
    gmres_ctx* c = R->c;
    const gmres_opts& o = c->opts;
    R->marks.clear();
    R->ran = R->cb;
    const int rc = enqueue_cycle(c, R->cb, o.timing ? &R->marks : nullptr);
    if (o.precision == GMRES_PREC_MIXED) ++R->r.ir_steps;
    ++R->cyc;
    return rc;
}

int run_finish(SolveRun* R, double* x) {
    gmres_ctx* c = R->c;
    cudaStream_t s = c->stream;
    const cudaMemcpyKind kout = R->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    int rc = cuda_rc(cudaMemcpyAsync(x, c->x, c->n * sizeof(double), kout, s), "copy x");
    if (c->opts.timing && !rc) cudaEventRecord(R->t1, s);
    if (!rc) rc = cuda_rc(cudaStreamSynchronize(s), "sync");
    if (c->opts.timing) {
        float ms = 0.f;
        if (!rc) cudaEventElapsedTime(&ms, R->t0, R->t1);
        R->r.t_total_ms = ms;
        cudaEventDestroy(R->t0);
        cudaEventDestroy(R->t1);
        R->t0 = R->t1 = nullptr;
    }
    R->r.status = rc ? rc : R->status;
    return rc;
}

}  // namespace gm

extern "C" {

int gmres_solve(gmres_ctx* c, const double* b, double* x, int32_t ptr_on_device, gmres_result* res) {
    clear_error();
    GM_ARG(c != nullptr && b != nullptr && x != nullptr, "NULL argument");
    SolveRun R;
    int rc = run_begin(c, &R, b, x, ptr_on_device);
    while (!rc && !R.finished) {
        rc = run_enqueue_check(&R);
        if (!rc) rc = cuda_rc(cudaStreamSynchronize(c->stream), "sync");
        if (rc || run_decide(&R)) break;
        rc = run_enqueue_cycle(&R);
    }
    if (!rc) rc = run_finish(&R, x);
    R.r.status = rc ? rc : R.status;
    if (res) *res = R.r;
    return R.r.status;
}

size_t gmres_footprint(int64_t n, int64_t nnz, const gmres_opts* opts) {
    if (n <= 0 || nnz < 0) return 0;
    gmres_opts o;
    if (opts) o = *opts; else gmres_default_opts(&o);
    if (o.ortho != GMRES_ORTHO_TWO_STAGE) o.panel = o.s;
    if (check_opts(&o)) return 0;
    return ctx_bytes(n, nnz, o);
}

static int check_pip_args(int64_t n, const void* Q, int64_t ldq, int32_t k, const void* V, int64_t ldv,
                          int32_t nb, const double* R, int32_t ldr, void* d_work, size_t work_bytes,
                          const int32_t* d_status, int* code) {
    *code = GMRES_ERR_ARG;
    GM_ARG(n >= 1, "n must be >= 1");
    GM_ARG(k >= 0 && nb >= 1 && nb <= kMaxNB && k + nb <= kMaxKX, "need k >= 0, 1 <= nb <= 64, k + nb <= 256");
    GM_ARG(k == 0 || (Q != nullptr && ldq >= n), "Q must be non-NULL with ldq >= n when k > 0");
    GM_ARG(V != nullptr && ldv >= n, "V must be non-NULL with ldv >= n");
    GM_ARG(R != nullptr && ldr >= k + nb, "R must be non-NULL with ldr >= k + nb");
    GM_ARG(d_status != nullptr, "d_status is NULL");
    GM_ARG(d_work != nullptr, "d_work is NULL");
    GM_ARG((reinterpret_cast<uintptr_t>(V) & 15) == 0 && (k == 0 || (reinterpret_cast<uintptr_t>(Q) & 15) == 0),
           "Q and V must be 16-byte aligned");
    GM_ARG((reinterpret_cast<uintptr_t>(d_work) & 255) == 0, "d_work must be 256-byte aligned");
    if (work_bytes < ortho_workspace_bytes(n, k, nb)) {
        set_error("d_work holds %zu bytes, need %zu", work_bytes, ortho_workspace_bytes(n, k, nb));
        *code = GMRES_ERR_WORKSPACE;
        return *code;
    }
    *code = GMRES_OK;
    return GMRES_OK;
}

}  // extern "C"

template <typename T>
static int ortho_pip(void* stream, int64_t n, const T* Q, int64_t ldq, int32_t k, T* V, int64_t ldv,
                     int32_t nb, double* R, int32_t ldr, void* d_work, size_t work_bytes, int32_t* d_status) {
    clear_error();
    int code = GMRES_OK;
    if (check_pip_args(n, Q, ldq, k, V, ldv, nb, R, ldr, d_work, work_bytes, d_status, &code)) return code;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PipWork w = pip_work_layout(d_work, n, k, nb);
    cudaError_t e = cudaMemsetAsync(w.counter, 0, 256, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(int32_t), s);
    if (e == cudaSuccess)
        e = launch_pip_gram_chol(s, n, Q, ldq, k, V, ldv, nb, R, ldr, w, d_status, nullptr, reduction_grid(n));
    if (e == cudaSuccess) e = launch_pip_update(s, n, Q, ldq, k, V, ldv, nb, R, ldr, d_status, nullptr);
    return cuda_rc(e, "ortho launch");
}

extern "C" {

static int gram_chol_impl(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k, const double* V,
                    int64_t ldv, int32_t nb, double* R, int32_t ldr, void* d_work, size_t work_bytes,
                    int32_t* d_status, int arith) {
    clear_error();
    int code = GMRES_OK;
    if (check_pip_args(n, Q, ldq, k, V, ldv, nb, R, ldr, d_work, work_bytes, d_status, &code)) return code;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PipWork w = pip_work_layout(d_work, n, k, nb);
    cudaError_t e = cudaMemsetAsync(w.counter, 0, 256, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(int32_t), s);
    if (e == cudaSuccess)
        e = launch_pip_gram_chol(s, n, Q, ldq, k, V, ldv, nb, R, ldr, w, d_status, nullptr, reduction_grid(n), 0,
                                 arith);
    return cuda_rc(e, "gram launch");
}

int ortho_gram_chol(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k, const double* V,
                    int64_t ldv, int32_t nb, double* R, int32_t ldr, void* d_work, size_t work_bytes,
                    int32_t* d_status) {
    return gram_chol_impl(stream, n, Q, ldq, k, V, ldv, nb, R, ldr, d_work, work_bytes, d_status, kArithFP64);
}

int ortho_gram_chol_dd(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k, const double* V,
                       int64_t ldv, int32_t nb, double* R, int32_t ldr, void* d_work, size_t work_bytes,
                       int32_t* d_status) {
    return gram_chol_impl(stream, n, Q, ldq, k, V, ldv, nb, R, ldr, d_work, work_bytes, d_status, kArithDD);
}

int ortho_gram_chol_tc(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k, const double* V,
                       int64_t ldv, int32_t nb, double* R, int32_t ldr, void* d_work, size_t work_bytes,
                       int32_t* d_status) {
    return gram_chol_impl(stream, n, Q, ldq, k, V, ldv, nb, R, ldr, d_work, work_bytes, d_status, kArithTC);
}

static int update_impl(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k, double* V, int64_t ldv,
                 int32_t nb, const double* R, int32_t ldr, const int32_t* d_status, int arith) {
    clear_error();
    int code = GMRES_OK;
    // workspace is not used by the update: pass a dummy that satisfies the checks
    GM_ARG(n >= 1, "n must be >= 1");
    GM_ARG(k >= 0 && nb >= 1 && nb <= kMaxNB && k + nb <= kMaxKX, "need k >= 0, 1 <= nb <= 64, k + nb <= 256");
    GM_ARG(k == 0 || (Q != nullptr && ldq >= n), "Q must be non-NULL with ldq >= n when k > 0");
    GM_ARG(V != nullptr && ldv >= n, "V must be non-NULL with ldv >= n");
    GM_ARG(R != nullptr && ldr >= k + nb, "R must be non-NULL with ldr >= k + nb");
    GM_ARG(d_status != nullptr, "d_status is NULL");
    (void)code;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_pip_update(s, n, Q, ldq, k, V, ldv, nb, R, ldr, d_status, nullptr, 0, arith);
    return cuda_rc(e, "update launch");
}

int ortho_update(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k, double* V, int64_t ldv,
                 int32_t nb, const double* R, int32_t ldr, const int32_t* d_status) {
    return update_impl(stream, n, Q, ldq, k, V, ldv, nb, R, ldr, d_status, kArithFP64);
}

int ortho_update_dd(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k, double* V, int64_t ldv,
                    int32_t nb, const double* R, int32_t ldr, const int32_t* d_status) {
    return update_impl(stream, n, Q, ldq, k, V, ldv, nb, R, ldr, d_status, kArithDD);
}

int ortho_update_tc(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k, double* V, int64_t ldv,
                    int32_t nb, const double* R, int32_t ldr, const int32_t* d_status) {
    return update_impl(stream, n, Q, ldq, k, V, ldv, nb, R, ldr, d_status, kArithTC);
}

static bool col16(const double* p, int64_t ld) {
    return (reinterpret_cast<uintptr_t>(p) & 15) == 0 && (ld % 2) == 0;
}

size_t ortho_digits_bytes(int64_t n, int32_t capc) {
    if (n < 1 || capc < 1 || capc > kMaxNB) return 0;
    return tc_digits_bytes(n, capc);
}

int ortho_digits_fill(void* stream, int64_t n, const double* X, int64_t ldx, int32_t c0, int32_t nc,
                      void* d_digits, int32_t capc) {
    clear_error();
    GM_ARG(n >= 1 && nc >= 1 && c0 >= 0 && capc >= 1 && capc <= kMaxNB && c0 + nc <= capc,
           "need n >= 1, nc >= 1, 0 <= c0, c0 + nc <= capc <= 64");
    GM_ARG(X != nullptr && ldx >= n && col16(X, ldx), "X must be non-NULL, ldx >= n, columns 16-byte aligned");
    GM_ARG(d_digits != nullptr && (reinterpret_cast<uintptr_t>(d_digits) & 15) == 0,
           "d_digits must be non-NULL and 16-byte aligned");
    cudaError_t e = launch_digits_fill_cols(static_cast<cudaStream_t>(stream), n, X, ldx, c0, nc, d_digits, capc);
    return cuda_rc(e, "digits fill launch");
}

int ortho_gram_chol_tcd(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k, const double* V,
                        int64_t ldv, int32_t nb, double* R, int32_t ldr, void* d_work, size_t work_bytes,
                        int32_t* d_status, const void* d_digits, int32_t capc, int32_t kc) {
    clear_error();
    int code = GMRES_OK;
    if (check_pip_args(n, Q, ldq, k, V, ldv, nb, R, ldr, d_work, work_bytes, d_status, &code)) return code;
    GM_ARG(k + nb <= kMaxNB && k + nb <= capc && capc <= kMaxNB && kc >= 0 && kc <= k + nb,
           "need k + nb <= capc <= 64 and 0 <= kc <= k + nb");
    GM_ARG(col16(V, ldv) && (k == 0 || col16(Q, ldq)), "Q and V columns must start on 16-byte boundaries");
    GM_ARG(d_digits != nullptr && (reinterpret_cast<uintptr_t>(d_digits) & 15) == 0,
           "d_digits must be non-NULL and 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PipWork w = pip_work_layout(d_work, n, k, nb);
    cudaError_t e = cudaMemsetAsync(w.counter, 0, 256, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(int32_t), s);
    if (e == cudaSuccess)
        e = launch_gram_tc_digits(s, n, Q, ldq, k, V, ldv, nb, R, ldr, w, d_status, reduction_grid(n), d_digits, capc,
                                  kc);
    return cuda_rc(e, "gram launch");
}

int ortho_update_tcd(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k, double* V, int64_t ldv,
                     int32_t nb, const double* R, int32_t ldr, const int32_t* d_status, void* d_digits,
                     int32_t capc) {
    clear_error();
    GM_ARG(n >= 1, "n must be >= 1");
    GM_ARG(k >= 0 && nb >= 1 && k + nb <= kMaxNB && k + nb <= capc && capc <= kMaxNB,
           "need k >= 0, nb >= 1, k + nb <= capc <= 64");
    GM_ARG(k == 0 || (Q != nullptr && ldq >= n), "Q must be non-NULL with ldq >= n when k > 0");
    GM_ARG(V != nullptr && ldv >= n, "V must be non-NULL with ldv >= n");
    GM_ARG(R != nullptr && ldr >= k + nb, "R must be non-NULL with ldr >= k + nb");
    GM_ARG(d_status != nullptr, "d_status is NULL");
    GM_ARG(col16(V, ldv) && (k == 0 || col16(Q, ldq)), "Q and V columns must start on 16-byte boundaries");
    GM_ARG(d_digits != nullptr && (reinterpret_cast<uintptr_t>(d_digits) & 15) == 0,
           "d_digits must be non-NULL and 16-byte aligned");
    cudaError_t e = launch_update_tc_digits(static_cast<cudaStream_t>(stream), n, Q, ldq, k, V, ldv, nb, R, ldr,
                                            d_status, d_digits, capc);
    return cuda_rc(e, "update launch");
}

int ortho_stage1(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k, double* V, int64_t ldv,
                 int32_t nb, double* R, int32_t ldr, void* d_work, size_t work_bytes, int32_t* d_status) {
    return ortho_pip(stream, n, Q, ldq, k, V, ldv, nb, R, ldr, d_work, work_bytes, d_status);
}

int ortho_stage2(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k, double* V, int64_t ldv,
                 int32_t nb, double* R, int32_t ldr, void* d_work, size_t work_bytes, int32_t* d_status) {
    return ortho_pip(stream, n, Q, ldq, k, V, ldv, nb, R, ldr, d_work, work_bytes, d_status);
}

int ortho_stage1_shifted(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k, double* V,
                         int64_t ldv, int32_t nb, double* R, int32_t ldr, void* d_work, size_t work_bytes,
                         int32_t* d_status) {
    clear_error();
    int code = GMRES_OK;
    if (check_pip_args(n, Q, ldq, k, V, ldv, nb, R, ldr, d_work, work_bytes, d_status, &code)) return code;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    PipWork w = pip_work_layout(d_work, n, k, nb);
    cudaError_t e = cudaMemsetAsync(w.counter, 0, 256, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(int32_t), s);
    if (e == cudaSuccess)
        e = launch_pip_gram_chol(s, n, Q, ldq, k, V, ldv, nb, R, ldr, w, d_status, nullptr, reduction_grid(n),
                                 kPipShift, kArithFP64);
    if (e == cudaSuccess) e = launch_pip_update(s, n, Q, ldq, k, V, ldv, nb, R, ldr, d_status, nullptr);
    return cuda_rc(e, "ortho launch");
}

int ortho_stage1_f32(void* stream, int64_t n, const float* Q, int64_t ldq, int32_t k, float* V, int64_t ldv,
                     int32_t nb, double* R, int32_t ldr, void* d_work, size_t work_bytes, int32_t* d_status) {
    return ortho_pip(stream, n, Q, ldq, k, V, ldv, nb, R, ldr, d_work, work_bytes, d_status);
}

int ortho_stage2_f32(void* stream, int64_t n, const float* Q, int64_t ldq, int32_t k, float* V, int64_t ldv,
                     int32_t nb, double* R, int32_t ldr, void* d_work, size_t work_bytes, int32_t* d_status) {
    return ortho_pip(stream, n, Q, ldq, k, V, ldv, nb, R, ldr, d_work, work_bytes, d_status);
}

int gmres_precond_apply(gmres_ctx* c, const double* r, double* z) {
    clear_error();
    GM_ARG(c != nullptr && r != nullptr && z != nullptr && r != z, "need a context and distinct r, z");
    GM_ARG(c->gs.perm != nullptr, "the context has no preconditioner (opts.precond = GMRES_PRECOND_NONE)");
    cudaError_t e = cudaSetDevice(c->device);
    if (e == cudaSuccess) e = launch_gs_sweep(c->stream, c->A, c->gs, r, z, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_rc(e, "preconditioner launch");
}

int gmres_mpk(gmres_ctx* c, const double* v, double* W, int64_t ldw, int32_t s, double sigma, const double* theta) {
    clear_error();
    GM_ARG(c != nullptr && v != nullptr && W != nullptr, "NULL argument");
    GM_ARG(s >= 1 && s <= 16 && ldw >= c->n, "need 1 <= s <= 16 and ldw >= n");
    GM_ARG(sigma != 0.0 && std::isfinite(sigma), "sigma must be finite and nonzero");
    GM_ARG(c->opts.precision == GMRES_PREC_FP64, "gmres_mpk works on FP64 vectors: create the context with FP64");
    cudaError_t e = cudaSetDevice(c->device);
    const double sinv = 1.0 / sigma;
    const double* prev = v;
    for (int i = 0; i < s && e == cudaSuccess; ++i) {
        e = launch_spmv(c->stream, c->A, prev, W + (size_t)i * ldw, theta ? theta[i] : 0.0, sinv, nullptr);
        prev = W + (size_t)i * ldw;
    }
    return cuda_rc(e, "mpk launch");
}

}  // extern "C"
