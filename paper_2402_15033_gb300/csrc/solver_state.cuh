// Device-resident state of one restart cycle and the launchers of the solver's
// non-orthogonalization kernels.
#pragma once
#include <vector>
#include "common.cuh"

namespace gm {

constexpr int kMaxCols = 64;   // m + 1 <= 64: one big panel per restart fits one CTA tile

struct DevCSR {
    int64_t n = 0, nnz = 0;
    int32_t* rowptr = nullptr;
    int32_t* colind = nullptr;
    double* vals = nullptr;
    float* vals32 = nullptr;   // FP32 copy for the mixed-precision MPK (else null)
};

// Multicolor Gauss-Seidel preconditioner: the rows sorted by color (perm,
// device; color c is perm[off[c] .. off[c+1]-1], host offsets), the diagonal
// (device), and two work vectors of n (device).
struct McGs {
    int32_t* perm = nullptr;
    std::vector<int64_t> off;
    double* diag = nullptr;
    double* z = nullptr;
    double* t = nullptr;
};

// One restart cycle's scalars and small matrices (all FP64, column-major,
// leading dimension kMaxCols).  Lives in device memory; the host reads it
// once per cycle.
struct DevState {
    double beta;          // ||r|| at the start of the cycle
    double inv_beta;
    double bnorm;         // ||b||
    double tol_abs;       // tol * ||b||
    double resid;         // |g_k| after the latest least-squares update
    double sigma;         // MPK scale
    double theta[16];     // MPK shifts (zero for the monomial basis)
    int32_t cheb;         // 1: Chebyshev basis (three-term MPK recurrence, cheb_coeffs)
    int32_t m, s, panel;
    int32_t k_used;       // iterations used by this cycle (0 until decided)
    int32_t done;         // 1: the rest of the cycle's kernels return at once
    int32_t iters;        // total iterations over all cycles
    int32_t nrot;         // Givens rotations applied so far in this cycle
    int32_t pad_;
    int32_t blkstat[2 * kMaxCols];  // Cholesky status per PIP call of the cycle (blocks, then panels)
    double y[kMaxCols];         // least-squares solution
    double g[kMaxCols + 1];     // rotated right-hand side
    double cs[kMaxCols], sn[kMaxCols];
    double Rhat[kMaxCols * kMaxCols];  // stage-1 factors  (V = Q^ Rhat)
    double Cm[kMaxCols * kMaxCols];    // stage-2 factors  (Q^ = Q Cm)
    double Rfin[kMaxCols * kMaxCols];  // Cm Rhat
    double H[kMaxCols * kMaxCols];     // upper Hessenberg, A Q_k = Q_{k+1} H
    double Rg[kMaxCols * kMaxCols];    // H after the Givens rotations
};

// Basis of one restart cycle: step size, panel, MPK scale and shifts.  The
// cycle-begin kernel writes it into DevState, so cycles of one solve may
// differ (GMRES_BASIS_NEWTON_AUTO runs its first cycle with s = 1).
struct CycleBasis {
    int32_t s = 1, panel = 1;
    double sigma = 1.0;
    double theta[16] = {};
    int32_t cheb = 0;
};

// Coefficients of product i (0-based within an s-step block) of the Chebyshev
// basis: A y_i = sig y_{i+1} + c y_i + nu y_{i-1}, with sigma = delta / 2 the
// first product has (2 sigma, 0) and the others (sigma, sigma) (the
// recurrence of T_i((z - c) / delta)); other bases have (sigma, 0).
__host__ __device__ inline void cheb_coeffs(int cheb, int i, double sigma, double* sig, double* nu) {
    *sig = (cheb && i == 0) ? 2.0 * sigma : sigma;
    *nu = (cheb && i != 0) ? sigma : 0.0;
}

// Newton-basis shifts and scale from a k x k Hessenberg matrix (newton.cu, host)
int newton_shifts(const double* H, int ldh, int k, int s, double* theta);
// Chebyshev interval [c - delta, c + delta] spanning the real parts of the
// eigenvalues of a k x k Hessenberg matrix (newton.cu, host)
int chebyshev_interval(const double* H, int ldh, int k, double* c, double* delta);
double newton_sigma(const double* theta, int s, double fallback);

int norm_grid(int64_t n);
cudaError_t launch_gs_sweep(cudaStream_t st, const DevCSR& A, const McGs& gs, const double* r, double* z,
                            const int32_t* d_skip);
cudaError_t launch_diag(cudaStream_t st, const DevCSR& A, double* diag, int32_t* bad);
cudaError_t launch_axpy1(cudaStream_t st, int64_t n, const double* z, double* x, const DevState* ds);
cudaError_t launch_spmv(cudaStream_t st, const DevCSR& A, const double* x, double* y, double theta,
                        double sinv, const int32_t* d_skip, const double* w = nullptr, const double* z = nullptr,
                        double nu = 0.0);
cudaError_t launch_spmv(cudaStream_t st, const DevCSR& A, const float* x, float* y, double theta,
                        double sinv, const int32_t* d_skip, const float* z = nullptr, double nu = 0.0);
cudaError_t launch_residual(cudaStream_t st, const DevCSR& A, const double* b, const double* x, double* out,
                            double* partial, unsigned* counter, DevState* ds, int which);
cudaError_t launch_scale(cudaStream_t st, int64_t n, const double* v, double* out, const DevState* ds);
cudaError_t launch_scale(cudaStream_t st, int64_t n, const double* v, float* out, const DevState* ds);
cudaError_t launch_xupdate(cudaStream_t st, int64_t n, const double* Q, int64_t ldq, double* x, DevState* ds,
                           bool assign = false);
cudaError_t launch_xupdate(cudaStream_t st, int64_t n, const float* Q, int64_t ldq, double* x, DevState* ds,
                           bool assign = false);
cudaError_t launch_narrow_vals(cudaStream_t st, int64_t m, const double* in, float* out);
cudaError_t launch_validate_csr(cudaStream_t st, int64_t n, int64_t nnz, const int32_t* rowptr,
                                const int32_t* colind, int32_t* bad);
cudaError_t launch_rowabs(cudaStream_t st, const DevCSR& A, unsigned long long* out);
cudaError_t launch_rowptr_narrow(cudaStream_t st, int64_t m, const int64_t* in, int32_t* out, int64_t nnz);
cudaError_t launch_cycle_begin(cudaStream_t st, DevState* ds, const CycleBasis& cb);
cudaError_t launch_hessenberg_ls(cudaStream_t st, DevState* ds, int lo, int t);
// BCGS2-CholQR2 block factor from the five reductions' factors (S: 5 blocks of kMaxCols^2)
cudaError_t launch_bcgs2_combine(cudaStream_t st, const DevState* ds, int k, int s, const double* S, double* R);
// identity stage-2 factor on the panel [lo, t] (one-stage schemes)
cudaError_t launch_eye_panel(cudaStream_t st, DevState* ds, int lo, int t);
// Stage-2 factor of a three-pass (shifted CholQR3) panel: S holds four
// kMaxCols^2 blocks (passes b and c, then two scratch blocks).
cudaError_t launch_pip3_combine(cudaStream_t st, DevState* ds, int lo, int t, const double* S);

}  // namespace gm
