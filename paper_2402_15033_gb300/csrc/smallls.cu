// Small dense steps of the s-step GMRES cycle, one CTA on the device:
// recovery of the upper Hessenberg matrix from the block-orthogonalization
// factors and its Givens least-squares update (the projected problem that the
// paper solves redundantly on the host, §VII).
//
// Change of basis.  SpMV number c (0-based) reads y_c and writes the raw MPK
// column c+1, A y_c = sigma w_{c+1} + theta_c y_c (§III, monomial basis of §VI
// scaled by a power of two).  After stage 2 of the big panel [lo, t] (§V):
//   Rfin[:, c] = E Rhat[:, c],  E = identity on columns < lo, Cm on [lo, t],
// where Rhat are the stage-1 factors (raw w = Q^ Rhat) and Cm the stage-2
// factors (Q^ = Q Cm).  In the orthonormal basis Q:
//   a_c = e_c         if c starts a block from an already final column,
//   a_c = Cm[:, c]    if c starts a block from a pre-processed column q^_c,
//   a_c = Rfin[:, c]  otherwise;     b_c = sigma Rfin[:, c+1] + theta_c a_c,
// and A Q_k = Q_{k+1} H with H = B A^{-1} (A upper triangular), obtained one
// column at a time from H a_c = b_c.  The right-hand side of the least-squares
// problem is ||r|| Cm[0,0] e_1 because q^_1 = r / ||r|| = Cm[0,0] q_1.
#include "solver_state.cuh"

namespace gm {

namespace {

constexpr int L = kMaxCols;

__global__ void cycle_begin_kernel(DevState* st) {
    const int t = threadIdx.x;
    if (t == 0) {
        st->k_used = 0;
        st->done = 0;
        st->nrot = 0;
        st->resid = 0.0;
    }
    for (int i = t; i < 2 * kMaxCols; i += blockDim.x) st->blkstat[i] = 0;
}

__global__ void __launch_bounds__(256) hessenberg_ls_kernel(DevState* st, int lo, int t) {
    __shared__ double a[L];
    if (st->done) return;   // a breakdown earlier in the cycle
    const int tid = threadIdx.x;
    const int m = st->m, s = st->s, panel = st->panel;
    const double sigma = st->sigma;
    const double* Rhat = st->Rhat;
    const double* Cm = st->Cm;
    double* Rfin = st->Rfin;
    double* H = st->H;

    // 1. final coordinates of the panel's raw columns
    const int ncol = t - lo + 1;
    for (int e = tid; e < ncol * (m + 1); e += blockDim.x) {
        const int c = lo + e / (m + 1), i = e % (m + 1);
        double acc;
        if (c == 0) {
            acc = Cm[i];
        } else {
            acc = (i < lo) ? Rhat[i + c * L] : 0.0;
            const int pe = c < t ? c : t;
            for (int p = lo; p <= pe; ++p) acc = fma(Cm[i + p * L], Rhat[p + c * L], acc);
        }
        Rfin[i + c * L] = acc;
    }
    __syncthreads();

    // 2. Hessenberg columns c_lo .. t-1 from H a_c = b_c
    const int c_lo = lo > 0 ? lo - 1 : 0;
    for (int c = c_lo; c < t; ++c) {
        const bool bstart = (c % s) == 0;
        const bool sfinal = bstart && c > 0 && (c % panel) == 0;
        for (int i = tid; i <= m; i += blockDim.x)
            a[i] = bstart ? (sfinal ? (i == c ? 1.0 : 0.0) : Cm[i + c * L]) : Rfin[i + c * L];
        __syncthreads();
        const double th = st->theta[c % s];
        const double inv_ac = 1.0 / a[c];
        for (int i = tid; i <= m; i += blockDim.x) {
            double acc = sigma * Rfin[i + (c + 1) * L];
            if (th != 0.0) acc = fma(th, a[i], acc);
            for (int p = 0; p < c; ++p) acc = fma(-H[i + p * L], a[p], acc);
            H[i + c * L] = acc * inv_ac;
        }
        __syncthreads();
    }

    // 3. Givens rotations of the new columns and the residual estimate
    if (tid == 0) {
        double* g = st->g;
        double* Rg = st->Rg;
        if (lo == 0) {
            g[0] = st->beta * Cm[0];
            for (int i = 1; i <= m; ++i) g[i] = 0.0;
        }
        for (int c = c_lo; c < t; ++c) {
            for (int i = 0; i <= c + 1; ++i) Rg[i + c * L] = H[i + c * L];
            for (int i = 0; i < c; ++i) {
                const double x0 = Rg[i + c * L], x1 = Rg[i + 1 + c * L];
                Rg[i + c * L] = st->cs[i] * x0 + st->sn[i] * x1;
                Rg[i + 1 + c * L] = -st->sn[i] * x0 + st->cs[i] * x1;
            }
            const double x0 = Rg[c + c * L], x1 = Rg[c + 1 + c * L];
            const double r = hypot(x0, x1);
            double cc = 1.0, ss = 0.0;
            if (r != 0.0) { cc = x0 / r; ss = x1 / r; }
            st->cs[c] = cc;
            st->sn[c] = ss;
            Rg[c + c * L] = r;
            Rg[c + 1 + c * L] = 0.0;
            const double gk = g[c];
            g[c] = cc * gk;
            g[c + 1] = -ss * gk;
        }
        st->nrot = t;
        const double res = fabs(g[t]);
        st->resid = res;
        if (res <= st->tol_abs || t == m) {
            for (int i = t - 1; i >= 0; --i) {
                double acc = g[i];
                for (int j = i + 1; j < t; ++j) acc -= Rg[i + j * L] * st->y[j];
                st->y[i] = acc / Rg[i + i * L];
            }
            st->k_used = t;
            st->done = 1;
        }
    }
}

}  // namespace

cudaError_t launch_cycle_begin(cudaStream_t st, DevState* ds) {
    cycle_begin_kernel<<<1, 64, 0, st>>>(ds);
    return cudaGetLastError();
}

cudaError_t launch_hessenberg_ls(cudaStream_t st, DevState* ds, int lo, int t) {
    hessenberg_ls_kernel<<<1, 256, 0, st>>>(ds, lo, t);
    return cudaGetLastError();
}

}  // namespace gm
