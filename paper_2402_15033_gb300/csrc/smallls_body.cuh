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
#pragma once
#include "solver_state.cuh"

namespace gm {

constexpr int kLsLd = kMaxCols;

// Reset a cycle's scalars; `stand_down` = 1 keeps every kernel of the cycle idle.
__device__ inline void cycle_begin_body(DevState* st, int stand_down) {
    const int t = threadIdx.x;
    if (t == 0) {
        st->k_used = 0;
        st->done = stand_down;
        st->nrot = 0;
        st->resid = 0.0;
    }
    for (int i = t; i < 2 * kMaxCols; i += blockDim.x) st->blkstat[i] = 0;
}

// Hessenberg recovery and Givens update for the big panel [lo, t] (one CTA).
__device__ inline void hessenberg_ls_body(DevState* st, int lo, int t) {
    __shared__ double a[kLsLd];
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
            acc = (i < lo) ? Rhat[i + c * kLsLd] : 0.0;
            const int pe = c < t ? c : t;
            for (int p = lo; p <= pe; ++p) acc = fma(Cm[i + p * kLsLd], Rhat[p + c * kLsLd], acc);
        }
        Rfin[i + c * kLsLd] = acc;
    }
    __syncthreads();

    // 2. Hessenberg columns c_lo .. t-1 from H a_c = b_c
    const int c_lo = lo > 0 ? lo - 1 : 0;
    for (int c = c_lo; c < t; ++c) {
        const bool bstart = (c % s) == 0;
        const bool sfinal = bstart && c > 0 && (c % panel) == 0;
        for (int i = tid; i <= m; i += blockDim.x)
            a[i] = bstart ? (sfinal ? (i == c ? 1.0 : 0.0) : Cm[i + c * kLsLd]) : Rfin[i + c * kLsLd];
        __syncthreads();
        const double th = st->theta[c % s];
        const double inv_ac = 1.0 / a[c];
        for (int i = tid; i <= m; i += blockDim.x) {
            double acc = sigma * Rfin[i + (c + 1) * kLsLd];
            if (th != 0.0) acc = fma(th, a[i], acc);
            for (int p = 0; p < c; ++p) acc = fma(-H[i + p * kLsLd], a[p], acc);
            H[i + c * kLsLd] = acc * inv_ac;
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
            for (int i = 0; i <= c + 1; ++i) Rg[i + c * kLsLd] = H[i + c * kLsLd];
            for (int i = 0; i < c; ++i) {
                const double x0 = Rg[i + c * kLsLd], x1 = Rg[i + 1 + c * kLsLd];
                Rg[i + c * kLsLd] = st->cs[i] * x0 + st->sn[i] * x1;
                Rg[i + 1 + c * kLsLd] = -st->sn[i] * x0 + st->cs[i] * x1;
            }
            const double x0 = Rg[c + c * kLsLd], x1 = Rg[c + 1 + c * kLsLd];
            const double r = hypot(x0, x1);
            double cc = 1.0, ss = 0.0;
            if (r != 0.0) { cc = x0 / r; ss = x1 / r; }
            st->cs[c] = cc;
            st->sn[c] = ss;
            Rg[c + c * kLsLd] = r;
            Rg[c + 1 + c * kLsLd] = 0.0;
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
                for (int j = i + 1; j < t; ++j) acc -= Rg[i + j * kLsLd] * st->y[j];
                st->y[i] = acc / Rg[i + i * kLsLd];
            }
            st->k_used = t;
            st->done = 1;
        }
    }
}

// BCGS2-CholQR2 block factor (§IV-B, Fig. 2b with CholQR2): from the five
// reductions' factors in scratch blocks of leading dimension kLsLd
//   S0 = P1 (k x s: first projection), S1 = T1a, S2 = T1b (CholQR2 of the
//   projected block, T1 = T1b T1a), S3 = P2 (second projection), S4 = T2,
// write R = [P1 + P2 T1; T2 T1] into the block column R (rows 0 .. k+s-1).
__device__ inline void bcgs2_combine_body(const DevState* st, int k, int s, const double* S, double* R) {
    __shared__ double T1[16 * 16];
    if (st->done) return;
    const int tid = threadIdx.x;
    const double* P1 = S;
    const double* T1a = S + kLsLd * kLsLd;
    const double* T1b = S + 2 * kLsLd * kLsLd;
    const double* P2 = S + 3 * kLsLd * kLsLd;
    const double* T2 = S + 4 * kLsLd * kLsLd;
    for (int e = tid; e < s * s; e += blockDim.x) {          // T1 = T1b T1a (upper triangular)
        const int i = e % s, j = e / s;
        double acc = 0.0;
        for (int l = i; l <= j; ++l) acc = fma(T1b[i + l * kLsLd], T1a[l + j * kLsLd], acc);
        T1[i + j * 16] = i <= j ? acc : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < (k + s) * s; e += blockDim.x) {
        const int i = e % (k + s), j = e / (k + s);
        double acc;
        if (i < k) {
            acc = P1[i + j * kLsLd];
            for (int l = 0; l <= j; ++l) acc = fma(P2[i + l * kLsLd], T1[l + j * 16], acc);
        } else {
            const int ii = i - k;
            acc = 0.0;
            for (int l = ii; l <= j; ++l) acc = fma(T2[ii + l * kLsLd], T1[l + j * 16], acc);
        }
        R[i + j * kLsLd] = acc;
    }
}

// Stage-2 factor of a one-stage scheme whose blocks come out final: the
// identity on the panel's columns [lo, t] (no projection part).
__device__ inline void eye_panel_body(DevState* st, int lo, int t) {
    if (st->done) return;
    for (int e = threadIdx.x; e < (t + 1) * (t - lo + 1); e += blockDim.x) {
        const int i = e % (t + 1), c = lo + e / (t + 1);
        st->Cm[i + c * kLsLd] = i == c ? 1.0 : 0.0;
    }
}

}  // namespace gm
