// Small dense steps of the s-step GMRES cycle, one CTA on the device:
// recovery of the upper Hessenberg matrix from the block-orthogonalization
// factors and its Givens least-squares update (the projected problem that the
// paper solves redundantly on the host, §VII).
//
// Change of basis.  SpMV number c (0-based) reads y_c and writes the raw MPK
// column c+1, A y_c = sigma w_{c+1} + theta_c y_c (§III, monomial basis of §VI
// scaled by a power of two); with the Chebyshev basis A y_c = sigma_c w_{c+1} +
// theta_c y_c + nu_c y_{c-1} (cheb_coeffs of c mod s; nu_c = 0 at a block's
// first column, so y_{c-1} is a column of the same block, and
// b_c = sigma_c Rfin[:, c+1] + theta_c a_c + nu_c a_{c-1}).  After stage 2 of
// the big panel [lo, t] (§V):
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
// Everything runs on shared copies (dynamic shared memory of
// hessenberg_ls_smem() bytes): the panel's blocks of Cm and Rhat, the final
// coordinates Rfin they give, H's columns (each row's previous entries feed its
// next one), the rotations, g, and, once the cycle ends, the rotated H for the
// back substitution; the results go back to the state.  The arithmetic and its
// order are those of the plain recurrences.
constexpr int kLsThreads = 512;
__host__ __device__ constexpr size_t hessenberg_ls_smem() { return (size_t)4 * kLsLd * kLsLd * sizeof(double); }

__device__ inline void hessenberg_ls_body(DevState* st, int lo, int t, double* dyn) {
    __shared__ double a2[2][kLsLd];             // a_c and a_{c-1} (alternating)
    __shared__ double sg[kLsLd + 1];
    __shared__ double scs[kLsLd], ssn[kLsLd];
    __shared__ double sy[kLsLd];
    __shared__ int s_done;
    __shared__ double s_inv;
    if (st->done) return;   // a breakdown earlier in the cycle
    const int tid = threadIdx.x, lane = tid & 31;
    const int m = st->m, s = st->s, panel = st->panel;
    const double sigma = st->sigma;
    const double* Rhat = st->Rhat;
    const double* Cm = st->Cm;
    double* Rfin = st->Rfin;
    double* H = st->H;
    double* Rg = st->Rg;
    const int c_lo = lo > 0 ? lo - 1 : 0;
    double* sH = dyn;                        // H columns, then their rotated form [i + c ld]
    double* sRf = dyn + kLsLd * kLsLd;       // Rfin columns c_lo .. t           [i + (c - c_lo) ld]
    double* sCm = dyn + 2 * kLsLd * kLsLd;   // Cm columns c_lo .. t             [i + (p - c_lo) ld]
    double* sRh = dyn + 3 * kLsLd * kLsLd;   // Rhat rows and columns lo .. t    [(p - lo) + (c - lo) ld]

    // 0. stage the panel's factors, the earlier H columns, rotations and g
    const int nc = t - c_lo + 1, ncol = t - lo + 1;
    for (int e = tid; e < (m + 1) * nc; e += blockDim.x) {
        const int i = e % (m + 1), p = c_lo + e / (m + 1);
        sCm[i + (p - c_lo) * kLsLd] = Cm[i + p * kLsLd];
        if (p < lo) sRf[i + (p - c_lo) * kLsLd] = Rfin[i + p * kLsLd];
    }
    for (int e = tid; e < ncol * ncol; e += blockDim.x) {
        const int p = lo + e % ncol, c = lo + e / ncol;
        sRh[(p - lo) + (c - lo) * kLsLd] = Rhat[p + c * kLsLd];
    }
    for (int e = tid; e < (m + 1) * c_lo; e += blockDim.x) {
        const int i = e % (m + 1), p = e / (m + 1);
        sH[i + p * kLsLd] = H[i + p * kLsLd];
    }
    for (int i = tid; i < c_lo; i += blockDim.x) {
        scs[i] = st->cs[i];
        ssn[i] = st->sn[i];
    }
    for (int i = tid; i <= m; i += blockDim.x) sg[i] = lo == 0 ? (i == 0 ? st->beta * Cm[0] : 0.0) : st->g[i];
    __syncthreads();

    // 1. final coordinates of the panel's raw columns
    for (int e = tid; e < ncol * (m + 1); e += blockDim.x) {
        const int c = lo + e / (m + 1), i = e % (m + 1);
        double acc;
        if (c == 0) {
            acc = sCm[i];
        } else {
            acc = (i < lo) ? Rhat[i + c * kLsLd] : 0.0;
            const int pe = c < t ? c : t;
            for (int p = lo; p <= pe; ++p)
                acc = fma(sCm[i + (p - c_lo) * kLsLd], sRh[(p - lo) + (c - lo) * kLsLd], acc);
        }
        sRf[i + (c - c_lo) * kLsLd] = acc;
        Rfin[i + c * kLsLd] = acc;
    }
    __syncthreads();

    // 2. Hessenberg columns c_lo .. t-1 from H a_c = b_c
    const int cheb = st->cheb;
    for (int c = c_lo; c < t; ++c) {
        const bool bstart = (c % s) == 0;
        const bool sfinal = bstart && c > 0 && (c % panel) == 0;
        double* a = a2[(c - c_lo) & 1];
        const double* ap = a2[(c - c_lo + 1) & 1];   // a_{c-1}, written in the previous pass
        for (int i = tid; i <= m; i += blockDim.x) {
            const double ai = bstart ? (sfinal ? (i == c ? 1.0 : 0.0) : sCm[i + (c - c_lo) * kLsLd])
                                     : sRf[i + (c - c_lo) * kLsLd];
            a[i] = ai;
            if (i == c) s_inv = 1.0 / ai;   // one FP64 division per column, not one per thread
        }
        __syncthreads();
        const double th = st->theta[c % s];
        double sig_c, nu_c;
        cheb_coeffs(cheb, c % s, sigma, &sig_c, &nu_c);
        const double inv_ac = s_inv;
        for (int i = tid; i <= m; i += blockDim.x) {
            double acc = sig_c * sRf[i + (c + 1 - c_lo) * kLsLd];
            if (th != 0.0) acc = fma(th, a[i], acc);
            if (nu_c != 0.0) acc = fma(nu_c, ap[i], acc);
            for (int p = 0; p < c; ++p) acc = fma(-sH[i + p * kLsLd], a[p], acc);
            sH[i + c * kLsLd] = acc * inv_ac;
        }
        __syncthreads();
    }
    for (int e = tid; e < (m + 1) * (t - c_lo); e += blockDim.x) {
        const int i = e % (m + 1), c = c_lo + e / (m + 1);
        H[i + c * kLsLd] = sH[i + c * kLsLd];
    }
    __syncthreads();

    // 3. Givens rotations of the new columns (in place) and the residual estimate.
    //    Column c takes rotations 0 .. c-1 in order, then defines rotation c; here
    //    rotation i is applied to every later new column at once (one thread per
    //    column), so each column sees the same operations in the same order.
    const int cfirst = c_lo;
    for (int i = 0; i < t; ++i) {
        if (i >= cfirst && tid == 0) {
            // rotation i from column i, which has all of rotations 0 .. i-1
            double* col = sH + i * kLsLd;
            const double x0 = col[i], x1 = col[i + 1];
            const double r = hypot(x0, x1);
            double cc = 1.0, ss = 0.0;
            if (r != 0.0) { cc = x0 / r; ss = x1 / r; }
            scs[i] = cc;
            ssn[i] = ss;
            col[i] = r;
            col[i + 1] = 0.0;
            const double gk = sg[i];
            sg[i] = cc * gk;
            sg[i + 1] = -ss * gk;
        }
        if (i >= cfirst) __syncthreads();
        // rotation i on the new columns after it
        for (int c = max(cfirst, i + 1) + tid; c < t; c += blockDim.x) {
            double* col = sH + c * kLsLd;
            const double x0 = col[i], x1 = col[i + 1];
            col[i] = scs[i] * x0 + ssn[i] * x1;
            col[i + 1] = -ssn[i] * x0 + scs[i] * x1;
        }
        __syncthreads();
    }
    if (tid == 0) {
        st->nrot = t;
        const double res = fabs(sg[t]);
        st->resid = res;
        s_done = (res <= st->tol_abs || t == m) ? 1 : 0;
    }
    __syncthreads();
    for (int c = c_lo + tid; c < t; c += blockDim.x) {
        st->cs[c] = scs[c];
        st->sn[c] = ssn[c];
    }
    for (int i = tid; i <= m; i += blockDim.x) st->g[i] = sg[i];
    for (int e = tid; e < (m + 1) * (t - c_lo); e += blockDim.x) {
        const int i = e % (m + 1), c = c_lo + e / (m + 1);
        if (i <= c + 1) Rg[i + c * kLsLd] = sH[i + c * kLsLd];
    }
    if (!s_done) return;

    // 4. the cycle ends here: y from R y = g (R the rotated H, upper triangular);
    //    the earlier panels' rotated columns come back from the state
    for (int e = tid; e < t * c_lo; e += blockDim.x) {
        const int i = e % t, p = e / t;
        if (i <= p) sH[i + p * kLsLd] = Rg[i + p * kLsLd];
    }
    __syncthreads();
    if (tid < 32) {
        for (int i = t - 1; i >= 0; --i) {
            double part = 0.0;
            for (int j = i + 1 + lane; j < t; j += 32) part = fma(sH[i + j * kLsLd], sy[j], part);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
            if (lane == 0) sy[i] = (sg[i] - part) / sH[i + i * kLsLd];
            __syncwarp();
        }
    }
    __syncthreads();
    for (int i = tid; i < t; i += blockDim.x) st->y[i] = sy[i];
    if (tid == 0) {
        st->k_used = t;
        st->done = 1;
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

// Stage-2 factor of a big panel orthogonalized by three passes (shifted
// CholQR3: a shifted BCGS-PIP, then two plain ones, against the finished
// columns 0 .. lo-1).  Pass a left [P_a; T_a] in Cm(:, lo..t); passes b and c
// left [P_b; T_b] and [P_c; T_c] in Sb and Sc (same layout, ld kLsLd: rows
// 0..lo-1 the projection, rows lo..t the triangular factor).  Since
// Q^ = Q_fin P_a + Q_a T_a, Q_a = Q_fin P_b + Q_b T_b, Q_b = Q_fin P_c + Q T_c:
//     Cm(:, lo..t) <- [P_a + P_b T_a + P_c T_b T_a; T_c T_b T_a].
// U = T_b T_a and P_ab = P_a + P_b T_a go through Su and Sp.
__device__ inline void pip3_combine_body(DevState* st, int lo, int t, const double* Sb, const double* Sc, double* Su,
                                         double* Sp) {
    if (st->done) return;
    const int np = t - lo + 1, tid = threadIdx.x;
    double* Cm = st->Cm;
    auto Ta = [&](int i, int j) { return Cm[(lo + i) + (size_t)(lo + j) * kLsLd]; };
    for (int e = tid; e < (lo + np) * np; e += blockDim.x) {
        const int i = e % (lo + np), j = e / (lo + np);
        double acc;
        if (i < lo) {           // P_ab = P_a + P_b T_a
            acc = Cm[i + (size_t)(lo + j) * kLsLd];
            for (int l = 0; l <= j; ++l) acc = fma(Sb[i + (size_t)(lo + l) * kLsLd], Ta(l, j), acc);
            Sp[i + (size_t)j * kLsLd] = acc;
        } else {                // U = T_b T_a (upper triangular)
            const int ii = i - lo;
            acc = 0.0;
            for (int l = ii; l <= j; ++l) acc = fma(Sb[(lo + ii) + (size_t)(lo + l) * kLsLd], Ta(l, j), acc);
            Su[ii + (size_t)j * kLsLd] = ii <= j ? acc : 0.0;
        }
    }
    __syncthreads();
    for (int e = tid; e < (lo + np) * np; e += blockDim.x) {
        const int i = e % (lo + np), j = e / (lo + np);
        double acc;
        if (i < lo) {           // P = P_ab + P_c U
            acc = Sp[i + (size_t)j * kLsLd];
            for (int l = 0; l <= j; ++l) acc = fma(Sc[i + (size_t)(lo + l) * kLsLd], Su[l + (size_t)j * kLsLd], acc);
        } else {                // T = T_c U
            const int ii = i - lo;
            acc = 0.0;
            for (int l = ii; l <= j; ++l)
                acc = fma(Sc[(lo + ii) + (size_t)(lo + l) * kLsLd], Su[l + (size_t)j * kLsLd], acc);
            if (ii > j) acc = 0.0;
        }
        Cm[i + (size_t)(lo + j) * kLsLd] = acc;
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
