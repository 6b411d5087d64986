/*
 * gmres.h -- C ABI of the GB300 s-step GMRES library with two-stage block
 * orthogonalization (Yamazaki, Higgins, Boman, Szyld, "Two-Stage Block
 * Orthogonalization to Improve Performance of s-step GMRES", arXiv 2402.15033).
 *
 * Conventions for every entry point
 *   - All functions are extern "C", never throw, never abort.  They return an
 *     int status: 0 = GMRES_OK, > 0 = warning, < 0 = error.  After an error
 *     gmres_last_error() returns a message for the calling host thread.
 *   - Dense blocks are column-major FP64 (or FP32 where named _f32) with a
 *     leading dimension ld >= n (elements).  Device pointers must be 16-byte
 *     aligned and ld a multiple of 2 (FP64) or 4 (FP32) so rows can be read
 *     with 128-bit loads.  Pointers are never retained after a call returns,
 *     except the CSR copy and workspace owned by a gmres_ctx.
 *   - "stream" is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Device-buffer calls are asynchronous on that stream and never
 *     allocate: their scratch space is the caller's d_work.
 *   - One GPU: the library uses the device current at gmres_create (or at the
 *     call, for the standalone ortho entry points).
 */
#ifndef GB300_SSTEP_GMRES_H
#define GB300_SSTEP_GMRES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define GMRES_OK              0
#define GMRES_WARN_MAXIT      1   /* not converged within max_restarts; x is valid        */
#define GMRES_ERR_ARG        -1   /* bad argument (sizes, alignment, options)             */
#define GMRES_ERR_CUDA       -2   /* a CUDA runtime call failed                           */
#define GMRES_ERR_OOM        -3   /* device allocation failed                             */
#define GMRES_ERR_BREAKDOWN  -4   /* Cholesky of a Gram matrix hit a pivot <= 0 or NaN:   */
                                  /* the block violated the stability condition of Eq. (1)/(5)/(9) */
#define GMRES_ERR_NAN        -5   /* non-finite residual                                   */
#define GMRES_ERR_TIMEOUT    -6   /* a bounded device wait ran out                         */
#define GMRES_ERR_WORKSPACE  -7   /* d_work smaller than ortho_workspace_bytes()          */
#define GMRES_ERR_EIG        -8   /* the QR iteration for the Ritz values did not converge */

/* ---------------------------------------------------------------- options */
#define GMRES_ORTHO_TWO_STAGE      0  /* §V, Fig. 5: BCGS-PIP per block + BCGS-PIP per big panel   */
#define GMRES_ORTHO_BCGS_PIP2      1  /* §IV-C, Fig. 4b: the two-stage scheme with panel = s (§V)  */
#define GMRES_ORTHO_BCGS2_CHOLQR2  2  /* §IV-B, Fig. 2b with CholQR2 (the paper's baseline): per   */
                                      /* block BCGS, CholQR2, BCGS, CholQR = five reductions;      */
                                      /* panel = s.  Single-system solver and server only.         */
#define GMRES_PREC_FP64            0  /* everything FP64                                          */
#define GMRES_PREC_MIXED           1  /* FP32 basis + MPK, FP64 Gram/Cholesky/Hessenberg, FP64 IR */
#define GMRES_BASIS_MONOMIAL       0  /* §VI: monomial basis (scaled by a power of two)           */
#define GMRES_BASIS_NEWTON         1  /* shifted products (A - theta_i I) v, shifts in opts.theta  */
#define GMRES_BASIS_NEWTON_AUTO    2  /* Newton basis with shifts from the solve itself: the first  */
                                      /* restart cycle is standard GMRES (s = panel = 1: each      */
                                      /* vector orthogonalized twice, same kernels); the           */
                                      /* real parts of its Ritz values (eigenvalues of its k x k    */
                                      /* Hessenberg matrix) in Leja order give theta_0..theta_{s-1} */
                                      /* (gmres_newton_shifts) for every later cycle, whose MPK     */
                                      /* scale is the power of two nearest the shifts' capacity     */
                                      /* unless opts.sigma > 0.  Per solve: a context that solves   */
                                      /* again starts again from s = 1.  A breakdown in the first   */
                                      /* cycle is numbered in its own blocks (m stage-1 blocks of   */
                                      /* s = 1, then m panels).  Not in the batched engine.          */
#define GMRES_BASIS_CHEBYSHEV      3  /* Chebyshev basis (named with the Newton basis in §VI):       */
                                      /* per s-step block y_1 = (A - c I) y_0 / delta and          */
                                      /* y_{i+1} = 2 (A - c I) y_i / delta - y_{i-1}, i.e. the      */
                                      /* Chebyshev polynomials T_i((z - c) / delta) of the interval */
                                      /* [c - delta, c + delta]; c = opts.theta[0], delta =         */
                                      /* opts.theta[1] > 0 (opts.sigma is not used).  The change of */
                                      /* basis is tridiagonal.  Not in the batched engine.          */
#define GMRES_BASIS_CHEBYSHEV_AUTO 4  /* Chebyshev basis on the interval spanned by the real parts   */
                                      /* of the first cycle's Ritz values (first cycle as for      */
                                      /* GMRES_BASIS_NEWTON_AUTO).  The result reports c in        */
                                      /* theta[0..s-1] and delta / 2 in sigma.                       */
#define GMRES_ARITH_FP64           0  /* native FP64 pipe (default)                                 */
#define GMRES_ARITH_DD             1  /* opt-in: double-float (hi + lo FP32) on the FP32 pipe:      */
                                      /* error-free products, renormalized sums, ~2^-48 relative;   */
                                      /* FP64 in/out.  32x less precise than FP64, so the block      */
                                      /* Pythagorean step (Eq. 5) breaks down sooner on marginal     */
                                      /* blocks; values must keep |x y| and partial sums inside the  */
                                      /* FP32 exponent range (|x| in [2^-50, 2^50] for unit-scale n) */
#define GMRES_ARITH_TC             2  /* opt-in: Gram reductions on the f16 tensor cores by exact     */
                                      /* integer slicing (Ozaki et al.): seven 8-bit digits per      */
                                      /* value against a per-chunk column exponent, digit products    */
                                      /* summed exactly in FP32, combined in 64-bit integers; FP64    */
                                      /* in/out, error normwise at the level of FP64 dot products.     */
                                      /* Both the Gram and the block update; blocks with k + nb > 64   */
                                      /* and FP32 bases use the FP64 kernels.  Single-system solver    */
                                      /* and the ortho calls only (the batched engine rejects it).     */
                                      /* GMRES_ARITH_DD and _TC stage 16-byte column pieces: columns   */
                                      /* that do not start on a 16-byte boundary (odd ld for FP64)     */
                                      /* run the FP64 kernels instead.                                 */

#define GMRES_SHIFT_NONE           0  /* stage 1 factors G - P^T P as in Fig. 4a (default)              */
#define GMRES_SHIFT_CHOLQR3        1  /* opt-in: shifted CholQR (§II, Fukaya et al. 2020) for blocks     */
                                      /* beyond the u^(-1/2) condition of Eq. (1): stage 1 factors      */
                                      /* G - P^T P + sigma I, sigma = 11 (n s + s (s+1)) u ||V||_F^2,    */
                                      /* so it does not break down on numerically full-rank blocks but  */
                                      /* leaves them only well conditioned; stage 2 is then shifted     */
                                      /* CholQR3 of the big panel (a shifted pass, two plain passes).   */
                                      /* A numerically rank-deficient panel still breaks down.  FP64    */
                                      /* basis, two-stage or BCGS-PIP2 ortho, any arithmetic; not in the  */
                                      /* batched engine.  The paper has no measurement of it.           */

#define GMRES_PRECOND_NONE         0  /* no preconditioner (default)                                 */
#define GMRES_PRECOND_MCGS         1  /* multicolor Gauss-Seidel (§VIII, Fig. 9), from the right: the  */
                                      /* MPK applies A M^{-1} and the correction is x += M^{-1} Q y,    */
                                      /* M^{-1} one forward Gauss-Seidel sweep from zero over the rows  */
                                      /* grouped by a greedy distance-1 coloring of the symmetrized     */
                                      /* pattern in natural row order (red-black on the grid stencils),  */
                                      /* colors in increasing order.  The rows need nonzero diagonals.   */
                                      /* The MPK scale defaults to 1 (sigma = 0).  A M^{-1} has many     */
                                      /* eigenvalues at or near 1, so the monomial basis loses rank fast: */
                                      /* use it with GMRES_BASIS_NEWTON_AUTO.  FP64 basis; not in the    */
                                      /* batched engine; gmres_mpk stays unpreconditioned.              */

typedef struct gmres_opts {
    int32_t m;             /* restart length: m+1 basis vectors per cycle (Table 1)            */
    int32_t s;             /* step size of the first stage (Table 1), 1 <= s <= 16            */
    int32_t panel;         /* second step size s^ (Table 1): s | panel | m, panel + 1 <= 64   */
    int32_t max_restarts;  /* restart cycles before GMRES_WARN_MAXIT                           */
    double  tol;           /* stop when ||b - A x|| / ||b|| <= tol                             */
    double  sigma;         /* MPK scale; 0 = 2^floor(log2 ||A||_inf) (exact in binary FP)     */
    int32_t ortho;         /* GMRES_ORTHO_*                                                    */
    int32_t precision;     /* GMRES_PREC_*                                                     */
    int32_t basis;         /* GMRES_BASIS_*                                                    */
    int32_t timing;        /* 1 = record per-phase CUDA-event times into gmres_result          */
    double  theta[16];     /* Newton shifts theta_0..theta_{s-1} (basis = NEWTON)              */
    double  inner_tol;     /* mixed precision: relative tolerance of each inner FP32 solve     */
    int32_t max_ir;        /* mixed precision: maximum FP64 refinement steps                   */
    int32_t arith;         /* GMRES_ARITH_*: arithmetic of the Gram and block-update kernels   */
    int32_t shift;         /* GMRES_SHIFT_*: shifted CholQR in the two-stage scheme             */
    int32_t precond;       /* GMRES_PRECOND_*: right preconditioner applied inside the MPK     */
    int32_t reserved[4];
} gmres_opts;

typedef struct gmres_result {
    int32_t status;            /* same value gmres_solve returned                          */
    int32_t iters;             /* Krylov iterations (SpMVs inside restart cycles)          */
    int32_t restarts;          /* restart cycles run                                       */
    int32_t ir_steps;          /* mixed precision: FP64 refinement steps (one per restart  */
                               /* cycle: r = b - A x in FP64, A d = r solved with the FP32 */
                               /* basis, x += d in FP64), else 0                           */
    int32_t breakdown_block;   /* s-step block index of a GMRES_ERR_BREAKDOWN, else -1     */
    int32_t breakdown_pivot;   /* 1-based Cholesky pivot of that breakdown, else 0         */
    double  relres_implicit;   /* |g_{k+1}| / ||b|| of the last least-squares solve        */
    double  relres_true;       /* ||b - A x|| / ||b|| recomputed in FP64 at exit           */
    double  t_mpk_ms, t_stage1_ms, t_stage2_ms, t_ls_ms, t_total_ms;  /* opts.timing = 1  */
    double  sigma;             /* MPK scale of the last restart cycle                      */
    double  theta[16];         /* its MPK shifts theta_0..theta_{s-1} (0: monomial); with  */
                               /* GMRES_BASIS_NEWTON_AUTO the shifts the solve chose, which */
                               /* a later solve can pass as opts.theta (basis = NEWTON);    */
                               /* with a Chebyshev basis the center c in every entry and    */
                               /* delta / 2 in sigma                                         */
} gmres_result;

typedef struct gmres_ctx gmres_ctx;   /* opaque: device CSR copy, Krylov basis, workspace */

/* Fill *o with the defaults: m=60, s=5, panel=60, tol=1e-8, max_restarts=10000,
 * two-stage, FP64, monomial basis, sigma automatic. */
int gmres_default_opts(gmres_opts* o);

/* Create a solver for the n x n CSR matrix A (rowptr[n+1] int64, colind[nnz]
 * int32 0-based, vals[nnz] FP64), on host (ptr_on_device = 0) or device
 * (ptr_on_device = 1) memory.  The context copies A and allocates the basis
 * ((m+1) columns of n, padded), the R/H/Givens state and the reduction
 * workspace; the caller's arrays are not retained.  Errors: GMRES_ERR_ARG
 * (n <= 0, nnz >= 2^31, bad options, a column index outside [0, n)),
 * GMRES_ERR_OOM, GMRES_ERR_CUDA. */
int gmres_create(gmres_ctx** out, int64_t n, int64_t nnz, const int64_t* rowptr,
                 const int32_t* colind, const double* vals, int32_t ptr_on_device,
                 const gmres_opts* opts, void* stream);

/* Solve A x = b by restarted s-step GMRES (Fig. 1, §III) with the block
 * orthogonalization chosen in opts (§IV-C, §V).  b[n] and x[n] are FP64 on
 * host or device (ptr_on_device); x holds x0 on entry (a restart checkpoint)
 * and the solution on exit.  Synchronizes the context's stream before it
 * returns.  Convergence is tested once per big panel; the reported
 * relres_true is recomputed from x.  Returns GMRES_OK, GMRES_WARN_MAXIT,
 * GMRES_ERR_BREAKDOWN (res->breakdown_block/pivot set), GMRES_ERR_NAN or an
 * error; res may be NULL. */
int gmres_solve(gmres_ctx* c, const double* b, double* x, int32_t ptr_on_device, gmres_result* res);

/* Release everything the context owns.  NULL-safe. */
int gmres_destroy(gmres_ctx* c);

/* Message of the last error on this host thread ("" if none).  Static storage. */
const char* gmres_last_error(void);

/* ------------------------------------------------ standalone block orthogonalization
 * Both stages are one BCGS-PIP (§IV-C, Fig. 4a) on caller-owned device buffers:
 *   [P; G] = [Q, V]^T V                 (one tall-skinny reduction over n rows)
 *   T      = Chol(G - P^T P)            (block Pythagorean theorem; T upper, T_ii > 0)
 *   V     <- (V - Q P) T^{-1}           (fused block update and triangular solve)
 * Stage 1 (§V) orthogonalizes one new s-step block against the accumulated
 * basis [Q_{1:l-1}, Q^_{l:j-1}]; stage 2 (§V) re-orthogonalizes a whole big
 * panel Q^_{l:t} against the finished basis Q_{1:l-1} (k = 0 gives CholQR of
 * the panel).  The two entry points compute the same operation and differ in
 * the kernels they pick: stage 1 is tuned for nb <= 16 new columns, stage 2
 * for panels up to 64 columns.
 *
 *   n        rows (n >= 1)
 *   Q, ldq   k columns of the basis to project against (k >= 0; unread if 0)
 *   V, ldv   nb new columns, overwritten by Q^_j (stage 1) or Q_{l:t} (stage 2)
 *   R, ldr   output block column, (k+nb) x nb, column-major, ldr >= k+nb:
 *            rows 0..k-1 = P, rows k..k+nb-1 = T (zeros below its diagonal)
 *   d_work   device scratch of at least ortho_workspace_bytes(n, k, nb) bytes;
 *            contents on entry are ignored
 *   d_status device int32: set to 0, or to the 1-based index of the first bad
 *            Cholesky pivot (then V is left unchanged and R holds P and the
 *            partial factor)
 * Arithmetic: FP64 (GMRES_ARITH_FP64).  ortho_gram_chol_dd/ortho_update_dd
 * run the same two halves in double-float arithmetic (GMRES_ARITH_DD).
 * Limits: k + nb <= 256, nb <= 64.  Returns GMRES_ERR_ARG / _WORKSPACE /
 * _CUDA for bad calls (nothing launched); a breakdown is reported only through
 * d_status, because the call is asynchronous. */
size_t ortho_workspace_bytes(int64_t n, int32_t k, int32_t nb);

int ortho_stage1(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k,
                 double* V, int64_t ldv, int32_t nb, double* R, int32_t ldr,
                 void* d_work, size_t work_bytes, int32_t* d_status);

int ortho_stage2(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k,
                 double* V, int64_t ldv, int32_t nb, double* R, int32_t ldr,
                 void* d_work, size_t work_bytes, int32_t* d_status);

/* Stage 1 with the shifted Cholesky of shifted CholQR (§II; GMRES_SHIFT_CHOLQR3):
 * [P; G] = [Q, V]^T V, T = Chol(G - P^T P + sigma I) with
 * sigma = 11 (n nb + nb (nb + 1)) u trace(G), u = 2^-53, and
 * V <- (V - Q P) T^{-1}.  V = Q P + V_out T holds as for ortho_stage1, but the
 * output block is only well conditioned (V_out^T V_out = I - sigma T^-T T^-1 for
 * an orthonormal Q); it does not break down on numerically full-rank blocks.
 * Arguments, limits and errors as for ortho_stage1 (FP64 arithmetic). */
int ortho_stage1_shifted(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k,
                         double* V, int64_t ldv, int32_t nb, double* R, int32_t ldr,
                         void* d_work, size_t work_bytes, int32_t* d_status);

/* FP32-basis variants (the mixed-precision pattern): Q and V are FP32, every
 * product and sum is formed in FP64 (FP32 inputs widen exactly), R and the
 * Cholesky factor are FP64, and the updated block is rounded to FP32.  Same
 * arguments, limits and errors as ortho_stage1/ortho_stage2 otherwise (ld a
 * multiple of 4). */
int ortho_stage1_f32(void* stream, int64_t n, const float* Q, int64_t ldq, int32_t k,
                     float* V, int64_t ldv, int32_t nb, double* R, int32_t ldr,
                     void* d_work, size_t work_bytes, int32_t* d_status);

int ortho_stage2_f32(void* stream, int64_t n, const float* Q, int64_t ldq, int32_t k,
                     float* V, int64_t ldv, int32_t nb, double* R, int32_t ldr,
                     void* d_work, size_t work_bytes, int32_t* d_status);

/* Stage 1 for callers that cannot allocate device memory.  No counterpart in
 * the paper: it is ortho_stage1 without the d_work argument, for code that
 * runs inside another framework's memory arena (which owns all device memory
 * and forbids cudaMalloc), plug-ins whose host program exposes no allocator,
 * and latency-critical loops that cannot pay the device-wide synchronization
 * of cudaMalloc/cudaFree.  Its scratch is a 2.5 MiB array that the library
 * owns in device memory; every GPU that loads the library keeps it until the
 * process exits.  Limits: nb <= 16 and k + nb <= 64 (any n); larger blocks
 * get GMRES_ERR_ARG with a message.  It calls no allocator: no cudaMalloc,
 * cudaFree or allocating library routine.
 * Set-up: the first call on a device (with that device current) looks up the
 * array's device address once; make that first call before any stream
 * capture.  The address is kept for the life of the process: after
 * cudaDeviceReset (or anything else that tears down the device's primary
 * context) the array may live at another address, and this entry point must
 * not be called on that device again.  Every call shares the one array: calls
 * that may overlap on the GPU (different streams, or different host threads)
 * race and must be serialized by the caller.  Arguments otherwise as for
 * ortho_stage1. */
int ortho_stage1_noalloc(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k,
                         double* V, int64_t ldv, int32_t nb, double* R, int32_t ldr,
                         int32_t* d_status);

/* The two halves of one BCGS-PIP, for callers that schedule or time them
 * separately; ortho_stage1/ortho_stage2 are exactly ortho_gram_chol followed
 * by ortho_update on the same stream with the same arguments.
 *   ortho_gram_chol: [P; G] = [Q, V]^T V and T = Chol(G - P^T P) into R, the
 *                    status into d_status (V is only read).
 *   ortho_update:    V <- (V - Q P) T^{-1} with P, T read from R; does nothing
 *                    when *d_status != 0.  d_work is not used.
 * Arguments, limits and errors as for ortho_stage1. */
int ortho_gram_chol(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k,
                    const double* V, int64_t ldv, int32_t nb, double* R, int32_t ldr,
                    void* d_work, size_t work_bytes, int32_t* d_status);

int ortho_update(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k,
                 double* V, int64_t ldv, int32_t nb, const double* R, int32_t ldr,
                 const int32_t* d_status);

/* The same two halves with double-float arithmetic (GMRES_ARITH_DD): faster on
 * GB300, whose FP64 pipe is 1/64 of its FP32 pipe, at ~2^-48 relative accuracy. */
int ortho_gram_chol_dd(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k,
                       const double* V, int64_t ldv, int32_t nb, double* R, int32_t ldr,
                       void* d_work, size_t work_bytes, int32_t* d_status);

int ortho_update_dd(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k,
                    double* V, int64_t ldv, int32_t nb, const double* R, int32_t ldr,
                    const int32_t* d_status);

/* The same two halves on the f16 tensor cores by exact slicing
 * (GMRES_ARITH_TC), for k + nb <= 64 (larger blocks run the FP64 kernels).
 * The update forms W = [-P T^{-1}; T^{-1}] and computes [Q, V] W. */
int ortho_gram_chol_tc(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k,
                       const double* V, int64_t ldv, int32_t nb, double* R, int32_t ldr,
                       void* d_work, size_t work_bytes, int32_t* d_status);

int ortho_update_tc(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k,
                    double* V, int64_t ldv, int32_t nb, const double* R, int32_t ldr,
                    const int32_t* d_status);

/* Two-stage orthogonalization of one panel in one call, on host or device
 * buffers (§V, Fig. 5): X = [x_0, V_0, ..., V_{nblk-1}] (n x (1 + s nblk),
 * column-major, ld ldx; x_0 of unit norm, the first column of a restart cycle)
 * goes through stage 1 (one BCGS-PIP of every block V_j against the
 * 1 + s j accumulated columns) and stage 2 (one BCGS-PIP = CholQR of the whole
 * panel).  Outputs: Q (n x (1 + s nblk), ld ldq) with X = Q R2 Rhat on the
 * panel's columns; Rhat (stage-1 factors: block column j in rows
 * 0 .. s(j+1), columns 1+sj .. s(j+1); column 0 untouched) and R2 (stage 2),
 * each (1+s nblk)^2, ld ldr, or NULL.  The same kernels as the ortho_* calls:
 * arith GMRES_ARITH_TC uses the digit basis (ortho_*_tcd), GMRES_ARITH_FP64 the
 * FP64 pipe.
 *   ortho_plan_create: allocates the device basis, digit basis, workspace and
 *                      factors for n rows (n >= 64), 1 <= s <= 16, 1 + s nblk
 *                      <= 64, on the current device; kernels run on `stream`.
 *   ortho_plan_run:    ptr_on_device = 0: X, Q, Rhat, R2 in host memory (page-
 *                      locked memory lets the copies overlap the kernels: the
 *                      columns go in block by block while stage 1 runs, Q comes
 *                      back in row ranges while the stage-2 update runs);
 *                      = 1: device memory.  X may equal Q.  Allocates nothing;
 *                      returns when the outputs are written.  block_status (host,
 *                      nblk + 1 entries, or NULL) receives each stage's Cholesky
 *                      status; any breakdown returns GMRES_ERR_BREAKDOWN.
 *   ortho_plan_destroy: NULL-safe.
 * The paper has no such call; it is the library's end-to-end entry point for
 * the step that the orthogonalization benchmark times. */
typedef struct ortho_plan ortho_plan;
int ortho_plan_create(ortho_plan** out, int64_t n, int32_t s, int32_t nblk, int32_t arith, void* stream);
int ortho_plan_run(ortho_plan* p, const double* X, int64_t ldx, double* Q, int64_t ldq, double* Rhat, double* R2,
                   int32_t ldr, int32_t ptr_on_device, int32_t* block_status);
int ortho_plan_destroy(ortho_plan* p);

/* Digit basis: the seven digit slices that the tensor-core arithmetic makes of
 * every FP64 value (per 64-row chunk of a column), kept in device memory so that
 * a basis column is sliced once however many blocks later read it (stage 1
 * projects every block against all accumulated columns, §V).  No counterpart in
 * the paper.
 *   ortho_digits_bytes: size of a digit basis of capc columns for n rows
 *                       (7 digit bytes per value plus one int32 exponent per
 *                       64-row chunk and column); capc <= 64.
 *   ortho_digits_fill:  slice X(:, 0:nc) into digit columns c0 .. c0+nc-1.
 *   ortho_gram_chol_tcd: ortho_gram_chol_tc whose first kc columns of [Q, V]
 *                       (kc <= k + nb) are read from digit columns 0 .. kc-1,
 *                       which must hold exactly those columns' current values;
 *                       bit-identical to ortho_gram_chol_tc, except that with
 *                       kc = k and nb <= 8 a streaming kernel (each warp copies
 *                       the digit bytes of its own chunks) runs, and with
 *                       kc = k + nb, nb >= 9 and k + nb <= 64 a kernel that sums
 *                       each CTA's chunks exactly and rounds once runs; both
 *                       agree to rounding.
 *   ortho_update_tcd:   ortho_update_tc that also writes the digits of the new V
 *                       into digit columns k .. k+nb-1; for nb <= 8 it reads Q's
 *                       digits from digit columns 0 .. k-1 (which must hold Q)
 *                       instead of slicing Q's rows, so results agree with
 *                       ortho_update_tc to rounding (not bit for bit).
 * Q, V and X columns must start on 16-byte boundaries (ld even); k + nb <= 64;
 * k + nb <= capc.  The digit buffer (d_digits) is owned by the caller, 16-byte
 * aligned, and may not be shared by calls that overlap on the GPU. */
size_t ortho_digits_bytes(int64_t n, int32_t capc);

int ortho_digits_fill(void* stream, int64_t n, const double* X, int64_t ldx, int32_t c0, int32_t nc,
                      void* d_digits, int32_t capc);

int ortho_gram_chol_tcd(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k,
                        const double* V, int64_t ldv, int32_t nb, double* R, int32_t ldr,
                        void* d_work, size_t work_bytes, int32_t* d_status,
                        const void* d_digits, int32_t capc, int32_t kc);

int ortho_update_tcd(void* stream, int64_t n, const double* Q, int64_t ldq, int32_t k,
                     double* V, int64_t ldv, int32_t nb, const double* R, int32_t ldr,
                     const int32_t* d_status, void* d_digits, int32_t capc);

/* ------------------------------------------------ batched solver (many uneven systems)
 * nsys independent systems of different sizes and matrices share one set of
 * options (m, s, panel, tol, precision) and advance together: one restart
 * cycle of every active system is one CUDA-graph launch of persistent kernels
 * over all systems' work (rows are concatenated, A is block diagonal).  A
 * system's reductions use the same split and order whatever the batch holds,
 * so its result does not depend on the other systems.  CSR arrays (rowptr
 * int64, colind int32, vals FP64) and b, x are per-system HOST arrays; x holds
 * x0 on entry.  res (may be NULL) receives nsys results.  A NULL stream makes
 * the batch create its own non-blocking stream (graph capture cannot use the
 * legacy default stream).  gmres_batch_solve returns GMRES_OK when every
 * system converged, else the most severe per-system status. */
typedef struct gmres_batch gmres_batch;

/* Device bytes a batch of these sizes would allocate (for admission control);
 * 0 for options gmres_batch_create rejects, n[i] < 1 or nnz[i] < 0. */
size_t gmres_batch_footprint(int32_t nsys, const int64_t* n, const int64_t* nnz, const gmres_opts* opts);

int gmres_batch_create(gmres_batch** out, int32_t nsys, const int64_t* n, const int64_t* const* rowptr,
                       const int32_t* const* colind, const double* const* vals, const gmres_opts* opts,
                       void* stream);

int gmres_batch_solve(gmres_batch* b, const double* const* rhs, double* const* x, gmres_result* res);

/* Time candidate persistent-grid sizes of the batched Gram and row kernels on
 * this batch's shapes and keep the fastest (res_ms[4] = best Gram ms, best
 * update ms, Gram grid, row grid; may be NULL).  Changes speed, never results. */
int gmres_batch_autotune(gmres_batch* b, double* res_ms);

int gmres_batch_destroy(gmres_batch* b);   /* NULL-safe */

/* Device bytes gmres_create would allocate for an n x n matrix with nnz
 * nonzeros under these options (0 for invalid arguments). */
size_t gmres_footprint(int64_t n, int64_t nnz, const gmres_opts* opts);

/* ------------------------------------------------ serving loop (continuous batching)
 * A worker thread serves independent solves of different sizes, matrices and
 * options.  Requests are admitted in arrival order whenever a slot is free
 * and their device footprint (gmres_footprint) fits the unused part of the
 * memory budget; admitted solves run concurrently on streams of their own,
 * one restart cycle at a time, each keeping its Krylov basis and Hessenberg
 * state resident on the device until it finishes.  A request that arrives
 * while others are running joins them at the next cycle boundary.  Results do
 * not depend on what else is being served.  Latency is submit-to-completion
 * on the host clock. */
typedef struct gmres_server gmres_server;

typedef struct gmres_server_stats {
    int64_t submitted, admitted, completed, rejected, failed, active, pending;
    double  p50_ms, p99_ms, mean_ms;    /* latency of completed requests            */
    double  solves_per_s, busy_s;       /* completed / (last completion - first submit) */
    size_t  mem_budget, mem_in_use;     /* bytes                                     */
} gmres_server_stats;

/* mem_budget = 0: 90% of the device memory free at start.  max_active >= 1. */
int gmres_server_start(gmres_server** out, size_t mem_budget, int32_t max_active);

/* Copies the host CSR (rowptr int64, colind int32, vals FP64), b and x0 (may
 * be NULL: zero) and queues the request; *id identifies it.  A request whose
 * footprint exceeds the whole budget finishes at once with GMRES_ERR_OOM. */
int gmres_server_submit(gmres_server* s, int64_t n, const int64_t* rowptr, const int32_t* colind,
                        const double* vals, const double* b, const double* x0, const gmres_opts* opts,
                        int64_t* id);

/* 1 = finished (x[n] and *res filled, the request released), 0 = not yet
 * (timeout_s < 0 waits forever; poll = wait with timeout 0), GMRES_ERR_ARG for
 * an id that was never submitted or has already been collected. */
int gmres_server_wait(gmres_server* s, int64_t id, double* x, gmres_result* res, double timeout_s);
int gmres_server_poll(gmres_server* s, int64_t id, double* x, gmres_result* res);

int gmres_server_get_stats(gmres_server* s, gmres_server_stats* st);

/* Serves every queued and running request to completion, then joins the
 * worker and frees the server (results not collected are dropped). */
int gmres_server_stop(gmres_server* s);

/* z = M^{-1} r for the context's preconditioner (opts.precond = GMRES_PRECOND_MCGS):
 * one forward multicolor Gauss-Seidel sweep from zero (§VIII, Fig. 9; the
 * coloring and order of GMRES_PRECOND_MCGS).  r and z are n FP64 values in
 * device memory, distinct; synchronizes the context's stream.  GMRES_ERR_ARG
 * when the context has no preconditioner. */
int gmres_precond_apply(gmres_ctx* c, const double* r, double* z);

/* ------------------------------------------------ matrix powers kernel
 * MPK of §III (standard, not communication-avoiding): s products in sequence,
 * W[:,0] = (A v - theta_0 v) / sigma, W[:,i] = (A W[:,i-1] - theta_i W[:,i-1]) / sigma,
 * with the context's matrix.  v[n] and W (n x s, ldw >= n) are device FP64;
 * theta is a HOST array of s shifts, or NULL for the monomial basis; sigma is
 * finite and nonzero; the context must be FP64 (GMRES_ERR_ARG otherwise).
 * Asynchronous on the context's stream. */
int gmres_mpk(gmres_ctx* c, const double* v, double* W, int64_t ldw, int32_t s,
              double sigma, const double* theta);

/* ------------------------------------------------ Newton-basis shifts
 * The shifts GMRES_BASIS_NEWTON_AUTO takes after its first cycle (host code,
 * no device work; the Newton basis is the better-conditioned alternative to
 * the monomial basis for large s that the paper names, with Leja-ordered Ritz
 * values as in Bai, Hu and Reichel 1994).
 *   H, ldh   HOST k x k upper Hessenberg matrix, column-major (entries below the
 *            subdiagonal are not read); k = 0 gives theta = 0
 *   theta    HOST out, s values: the real parts of the eigenvalues of H
 *            (Francis double-shift QR) in Leja order, the first s, cycled when
 *            k < s.  Leja order: start at the largest modulus, then the largest
 *            product of distances to the points taken; candidates scanned in
 *            ascending order, ties to the first
 *   sigma    HOST in/out, may be NULL: the power of two nearest (in log2) to the
 *            capacity (max theta - min theta) / 4 of the shifts' interval;
 *            unchanged when the shifts span no interval
 * Returns GMRES_ERR_ARG (0 <= k <= 256, 1 <= s <= 16, ldh >= k) or
 * GMRES_ERR_EIG (non-finite H, or an eigenvalue took more than 60 sweeps). */
int gmres_newton_shifts(const double* H, int32_t ldh, int32_t k, int32_t s, double* theta, double* sigma);

#ifdef __cplusplus
}
#endif
#endif /* GB300_SSTEP_GMRES_H */
