/*
 * gpk.h -- C ABI of libgpk: low-precision matrix-free Gaussian-process solves
 * on one NVIDIA GB300 (sm_103a).
 *
 * The library implements the hot path of "Low-Precision Arithmetic for Fast
 * Gaussian Processes" (Maddox, Potapczynski & Wilson, 2022): the matrix-free
 * kernel MVM of Eq. mvm on tensor cores in FP16/BF16 with FP32 accumulation,
 * inside the enhanced-stability preconditioned conjugate-gradient solve of
 * Alg. 2 (log-scale step sizes, re-orthogonalisation, pivoted-Cholesky /
 * Woodbury preconditioner of Eq. woodbury), and the pseudo-loss gradient of
 * Eq. approx.
 *
 * Conventions shared by every entry point
 *   - Return GP_OK (0) or a negative GP_ERR_* status; nothing is thrown.
 *   - Pointers named "device" are CUDA device pointers owned by the caller;
 *     the library never frees them.  "host" pointers are ordinary memory.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     are asynchronous on it unless they return host values, in which case
 *     they synchronise the stream before returning.
 *   - Inputs X are N x d row-major FP32 (point i is X[i*d .. i*d+d-1]).
 *     Blocks of vectors (right-hand sides, solutions, MVM inputs/outputs) are
 *     N x R column-major FP32: vector c is V[c*N .. c*N+N-1].
 *   - Device memory: every call that needs scratch space takes it from the
 *     context's workspace, which is allocated by gp_ctx_create / gp_ctx_reserve
 *     and never inside a compute call.  A call whose need exceeds the
 *     workspace returns GP_ERR_WORKSPACE; the *_workspace_size queries give
 *     the need in advance.
 *   - A context may be used by one host thread at a time.
 *   - Device-side waits in the kernels are bounded; a wait that runs out sets
 *     the context's device error word, reported as GP_ERR_TIMEOUT by the next
 *     call that checks it (gp_ctx_check, and every call returning host values).
 */
#ifndef GPK_H
#define GPK_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GPK_API __attribute__((visibility("default")))
#else
#define GPK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define GP_OK                  0
#define GP_ERR_INVALID        -1  /* argument out of range / inconsistent      */
#define GP_ERR_CUDA           -2  /* CUDA runtime or driver call failed        */
#define GP_ERR_WORKSPACE      -3  /* context workspace smaller than required   */
#define GP_ERR_BREAKDOWN      -4  /* LSE sum <= 0: d^T K d or r^T z not > 0     */
#define GP_ERR_NONFINITE      -5  /* NaN/Inf in an input or an iterate          */
#define GP_ERR_NOT_CONVERGED  -6  /* CG hit max_iter; solution and stats valid  */
#define GP_ERR_TIMEOUT        -7  /* a bounded device-side wait ran out         */
#define GP_ERR_OOM            -8  /* allocation refused (create/reserve only)   */
#define GP_ERR_UNSUPPORTED    -9  /* shape or option not supported             */

/* ---- kernels (k as a function of r, r^2 = sum_k (x_k - x'_k)^2 / l_k^2) -- */
#define GP_KERNEL_RBF       0   /* exp(-r^2/2)                    App. C.1   */
#define GP_KERNEL_MATERN32  1   /* (1 + sqrt3 r) exp(-sqrt3 r)    textbook   */
#define GP_KERNEL_MATERN12  2   /* exp(-r)                        Sec. 3.1   */
#define GP_KERNEL_MATERN52  3   /* (1 + sqrt5 r + 5r^2/3) exp(-sqrt5 r)      */

/* ---- MVM operand precision (low byte of `flags` / gp_cg_opts_t.precision) */
#define GP_PREC_FP32  0   /* SIMT FP32 throughout (the plain comparator)          */
#define GP_PREC_FP16  1   /* FP16 tensor-core operands, FP32 accumulation (Sec. 4.1) */
#define GP_PREC_BF16  2   /* BF16 tensor-core operands, FP32 accumulation          */

/* ---- gp_kmvm flags (OR-ed with a GP_PREC_* value) ------------------------ */
#define GP_MVM_ADD_NOISE     0x100  /* add sigma^2 v (needs Xr == Xc, Nr == Nc)     */
#define GP_MVM_XSPLIT        0x200  /* hi+lo split of the scaled inputs (more exact
                                       distances; default on for BF16)            */
#define GP_MVM_NO_XSPLIT     0x400  /* force the split off                         */
#define GP_MVM_SCALE_SQRT_N  0x800  /* paper-literal operand scaling v / N^{1/2}
                                       (Sec. 4.1) instead of the per-column power
                                       of two                                     */
#define GP_MVM_VSPLIT       0x1000  /* FP16: carry v as hi + lo (robust to heavy
                                       cancellation in K v; BF16 always does, and
                                       so does FP16 on the pair engine, where it
                                       costs no extra tensor-core instruction)   */
#define GP_MVM_BF16_SINGLE  0x2000  /* BF16: single-term kernel tile and v (faster,
                                       ~2^-8 rounding; the default carries both as
                                       hi + lo so the MVM meets 2e-3)             */
#define GP_MVM_PSPLIT       0x8000  /* FP16: carry the kernel tile as hi + lo (22
                                       bits; CG then needs about the FP32 iteration
                                       count, at about 1.5x the MVM time).  BF16
                                       does by default.                          */
#define GP_MVM_HALF_EXP    0x10000  /* FP16 RBF: the exp2 argument rounded to FP16
                                       by the tensor core and 2^s evaluated in
                                       FP16 (ex2.approx.f16x2), the paper's
                                       half-precision kernel evaluation (Sec. 4.1);
                                       pair engine, d <= 12 without input split  */
#define GP_MVM_SKIP_TILES  0x20000  /* compact support (Sec. 3.1, Fig. 2c): skip the
                                       tile pairs whose operand bounding boxes put
                                       every kernel value below half the smallest
                                       subnormal of the kernel tile's format, where
                                       it rounds to an exact 0 (bit-identical
                                       result); pair engine, FP16 / BF16            */
/* Summation-variant study (Sec. 4.1, Fig. 4b; App. B, Fig. A.1a), FP16 only, R <= 8:
 * a CUDA-core FP16 MVM (kernel value and products in FP16) whose row sums are
 * accumulated by scheme x: 1 FP32, 2 FP16 (one running sum), 3 FP16 per
 * 128-column block then FP32 across blocks, 4 Kahan-compensated FP16.  A study
 * engine, not the hot path.                                                    */
#define GP_MVM_SUM(x)     (((x) & 0x7) << 18)
#define GP_MVM_SUM_MASK   (0x7 << 18)
#define GP_MVM_SYMMETRIC 0x200000  /* FP32 only, square operator (Xc == Xr),
                                       R <= 24, d <= 32: K = K^T, each kernel value
                                       evaluated once for the row and the column
                                       it belongs to (N(N+1)/2 evaluations; an
                                       extension toward the Conclusion's future
                                       work); sums added with FP32 atomics, so the
                                       last bits vary from run to run.  Other
                                       shapes: GP_ERR_UNSUPPORTED (non-square,
                                       R > 24, d > 32) or GP_ERR_INVALID (with a
                                       non-FP32 precision). */
#define GP_MVM_FP32_PV    0x400000  /* FP16, pair engine, R <= 4: S on the tensor
                                       cores as usual, the kernel values kept in
                                       FP32 and the value product sum_j k_ij v_j
                                       done by the epilogue threads in FP32 FMAs
                                       (v as hi + lo), instead of rounding P to
                                       FP16 for a tensor-core product whose
                                       M = 128 rows would hold 1..4 right-hand
                                       sides.  For the single-column solves of
                                       serving.  Other shapes: GP_ERR_UNSUPPORTED. */
#define GP_MVM_ONE_TILE     0x4000  /* tensor-core MVM on the one-row-tile engine
                                       (P V with M = 128 rows, N = R) instead of
                                       the default pair engine (transposed
                                       V^T P^T, N = 256 rows); for comparison     */

/* GP hyperparameters theta = (l_1..l_d, a^2, sigma^2)   (Sec. 2.2, Eq. mvm) */
typedef struct {
    int kernel;                 /* GP_KERNEL_*                                   */
    int d;                      /* input dimension, 1..64                       */
    const float* lengthscale;   /* host [d], all > 0                            */
    double outputscale;         /* a^2 > 0                                      */
    double noise;               /* sigma^2 >= 0 (> 0 for solves)                */
} gp_hyp_t;

typedef struct gp_ctx gp_ctx;

/* Create a context on CUDA device `device` with `workspace_bytes` of device
 * scratch memory (may be 0 and grown later with gp_ctx_reserve).  Allocates. */
GPK_API int gp_ctx_create(int device, size_t workspace_bytes, gp_ctx** out);
/* Free the context and its workspace.  NULL is accepted. */
GPK_API void gp_ctx_destroy(gp_ctx* ctx);
/* Grow the workspace to at least `workspace_bytes` (synchronises the device;
 * allocates).  Never shrinks. */
GPK_API int gp_ctx_reserve(gp_ctx* ctx, size_t workspace_bytes);
/* Current workspace size in bytes. */
GPK_API size_t gp_ctx_workspace_bytes(const gp_ctx* ctx);
/* Synchronise `stream`, read and clear the device error word; returns
 * GP_ERR_TIMEOUT (or another GP_ERR_*) if a kernel recorded one. */
GPK_API int gp_ctx_check(gp_ctx* ctx, void* stream);
/* Failure-detection check of the device-side bounded waits: launches one warp
 * that waits on an mbarrier nothing completes, with the wait helper of the MVM
 * kernels (sleep = 0: spinning try_wait, 1: try_wait with a suspend hint) and
 * a limit of `limit_ms` (0 < limit_ms <= 1000).  The wait gives up, the kernel
 * records a timeout in the context's device error word and returns, so the
 * next gp_ctx_check on the stream returns GP_ERR_TIMEOUT and the context stays
 * usable.  If `waited_cycles` is not null, the SM clock cycles the wait lasted
 * are written there (the call then synchronises the stream and uses the first
 * 8 bytes of the workspace).  Errors: GP_ERR_INVALID, GP_ERR_WORKSPACE,
 * GP_ERR_CUDA. */
GPK_API int gp_wait_check(gp_ctx* ctx, double limit_ms, int sleep, long long* waited_cycles, void* stream);
/* Number of kernels this context has launched since creation (all entry
 * points; each CUDA kernel launch counts one). */
GPK_API int64_t gp_ctx_launch_count(const gp_ctx* ctx);
/* Static description of a status code. */
GPK_API const char* gp_strerror(int status);

/* ---- measurement support (Sec. 4.1 timing study) --------------------------
 * gp_ctx_profile(ctx, 1) records a CUDA event pair around every tensor-core
 * MVM launch on its stream (up to 8192 launches; creates the events, so call
 * it outside timed regions).  gp_ctx_profile_read synchronises those events,
 * returns the summed launch time in ms and the launch count, and resets.
 * gp_measure_peaks runs throughput loops (8 independent chains per thread,
 * 8 CTAs of 256 threads per SM) and returns the best of 5 rates in
 * operations/s for ex2.approx.f32 and sqrt.approx.f32 (special function
 * units) and FP32 FMA; it allocates 256 B of scratch.  Diagnostic only: the
 * paper has no counterpart. */
GPK_API int gp_ctx_profile(gp_ctx* ctx, int enable);
GPK_API int gp_ctx_profile_read(gp_ctx* ctx, double* total_ms, int64_t* launches);
GPK_API int gp_measure_peaks(gp_ctx* ctx, double* ex2_per_s, double* sqrt_per_s, double* ffma_per_s,
                             void* stream);
/* As gp_measure_peaks, plus FP32-pair -> FP16x2 pack conversions per second
 * (round trip, counted once per pair) and kernel values per second of the
 * FP16 epilogue mix (two ex2 and one pack per pair of values); any output
 * pointer may be NULL. */
GPK_API int gp_measure_peaks2(gp_ctx* ctx, double* ex2_per_s, double* sqrt_per_s, double* ffma_per_s,
                              double* pack_per_s, double* ex2pack_per_s, void* stream);

/* ---- matrix-free kernel MVM (Eq. mvm, Sec. 4.1) ---------------------------
 *   out[:, c] = a^2 K(Xr, Xc) V[:, c]  (+ sigma^2 V[:, c] with GP_MVM_ADD_NOISE)
 * K is never stored: 128 x 128 tiles of the kernel matrix are formed on chip
 * (distance contraction on tensor cores, kernel function on the special
 * function units) and contracted with V at once, block sums in FP32
 * (Sec. 4.1, "block summation in a higher precision").
 *   Xr   device, Nr x d row-major FP32      Xc   device, Nc x d row-major FP32
 *   V    device, Nc x R column-major FP32   out  device, Nr x R column-major FP32
 *   R    1..64 right-hand sides (more: call per block of 64)
 *   flags  GP_PREC_* | GP_MVM_*
 * Nr, Nc >= 1; Nc <= 2^31 - 128.  out must not alias V.
 * Errors: GP_ERR_INVALID (shape/flags), GP_ERR_WORKSPACE, GP_ERR_CUDA. */
GPK_API size_t gp_kmvm_workspace_size(const gp_hyp_t* hyp, int64_t Nr, int64_t Nc, int R, int flags);
GPK_API int gp_kmvm(gp_ctx* ctx, const gp_hyp_t* hyp,
            const float* Xr, int64_t Nr, const float* Xc, int64_t Nc,
            const float* V, int R, float* out, int flags, void* stream);

/* Evaluated and total (row-tile pair, column tile) entries of the MVM that
 * gp_kmvm would run for these arguments with GP_MVM_SKIP_TILES (without the
 * flag every entry is evaluated).  Prepares the operands in the context's
 * workspace; synchronises the stream.  One entry = 256 x 128 kernel pairs. */
GPK_API int gp_kmvm_tile_count(gp_ctx* ctx, const gp_hyp_t* hyp, const float* Xr, int64_t Nr, const float* Xc,
                               int64_t Nc, int flags, int64_t* evaluated, int64_t* total, void* stream);

/* ---- kernel MVM without any allocation -------------------------------------
 * gp_kmvm_noalloc computes exactly what gp_kmvm computes (same arguments and
 * flags, same kernels and results), for callers that cannot allocate device
 * memory: host applications that own every device allocation through their
 * own pool and forbid side allocations, latency-critical loops that cannot
 * afford an allocation, plugins handed device pointers but no way to allocate.
 * It takes no context and allocates nothing; the caller still passes the
 * inputs and the output.  Its scratch is a fixed array of
 * GPK_NOALLOC_SCRATCH_BYTES in device memory, held by every GPU that loads the
 * library until the process exits.  A problem whose scratch need (as
 * gp_kmvm_workspace_size reports for these arguments) exceeds that size is
 * rejected with GP_ERR_WORKSPACE.
 * - The first call on a device looks up the array's device address; make
 *   that first call before any stream capture.
 * - Every call shares the array: calls whose work overlaps on the GPU (for
 *   example on two unordered streams) race and corrupt each other.
 * - Asynchronous on `stream` like gp_kmvm; a device-side wait that runs out
 *   (or another device-side status) is recorded in an error word at the
 *   start of the shared array: read it with gp_kmvm_noalloc_check.
 * - The array's device address is cached per device for the life of the
 *   process; it does not survive a reset of the device's primary context
 *   (cudaDeviceReset): make no call after one.
 * The paper has no counterpart: this is a deployment variant of Eq. mvm. */
#define GPK_NOALLOC_SCRATCH_BYTES (16u << 20)
GPK_API int gp_kmvm_noalloc(const gp_hyp_t* hyp, const float* Xr, int64_t Nr, const float* Xc, int64_t Nc,
                            const float* V, int R, float* out, int flags, void* stream);
/* Status of the gp_kmvm_noalloc calls on the current device since the last
 * check: synchronises `stream`, reads the error word of the shared array and
 * clears it.  Returns GP_OK, GP_ERR_TIMEOUT (a bounded device-side wait ran
 * out), GP_ERR_NONFINITE, or GP_ERR_CUDA.  Allocates nothing. */
GPK_API int gp_kmvm_noalloc_check(void* stream);

/* ---- pivoted-Cholesky preconditioner (Sec. 4.2, Eq. woodbury) -------------
 * k = rank steps of partial pivoted Cholesky of K (no noise) from kernel rows
 * K e_p and the constant diagonal a^2: pivot = argmax of the remaining
 * diagonal (lowest index on ties); stops early when that value falls to
 * 1e-6 a^2 (FP32 rows).  Then the Woodbury core C = I + sigma^-2 L^T L is
 * formed and factored in FP64.  P = L L^T + sigma^2 I.
 *   X     device, N x d row-major FP32
 *   L     device, N x rank column-major FP32 (columns >= rank_out undefined)
 *   piv   device, int32 [rank] pivot indices
 *   core  device, rank_out x rank_out column-major FP64, lower factor Lc of C
 *         (C = Lc Lc^T; leading dimension rank_out)
 *   rank_out host: the rank reached.  Synchronises the stream.
 * Requires 1 <= rank <= min(N, 512) and noise > 0. */
GPK_API size_t gp_pivchol_workspace_size(const gp_hyp_t* hyp, int64_t N, int rank);
GPK_API int gp_pivchol_precond(gp_ctx* ctx, const gp_hyp_t* hyp, const float* X, int64_t N, int rank,
                               float* L, int32_t* piv, double* core, int* rank_out, void* stream);

/* Preconditioner handed to the solvers: P^{-1} w = sigma^-2 w -
 * sigma^-4 L C^{-1} L^T w (Eq. woodbury).  rank = 0 means no preconditioner
 * (P = I). */
typedef struct {
    const float* L;       /* device, N x rank column-major FP32               */
    const double* core;   /* device, rank x rank lower Cholesky factor of C   */
    int rank;
} gp_precond_t;

/* ---- preconditioned conjugate gradients (Alg. 1, Alg. 2, App. A) ---------- */
#define GP_CG_STABLE     0  /* Alg. 2: log-scale alpha/beta (LSE), re-orthogonalisation */
#define GP_CG_STANDARD   1  /* Alg. 1: textbook preconditioned CG                          */
#define GP_REORTH_NONE   0
#define GP_REORTH_PINV   1  /* project against past residuals in the P^{-1} inner product,
                               in which preconditioned residuals are orthogonal (default) */
#define GP_REORTH_EUCLID 2  /* literal Alg. 2: Euclidean-normalised past residuals
                               (exactly orthogonal only when P = I)                       */

typedef struct {
    double tol;          /* stop column c when ||r_c|| / ||b_c|| <= tol (recursive residual) */
    int max_iter;        /* 1 .. 1000                                                       */
    int min_iter;        /* iterations run before the tolerance is tested                   */
    int precision;       /* MVM flags: GP_PREC_* | GP_MVM_* option bits (no ADD_NOISE)      */
    int algorithm;       /* GP_CG_STABLE or GP_CG_STANDARD                                  */
    int reorth;          /* GP_REORTH_*; only used by GP_CG_STABLE                          */
    int reorth_passes;   /* 1 = classical Gram-Schmidt, 2 = twice (CGS2)                    */
    int x0_given;        /* nonzero: U holds the initial guess x_0 on entry                 */
    int restarts;        /* true-residual checks: when every column has met tol on its
                            recursive residual, r = K x - b is recomputed with the same
                            MVM and columns still above tol restart from their current x
                            (fresh basis); at most this many times.  0 = trust the
                            recursive residual (re-orthogonalisation changes r but not
                            x, so the two drift apart by rounding)                   */
    int check_precision; /* GP_PREC_* (optionally | GP_MVM_* operand flags) of the MVM
                            that recomputes r = K x - b at a true-residual check: the
                            restarts become mixed-precision iterative refinement, since a
                            single-rounded half-precision MVM cannot resolve the residual
                            of its own solution when K x cancels heavily (|x| >> |b| for
                            small sigma^2).  Use GP_PREC_FP32: the check's rounding error
                            scales with sum_j |k_ij x_j|, which near the solution exceeds
                            |(K x)_i| by the cancellation factor (hundreds on the bench
                            workload), so even the hi + lo FP16 MVM (~1e-5) misreports
                            a 1e-2 residual by ~10 %                                 */
    int escalate;        /* nonzero: when a run ends with a breakdown (a non-positive
                            d^T K d or r^T z: the low-precision operator is not positive
                            definite to the accuracy the solve has reached), the
                            true-residual restart continues the solve with the
                            check_precision MVM.  Needs restarts > 0.                */
    int refine_precision; /* 0 = off; else the MVM flags (GP_PREC_* | GP_MVM_*) the
                            solve switches to, for the rest of the solve, at the moment
                            refine_resid sets                                          */
    double refine_resid;  /* > 0: switch once the recursive relative residual of every
                            active column is <= refine_resid (within the run: with an
                            accurate first MVM and a cheaper refine MVM this relaxes the
                            operator as the residual falls, whose rounding then moves
                            the true residual less; after a switch below the starting
                            residual a guard returns to the solve's MVM for good if the
                            largest residual has not halved within max(20, k_switch / 4)
                            iterations of the switch or has doubled); 0: switch at the first
                            true-residual check (the restarts run on the refine MVM:
                            refinement in the operator; needs restarts > 0)           */
} gp_cg_opts_t;

/* Host-side statistics (every pointer may be NULL). */
typedef struct {
    int iters;           /* iterations run (max over columns)                 */
    int converged;       /* columns that reached tol                          */
    int breakdowns;      /* columns stopped by an LSE breakdown               */
    int restarts;        /* true-residual restarts performed                  */
    int escalated;       /* 1 if a breakdown moved the solve to check_precision */
    int* col_iters;      /* [R]                                               */
    double* rel_resid;   /* [R] final relative residual: the recomputed one after a
                            true-residual check, else the recursive one           */
    double* alpha;       /* [max_iter * R]: alpha_k of column c at k*R + c    */
    double* beta;        /* [max_iter * R]: beta_{k+1} of column c at k*R + c */
    double* gamma0;      /* [R] r_0^T z_0                                     */
    double* resid_hist;  /* [(max_iter + 1) * R] relative residual per iterate */
    int* lanczos_len;    /* [R] iterations before the first true-residual restart: the
                            length of the Lanczos process the step sizes describe     */
} gp_cg_stats_t;

/* Solve (K + sigma^2 I) U = B for R right-hand sides at once (Eq. cg; mBCG of
 * App. A: every column has its own alpha_k, beta_k and stops on its own).
 * The MVM inside is gp_kmvm's (precision from opts).  Scalars alpha, beta,
 * gamma, the residual norms and the re-orthogonalisation coefficients are
 * FP64; vectors are FP32.
 *   X  device N x d; B device N x R column-major; U device N x R (in: x_0 when
 *   opts->x0_given, out: solution).  1 <= R <= 64.
 * Synchronises the stream once per iteration (convergence flags).
 * Returns GP_OK when every column converged, GP_ERR_NOT_CONVERGED when some
 * did not within max_iter (U and stats still valid), GP_ERR_BREAKDOWN when a
 * column's LSE sum was not positive (that column keeps its last iterate). */
GPK_API size_t gp_cg_workspace_size(const gp_hyp_t* hyp, int64_t N, int R, int rank, const gp_cg_opts_t* opts);
GPK_API int gp_cg_solve(gp_ctx* ctx, const gp_hyp_t* hyp, const float* X, int64_t N, const float* B, int R,
                        float* U, const gp_precond_t* precond, const gp_cg_opts_t* opts, gp_cg_stats_t* stats,
                        void* stream);

/* ---- low-precision preconditioned MINRES (Conclusion, future work) ----------
 * MINRES (Paige and Saunders' Lanczos-based minimum-residual method) for
 * (K + sigma^2 I) U = B with the same kernel MVM engines and the same
 * pivoted-Cholesky preconditioner P as gp_cg_solve: the Conclusion names the
 * low-precision and mixed-precision approach of the paper as applicable to
 * MINRES.  Over the Krylov space of P^-1 Ktilde it minimises the residual in
 * the P^-1 norm, ||r||_{P^-1} = sqrt(r^T P^-1 r) (the 2-norm without a
 * preconditioner); each column runs its own Lanczos process and QR
 * factorisation (Givens rotations) in FP64 on the device, all columns share
 * one MVM per iteration.  A column stops when ||r_k||_{P^-1} / ||b||_{P^-1}
 * <= tol (the recurrence's estimate).  With restarts > 0, when every column
 * has stopped, r = b - Ktilde x is recomputed with the check_precision MVM and
 * the columns whose true P^-1-norm residual is above tol restart from their
 * current x (fresh Lanczos process).                                          */
typedef struct {
    double tol;          /* relative residual in the P^-1 norm                      */
    int max_iter;        /* 1 .. 1000 (iterations over all runs)                    */
    int precision;       /* MVM flags: GP_PREC_* | GP_MVM_* option bits              */
    int restarts;        /* true-residual checks, 0 .. 16                           */
    int check_precision; /* MVM flags of the checks and of the final residual       */
    int norm;            /* GP_MINRES_NORM_P (0): tol applies to ||r||_{P^-1}; or
                            GP_MINRES_NORM_2 (1): tol applies to ||r||_2 / ||b||_2 at
                            the true-residual checks (and for the status); after a
                            check each column's recurrence stops at
                            tol * 0.95 * (P^-1-norm / 2-norm of its recomputed
                            residual), the norms' observed ratio.  Needs restarts > 0. */
    int refine_precision; /* 0 = off; else MVM flags the solve switches to once the
                            recurrence's relative residual of every active column is
                            <= refine_resid (> 0), with the stagnation guard of
                            gp_cg_opts_t: the relaxed schedule of the CG solve     */
    double refine_resid;
} gp_minres_opts_t;
#define GP_MINRES_NORM_P 0
#define GP_MINRES_NORM_2 1

typedef struct {
    int iters;           /* iterations run (over all runs)                          */
    int converged;       /* columns whose final residual (in the opts' norm) is <= tol */
    int breakdowns;      /* columns stopped because r^T P^-1 r was negative or NaN  */
    int restarts;        /* true-residual restarts performed                        */
    int* col_iters;      /* [R] or null: iterations of each column                  */
    double* rel_resid;   /* [R] or null: final ||Ktilde x - b||_2 / ||b||_2 (check MVM) */
    double* rel_resid_p; /* [R] or null: final ||Ktilde x - b||_{P^-1} / ||b||_{P^-1}   */
    double* resid_hist;  /* [(max_iter + 1) * R] or null: the recurrence's P^-1-norm
                            relative residual after each iteration (k * R + c)      */
} gp_minres_stats_t;

/* B, U: R x N row-major (right-hand side c at c * N), device, FP32; U is
 * overwritten with the solution (x_0 = 0).  precond may be null (P = I).
 * Workspace from the context (gp_minres_workspace_size).  Returns GP_OK when
 * every column meets tol, GP_ERR_NOT_CONVERGED when some did not within
 * max_iter (U and stats still valid), GP_ERR_BREAKDOWN when a column's
 * r^T P^-1 r was not positive (that column keeps its last iterate),
 * GP_ERR_INVALID / GP_ERR_WORKSPACE / GP_ERR_CUDA / GP_ERR_TIMEOUT otherwise. */
GPK_API size_t gp_minres_workspace_size(const gp_hyp_t* hyp, int64_t N, int R, int rank,
                                        const gp_minres_opts_t* opts);
GPK_API int gp_minres_solve(gp_ctx* ctx, const gp_hyp_t* hyp, const float* X, int64_t N, const float* B, int R,
                            float* U, const gp_precond_t* precond, const gp_minres_opts_t* opts,
                            gp_minres_stats_t* stats, void* stream);

/* ---- backward of the kernel MVM (gradient of a bilinear form) --------------
 * grad_theta[0..d+2) = d/d(l_1..l_d, a^2, sigma^2) of  q = sum_c u_c^T Ktilde w_c,
 * and, when grad_X is not NULL, grad_X = dq/dX (device, N x d row-major).
 * With r^2 = sum_m (x_im - x_jm)^2 / l_m^2 and G_ij = sum_c u_ic w_jc:
 *   dq/da^2 = sum_ij G_ij k(r^2);  dq/dl_m = -(2/l_m^3) sum_ij G_ij a^2 k'(r^2) (x_im - x_jm)^2;
 *   dq/dsigma^2 = sum_c u_c^T w_c;  dq/dx_im = (2/l_m^2) sum_j (G_ij + G_ji) a^2 k' (x_im - x_jm).
 * Pairs are evaluated on the fly in FP32 (CUDA cores), sums reduced in FP64.
 *   X device N x d; U, W device N x R column-major, 1 <= R <= 32; d <= 32.
 * grad_theta is host memory; the call synchronises the stream. */
GPK_API size_t gp_kmvm_vjp_workspace_size(const gp_hyp_t* hyp, int64_t N, int R);
GPK_API int gp_kmvm_vjp(gp_ctx* ctx, const gp_hyp_t* hyp, const float* X, int64_t N, const float* U,
                        const float* W, int R, double* grad_theta, float* grad_X, void* stream);

/* The same gradient with a choice of arithmetic:
 *   GP_PREC_FP32  the CUDA-core FP32 backward above (gp_kmvm_vjp);
 *   GP_PREC_FP16  the tensor-core backward (flash-attention-backward shape):
 *     S = X_i X_j^T and H = [u | w]_i [w | u]_j^T on tcgen05 (FP16 operands,
 *     FP32 accumulation in TMEM), W' = a^2 k'(r^2) H elementwise (exp / sqrt on
 *     the special function units), then W' [x / l, 1] on tcgen05 gives the row
 *     sums and W' X from which every derivative follows (Eq. gradient: with
 *     H = G + G^T symmetric, sum_ij a^2 k' G_ij (x_im - x_jm)^2 and
 *     sum_j (G_ij + G_ji) a^2 k' (x_im - x_jm) are sums of W' (x_im - x_jm)).
 *     RBF, Matern-3/2 and Matern-5/2 with d <= 31 (d <= 20 when d > 12, where
 *     the inputs are carried as hi + lo); Matern-1/2 (k' ~ 1/r, singular at
 *     coincident points) and wider inputs return GP_ERR_UNSUPPORTED.
 * gp_mll_and_grad uses the FP16 backward whenever its solve's MVM precision is
 * not FP32 and the shape is supported. */
GPK_API size_t gp_kmvm_vjp_prec_workspace_size(const gp_hyp_t* hyp, int64_t N, int R, int precision);
GPK_API int gp_kmvm_vjp_prec(gp_ctx* ctx, const gp_hyp_t* hyp, const float* X, int64_t N, const float* U,
                             const float* W, int R, int precision, double* grad_theta, float* grad_X, void* stream);

/* ---- stochastic Lanczos quadrature from CG step sizes (host) ---------------
 * out = gamma0 * e1^T log(T) e1 for the Lanczos tridiagonal T of a CG run
 * with step sizes alpha[0..J) and beta[0..J-1) (beta[k] = beta_{k+1} of
 * Alg. 2): T_kk = 1/alpha_k + beta_k/alpha_{k-1}, T_{k,k+1} = sqrt(beta_{k+1})/alpha_k.
 * gamma0 = r_0^T z_0 of that run.  Host only (no GPU needed).  FP64
 * eigen-decomposition of T by implicit-shift QL. */
GPK_API int gp_slq_quadrature(const double* alpha, const double* beta, int J, double gamma0, double* out);

/* ---- loss and gradient (Sec. 4.3, Eq. loss / approx_loss / approx) ---------- */
#define GP_MLL_PRECOND_PROBES 0x1  /* z_j = L e_j + sigma z~_j (E[zz^T] = P) from the
                                      standard normals Z (z~) and E; gradient pairs
                                      u_j with P^{-1} z_j; enables the SLQ log|Ktilde|
                                      with log|P| added exactly                       */
#define GP_MLL_WANT_LOGDET    0x2  /* estimate log|Ktilde| by SLQ for the loss value
                                      (needs PRECOND_PROBES, or no preconditioner)     */
/* Lanczos depth of the loss value, decoupled from the solve tolerance: with
 * GP_MLL_WANT_LOGDET every column runs at least n (<= 255) CG iterations, so
 * that the SLQ quadrature of each probe and y^T u_0 are taken from at least
 * n Lanczos steps even at a loose training tolerance (such as 1.0, where the
 * solve would otherwise stop at the iteration floor and the printed loss is
 * not an estimate of the loss).  OR it into `flags`. */
#define GP_MLL_SLQ_MIN_ITER(n) ((((int)(n)) & 0xff) << 8)
/* Solves Ktilde [u_0 .. u_M] = [y, z_1 .. z_M] with gp_cg_solve's method, then
 *   grad[0..d+2) = gradient of 1/(2M) sum_j u_j^T (dKtilde w_j) - 1/2 u_0^T (dKtilde u_0)
 *                  w.r.t. (l_1..l_d, a^2, sigma^2)  (Eq. approx; host),
 *   grad_X       = the same w.r.t. X (device N x d, optional),
 *   mll          = 1/2 log|Ktilde| + 1/2 y^T u_0 + N/2 log 2 pi  (host, NaN when no
 *                  log-determinant was requested or it cannot be estimated),
 *   U            = the solutions (device N x (M+1), optional).
 *   Z  device, M x N (row j = probe j): Rademacher / Gaussian probes, or the
 *      standard normals z~ with GP_MLL_PRECOND_PROBES
 *   E  device, M x rank standard normals (GP_MLL_PRECOND_PROBES only)
 *   1 <= M <= 31, d <= 32.  Synchronises the stream. */
GPK_API size_t gp_mll_workspace_size(const gp_hyp_t* hyp, int64_t N, int M, int rank, const gp_cg_opts_t* opts);
GPK_API int gp_mll_and_grad(gp_ctx* ctx, const gp_hyp_t* hyp, const float* X, const float* y, int64_t N,
                            const float* Z, int M, const float* E, const gp_precond_t* precond,
                            const gp_cg_opts_t* opts, int flags, double* mll, double* grad, float* grad_X,
                            float* U, gp_cg_stats_t* stats, void* stream);

/* ---- serving with continuous batching (predictive mean, Sec. 2.1) ----------- *
 * A server owns one device arena (allocated once by gp_server_create, never
 * grown) and a fixed number of request slots, each with its own CUDA stream.
 * An engine thread admits queued requests in arrival order whenever a slot is
 * free and the request's exact footprint (gp_server_request_bytes) fits in the
 * arena's free space, then advances every admitted request one phase at a time
 * without blocking: upload -> pivoted-Cholesky preconditioner -> one stable-CG
 * iteration per phase (Alg. 2, Eq. woodbury) -> true-residual checks ->
 * predictive mean mu* = K(X*, X) v with v = Ktilde^{-1} y (the posterior mean
 * of Sec. 2.1, a rectangular kernel MVM) -> download.  Requests arriving while
 * others run are admitted as slots and memory free up, and the phases of all
 * admitted requests overlap on the device.  A request's arithmetic does not
 * depend on what else is in flight: its result is the same alone and in a mix.
 */
typedef struct {
    size_t arena_bytes;  /* device memory for all admitted requests (> 0)         */
    int max_slots;       /* requests in flight at once, 1..64                      */
    int rank;            /* pivoted-Cholesky rank per request, 0..512 (0: none)     */
    int precision;       /* MVM precision inside CG: GP_PREC_* (and GP_MVM_* flags) */
    int mean_precision;  /* precision of the predictive-mean MVM                    */
    double tol;          /* CG relative-residual tolerance                          */
    int max_iter;        /* CG iteration limit (bounds the re-orthogonalisation store) */
    int restarts;        /* FP32 true-residual checks, 0..16                        */
    int reorth;          /* GP_REORTH_*                                             */
    int refine_precision; /* 0 = off; else the MVM flags CG switches to once every
                            recursive relative residual is <= refine_resid (> 0), or at
                            the first true-residual check (0): gp_cg_opts_t's fields */
    double refine_resid;
    int64_t large_n;     /* requests with N >= large_n plan their kernels for all but
                            large_reserve SMs, which stay free for the kernels of
                            smaller requests (a large request's MVM otherwise holds
                            every SM for milliseconds at a time); large_reserve = 0:
                            every request uses all SMs.  A request's launch plans
                            depend on its own N only, so its result is still the same
                            alone and in a mix.                                      */
    int large_reserve;
} gp_server_opts_t;

typedef struct {
    int status;          /* GP_OK, GP_ERR_NOT_CONVERGED (mean still written), ...   */
    int iters;           /* CG iterations                                           */
    int restarts;        /* true-residual checks taken                              */
    double rel_resid;    /* final ||Ktilde v - y|| / ||y|| (FP32 check MVM)         */
    double t_submit_ms;  /* host clock, ms since gp_server_create                   */
    double t_admit_ms;
    double t_done_ms;    /* engine saw the download complete                        */
    size_t bytes;        /* the request's arena footprint                           */
} gp_request_stats_t;

typedef struct {
    uint64_t submitted, completed;
    size_t arena_bytes;   /* budget                                                */
    size_t peak_bytes;    /* largest arena use seen (never above arena_bytes)      */
    size_t in_use_bytes;
    int max_inflight;     /* most requests admitted at once                        */
    int64_t launches;     /* kernels launched for requests                         */
} gp_server_stats_t;

typedef struct gp_server gp_server;

/* Exact arena footprint of one request (0 for invalid arguments). */
GPK_API size_t gp_server_request_bytes(const gp_server_opts_t* opts, const gp_hyp_t* hyp, int64_t N, int64_t n_test);
/* Allocates the arena and the slots' streams, starts the engine thread. */
GPK_API int gp_server_create(int device, const gp_server_opts_t* opts, gp_server** out);
/* Queues one request; returns at once.  Host buffers (X: N x d row-major,
 * y: N, X_test: n_test x d row-major, mean_out: n_test) are owned by the caller
 * and must stay valid until gp_server_wait returns for this id; page-locked
 * buffers make the copies asynchronous.  hyp->lengthscale is copied.
 * GP_ERR_WORKSPACE if the footprint exceeds the whole arena (never admissible),
 * GP_ERR_INVALID for bad arguments or a stopped server. */
GPK_API int gp_server_submit(gp_server* srv, const gp_hyp_t* hyp, const float* X, int64_t N, const float* y,
                             const float* X_test, int64_t n_test, float* mean_out, uint64_t* id_out);
/* Blocks until request `id` completes (timeout_s < 0: no limit) and returns
 * its status (GP_ERR_TIMEOUT when the host wait ran out, the request is then
 * still pending and may be waited for again).  Each id is reported once. */
GPK_API int gp_server_wait(gp_server* srv, uint64_t id, double timeout_s, gp_request_stats_t* stats);
GPK_API int gp_server_stats(gp_server* srv, gp_server_stats_t* out);
/* Finishes every queued and admitted request, stops the engine, frees all. */
GPK_API void gp_server_destroy(gp_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* GPK_H */
