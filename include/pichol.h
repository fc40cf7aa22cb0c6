/*
 * pichol.h -- C ABI of the GB300 (sm_103a) piCholesky cross-validation library.
 *
 * Method: Kuang, Gittens, Hamid, "Cholesky Factor Interpolation for Efficient
 * Approximate Cross-Validation" (arXiv 1404.0466).  For k-fold cross-validation
 * of multi-output ridge regression over a grid of q regularisation values, the
 * library factors H_f + lambda_s I exactly at g sampled lambdas only
 * (Algorithm 1: the exact factors), fits a degree-r polynomial in lambda to every
 * entry of the lower Cholesky factor (Algorithm 1: the fit), and scores the hold-out
 * error at all q lambdas through triangular solves with the interpolated
 * factor (Sec. 3.2 and the last paragraph of Sec. 3.3).
 *
 * Around that path: exact-Cholesky CV with the same kernels (the `Chol`
 * comparator of Sec. 6.2), the multi-level range search MChol (Sec. 6.2) that
 * can narrow the grid before piCholesky, PINRMSE (the sampled hold-out errors
 * interpolated directly, the paper's supplementary comparator), a warm start
 * of the fit across folds (the future work of Sec. 7), the derivative of the
 * hold-out error in log(lambda), and batches of independent problems.
 *
 * Conventions shared by every call:
 *  - Pointers are DEVICE pointers owned by the caller unless marked "host".
 *  - Matrices are row-major.  X is n x d, Y is n x c, both of the mode's input
 *    type (double in PICHOL_MODE_FP64, float in PICHOL_MODE_MIXED).
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Every compute call only enqueues work on that stream and returns; nothing
 *    synchronises except pichol_get_info and pichol_destroy.
 *  - Argument errors are returned immediately and enqueue nothing.  Errors met
 *    on the device (a non-positive pivot, a bounded wait that ran out) are
 *    latched in a status word in the workspace: the first one wins, later
 *    kernels keep running on safe values, and pichol_get_info reports it.  No
 *    call traps, asserts, aborts or prints.
 *  - The library allocates no device memory.  The caller provides one
 *    workspace buffer of pichol_workspace_size() bytes (256-byte aligned) that
 *    must stay valid, and must not be used by anyone else, while work enqueued
 *    by this context is in flight.
 *  - Calls on one context must not overlap on the GPU; use one context per
 *    concurrent problem.
 */
#ifndef PICHOL_H
#define PICHOL_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PICHOL_API __attribute__((visibility("default")))
#else
#define PICHOL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Version of this interface.  The minor number grows when calls or fields
 * are added (old callers keep working: new config fields take the place of
 * reserved ones, which must be zero); the major number grows when a call or
 * a layout changes incompatibly. */
#define PICHOL_VERSION_MAJOR 2
#define PICHOL_VERSION_MINOR 0

typedef enum {
    PICHOL_OK = 0,
    PICHOL_ERR_INVALID_ARG = 1,   /* bad size, null pointer, unsupported combination */
    PICHOL_ERR_NOT_SPD = 2,       /* H_f + lambda I had a non-positive pivot */
    PICHOL_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    PICHOL_ERR_WORKSPACE = 4,     /* workspace missing, too small or misaligned */
    PICHOL_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
    PICHOL_ERR_UNSUPPORTED = 6,   /* feature not available in this build / mode */
    PICHOL_ERR_STATE = 7          /* calls made out of order (e.g. fit before factor) */
} pichol_status;

typedef enum {
    /* every step in double precision */
    PICHOL_MODE_FP64 = 0,
    /* float inputs; Hessian on tensor cores (TF32, optionally split 3-term),
     * diagonal Cholesky blocks and the Vandermonde fit in double, panel and
     * trailing updates, coefficient storage and solves in float, hold-out
     * scoring with double accumulation, optional refinement with a
     * double-float residual */
    PICHOL_MODE_MIXED = 1
} pichol_mode;

typedef enum {
    /* phi_m(lambda) = (lambda / max_s lambda_s)^m: the monomials of
     * Algorithm 1, divided by the largest sample (same fitted polynomial) */
    PICHOL_BASIS_MONO = 0,
    /* phi_m(lambda) = T_m(u), u = 2 (ln lambda - ln min lambda_s) /
     * (ln max lambda_s - ln min lambda_s) - 1: Chebyshev polynomials (named in
     * Sec. 3.3 as the more stable basis) in log lambda */
    PICHOL_BASIS_CHEB_LOG = 1
} pichol_basis;

typedef struct {
    int64_t n;            /* rows of X and Y, >= k */
    int64_t d;            /* features, 1 .. 16384 */
    int64_t c;            /* outputs (right-hand sides), 1 .. 32 */
    int32_t k;            /* folds, 2 .. 64; fold f = rows [floor(f n/k), floor((f+1) n/k)) */
    int32_t g;            /* sampled lambdas, r < g <= min(q, 32) (Algorithm 1 needs g > r) */
    int32_t r;            /* polynomial degree, 0 .. 5 */
    int32_t q;            /* grid size, 1 .. 4096 */
    double lam_lo;        /* grid: lambda_t = s * lam_lo * (lam_hi/lam_lo)^(t/(q-1)) */
    double lam_hi;        /*   with s = tr(X^T X)/d if scale_by_trace else 1; 0 < lo <= hi, hi finite */
    int32_t scale_by_trace;
    int32_t basis;        /* pichol_basis */
    int32_t mode;         /* pichol_mode */
    int32_t refine_steps; /* mixed mode: refinement steps after each solve (0..4) */
    int32_t gram_passes;  /* mixed mode: 1 = plain TF32 products, 3 = split TF32 (hi*hi + hi*lo + lo*hi) */
    int32_t exact_batch;  /* lambdas factored per batch by pichol_eval_holdout_exact (0 = all q) */
    int32_t refine_target;/* mixed mode, which system each refinement step takes its residual from:
                             PICHOL_REFINE_INTERPOLATED (default): B - L~ (L~^T W), in double-float,
                             so the result stays the interpolated solution of Algorithm 1;
                             PICHOL_REFINE_EXACT: B - (H_f + lambda I) W from two tensor-core
                             products (split TF32), so the interpolated factor acts as a
                             preconditioner and the result moves toward exact CV (not in the paper) */
    int32_t warm_samples; /* 0, or g' with 2 <= g' <= min(g, 8): warm start across folds (the paper's future
                             work, Sec. 7).  Fold 0 is fitted from its g sampled factors; every other
                             fold f factors only g' lambdas, at grid indices round(i (q-1)/(g'-1)),
                             and takes Theta_f = Theta_0 + V'^+ (T'_f - V' Theta_0), V' = the first
                             min(g', r+1) basis functions at those lambdas (the basis normalised by
                             the g samples); its other coefficient planes are fold 0's */
    int32_t refine_residual; /* mixed mode with refine_target PICHOL_REFINE_INTERPOLATED, how the residual
                             B - L~ (L~^T W) is formed:
                             PICHOL_RESIDUAL_TENSOR (default): both triangular products for every
                             lambda at once on the tensor cores, sum_m phi_m(lambda) Theta_m applied as
                             one product per coefficient plane (split TF32, compensated accumulation
                             every 128 rows of K);
                             PICHOL_RESIDUAL_DOUBLE_FLOAT: per lambda on the FP32 pipes in double-float
                             arithmetic (error-free products and TwoSum), an FP64-class residual */
    int32_t reserved[3];  /* must be zero */
} pichol_config;

enum { PICHOL_REFINE_INTERPOLATED = 0, PICHOL_REFINE_EXACT = 1 };
enum { PICHOL_RESIDUAL_TENSOR = 0, PICHOL_RESIDUAL_DOUBLE_FLOAT = 1 };

/* First device error, as latched by the kernels. */
typedef struct {
    pichol_status code;   /* PICHOL_OK if none */
    int32_t fold;         /* fold of the failing factorisation, -1 if n/a */
    int32_t index;        /* sample (or grid index in exact mode), -1 if n/a */
    int64_t pivot;        /* row of the non-positive pivot, -1 if n/a */
    int32_t unusable;     /* count of (fold, lambda) pairs whose interpolated
                             diagonal was <= 1e3 eps max|diag| (scored +inf) */
} pichol_info;

typedef struct pichol_ctx pichol_ctx;

/* Fills *cfg with defaults: lam_lo = 1e-3, lam_hi = 1e1, scale_by_trace = 1,
 * basis MONO, mode FP64, refine_steps 0, gram_passes 3, exact_batch 0,
 * refine_target PICHOL_REFINE_INTERPOLATED, warm_samples 0, refine_residual
 * PICHOL_RESIDUAL_TENSOR; the sizes are left zero.
 * refine_target PICHOL_REFINE_EXACT needs mode MIXED (else
 * PICHOL_ERR_UNSUPPORTED from pichol_create). */
PICHOL_API void pichol_config_default(pichol_config* cfg);

/* Validates cfg and creates a context (host memory only).  *out is NULL on
 * error.  Every value out of the ranges documented in pichol_config returns
 * PICHOL_ERR_INVALID_ARG. */
PICHOL_API pichol_status pichol_create(const pichol_config* cfg, pichol_ctx** out);

/* Bytes of device workspace the context needs. */
PICHOL_API pichol_status pichol_workspace_size(const pichol_ctx* ctx, size_t* bytes);

/* Attaches the caller's workspace (device pointer, >= pichol_workspace_size
 * bytes, 256-byte aligned).  Contents need not be initialised: the call zeroes
 * the status word with a blocking cudaMemset on the current device.  The first
 * call also creates, on the current device, the context's one internal stream
 * (at the highest stream priority) and four events (factorisation look-ahead,
 * see pichol_factor_samples); pichol_destroy frees them. */
PICHOL_API pichol_status pichol_set_workspace(pichol_ctx* ctx, void* workspace, size_t bytes);

/*
 * Call 1 of the path: normal-equation blocks (Sec. 3.1, Eq. 2: H = X^T X, g = X^T y).
 * For every fold j: G_j = X_j^T X_j (X_j = rows of fold j), Bv_j = X_j^T Y_j,
 * yy_j = ||Y_j||_F^2; then tau = tr(sum_j G_j)/d, the default lambda grid
 * lambda_t = s lam_lo (lam_hi/lam_lo)^(t/(q-1)) (s = tau if scale_by_trace
 * else 1), the default samples lambda_{idx_s}, idx_s = round(s (q-1)/(g-1))
 * (Sec. 6.3: samples taken from the grid), and the training right-hand sides
 * B_f = sum_{j != f} Bv_j.
 *   X, Y         : device, row-major, n x d and n x c, double (FP64 mode) or
 *                  float (mixed mode); only read during this call's kernels
 *   fold_offsets : HOST, k+1 int64 row offsets, fold f = rows
 *                  [fold_offsets[f], fold_offsets[f+1]); offsets[0] = 0,
 *                  offsets[k] = n, every fold at least one row (else
 *                  PICHOL_ERR_INVALID_ARG, nothing enqueued).  NULL: the
 *                  contiguous split fold f = rows [floor(f n/k), floor((f+1) n/k))
 *                  (Sec. 1 leaves the split to the user).  Read during the call.
 * A grid that is not finite and positive, or sampled lambdas that give a
 * rank-deficient V, latch PICHOL_ERR_INVALID_ARG on the device (e.g. a NaN in
 * X with scale_by_trace set).
 */
PICHOL_API pichol_status pichol_hessian(pichol_ctx* ctx, const void* X, const void* Y, const int64_t* fold_offsets,
                                        void* stream);

/*
 * Call 2 (Algorithm 1, the exact factors at the samples): exact Cholesky factors L_{f,s} of
 * H_f + lambda_s I for every fold f and each of the g sampled lambdas, with
 * H_f = sum_{j != f} G_j.  Blocked right-looking factorisation, all k*g
 * problems per launch.  A non-positive pivot latches PICHOL_ERR_NOT_SPD.
 *   lam_s : HOST, g doubles, or NULL.  The sampled lambdas (absolute values,
 *           finite and > 0, else PICHOL_ERR_INVALID_ARG and nothing enqueued);
 *           NULL takes the grid samples of pichol_hessian.  They also set the
 *           observation matrix V[s][m] = phi_m(lambda_s) of pichol_fit and the
 *           basis normalisation (largest sample for MONO, log range of the
 *           samples for CHEB_LOG).  Values that make V rank deficient latch
 *           PICHOL_ERR_INVALID_ARG.  With warm_samples the folds f > 0 factor
 *           the warm-start lambdas of the default grid (see pichol_config).
 *           Passed to the device as kernel arguments, so the call stays
 *           capturable.
 * Part of each trailing update runs on the context's internal stream, forked
 * from `stream` by an event and joined back before the call's last enqueued
 * work, so the call orders like a single-stream call and can be captured.
 */
PICHOL_API pichol_status pichol_factor_samples(pichol_ctx* ctx, const double* lam_s, void* stream);

/*
 * Call 3 (Algorithm 1, the fit): V[s][m] = phi_m(lambda_s) (g x (r+1)),
 * P = V^+ by QR in double precision, and Theta_f = P T_f for every fold, where
 * row s of T_f holds the entries of L_{f,s}.  The coefficients stay in the
 * workspace for pichol_eval_holdout.
 *   theta_out : device or NULL.  When given, also receives a copy of every
 *               fold's coefficients in the library's tile-major layout, of the
 *               mode's type: k * T * (r+1) * 64 * 64 values, T = nt (nt+1)/2,
 *               nt = ceil(d/64); value [f][i(i+1)/2 + j][m][a][b] is entry
 *               (64 i + a, 64 j + b) of Theta_{f,m} (lower tiles j <= i;
 *               entries above the diagonal and past d are zero, except on
 *               the padded diagonal, whose factors are 1: there the fit of
 *               that constant, 1 in Theta_{f,0} and 0 in the others up to
 *               the rounding of V^+).
 *               pichol_export_theta gives one fold as a dense matrix instead.
 */
PICHOL_API pichol_status pichol_fit(pichol_ctx* ctx, void* theta_out, void* stream);

/*
 * Call 4 (Sec. 3.3 evaluation, Sec. 3.2 solves, Sec. 3.1 selection): for every
 * fold f and each of the q evaluation lambdas lambda_t, W_{f,t} = (L~ L~^T)^{-1} B_f with
 * L~ = sum_m phi_m(lambda_t) Theta_{f,m} built tile by tile on the device, then
 * E[f*q + t] = ||Y_f - X_f W_{f,t}||_F^2 / (n_f c) evaluated as
 * (yy_f - 2 <Bv_f, W> + <W, G_f W>) / (n_f c), and *t_star = the smallest t
 * minimising mean_f E[f*q + t] over finite values (-1 if none).
 *   lam_t   : HOST, q doubles, or NULL.  The evaluation lambdas (absolute,
 *             finite and > 0, any order; else PICHOL_ERR_INVALID_ARG and
 *             nothing enqueued): the interpolant of Algorithm 1 is evaluated at
 *             any lambda without a new factorisation (Sec. 3.3).  NULL takes
 *             the grid of pichol_hessian.  pichol_get_lambdas then returns these
 *             values.  Passed as kernel arguments (capturable).
 *   E_out   : device, k*q doubles
 *   t_star  : device, one int32
 *   W_out   : device or NULL; k*q*d*c values of the mode's type, [f][t][d][c]
 * A (fold, lambda) whose interpolated diagonal is unusable scores +inf.
 */
PICHOL_API pichol_status pichol_eval_holdout(pichol_ctx* ctx, const double* lam_t, double* E_out, int32_t* t_star,
                                             void* W_out, void* stream);

/*
 * Exact-Cholesky cross-validation (the `Chol` comparator of Sec. 6.2) with the
 * same kernels: factor H_f + lambda_t I at every evaluation lambda, solve,
 * score.  Needs only pichol_hessian before it.  Same arguments and outputs as
 * pichol_eval_holdout (lam_t: host q doubles or NULL for the grid).
 */
PICHOL_API pichol_status pichol_eval_holdout_exact(pichol_ctx* ctx, const double* lam_t, double* E_out,
                                                   int32_t* t_star, void* W_out, void* stream);

/*
 * Hold-out error and its derivative in log(lambda) at any lambda = exp(log_lam),
 * through the interpolated factor (after pichol_fit): with
 * L~ = sum_m phi_m(lambda) Theta_m and L~' = sum_m phi_m'(lambda) Theta_m
 * (Sec. 3.3's polynomials and their derivative), A = L~ L~^T,
 * W = A^{-1} B_f, V = G_f W - Bv_f, U = A^{-1} V:
 *   E_out[f]  = ||Y_f - X_f W||^2 / (n_f c)
 *   dE_out[f] = lambda * (-2 / (n_f c)) (<L~'^T U, L~^T W> + <L~^T U, L~'^T W>)
 * which is d E_f / d log(lambda) (chain rule on dW = -A^{-1} dA W; not in the
 * paper).  E_out, dE_out: device, k doubles each.  The diagonal of L~ at this
 * lambda is not checked for usability.  log_lam must be finite (|.| <= 700).
 */
PICHOL_API pichol_status pichol_holdout_grad(pichol_ctx* ctx, double log_lam, double* E_out, double* dE_out,
                                             void* stream);

/*
 * PINRMSE, the comparator of the paper's supplementary material: Algorithm 1
 * with the g x D target matrix T replaced by the g x 1 vector t_f of exact
 * hold-out errors at the sampled lambdas.  After pichol_factor_samples, the
 * sampled factors L_{f,s} are used for exact solves and scores, t_f[s] =
 * ||Y_f - X_f W||^2 / (n_f c) with W = (L_{f,s} L_{f,s}^T)^{-1} B_f; then
 * theta_f = V^+ t_f (the same V^+ as pichol_fit) and
 *   E_out[f*q + t] = sum_m phi_m(lambda_t) theta_f[m]
 * at the current evaluation lambdas (pichol_get_lambdas),
 * and *t_star = the smallest t minimising mean_f E_out[f*q + t] over finite
 * values (-1 if none).  A fold with an unusable sampled factor scores +inf at
 * every t (pichol_info.unusable counts such samples).  E_out: device, k*q
 * doubles; t_star: device, one int32.  The sampled factors and the fit stay
 * valid; the solution buffer of pichol_eval_holdout is reused.  Not with
 * warm_samples (PICHOL_ERR_UNSUPPORTED): the folds then have no common samples.
 */
PICHOL_API pichol_status pichol_eval_pinrmse(pichol_ctx* ctx, double* E_out, int32_t* t_star, void* stream);

/*
 * Multi-level narrowing of the lambda range (MChol, Sec. 6.2), then a new grid
 * on the final range.  Starting from (c, s), each level
 *   (a) evaluates the exact hold-out error of every fold at the three lambdas
 *       tau 10^(c-s), tau 10^c, tau 10^(c+s) (exact Cholesky, as in
 *       pichol_eval_holdout_exact), tau = tr(X^T X)/d if scale_by_trace else 1;
 *   (b) takes lambda_opt = the first of the three with the smallest finite mean
 *       over folds (c is kept if none is finite);
 *   (c) sets c <- log10(lambda_opt / tau), s <- s / 2;
 * and the levels repeat until s <= s_min (at least one level; their number is
 * pichol_mchol_levels(s, s_min)).  Afterwards the grid, the samples and V^+
 * are set up again as in pichol_hessian with lam_lo = 10^(c-s) and
 * lam_hi = 10^(c+s) from the final (c, s), so pichol_factor_samples,
 * pichol_fit and pichol_eval_holdout run piCholesky over that range (and
 * pichol_get_lambdas returns it).  Everything runs on the device; nothing
 * synchronises.
 *   c, s, s_min : |c| <= 300; 0 < s <= 300; 0 < s_min <= 300; at most 64 levels
 *   trace_out   : device or NULL; levels x 8 doubles, one row per level:
 *                 the three lambdas, their mean hold-out errors, then c and s
 *                 after the level's update
 * Needs pichol_hessian before it and q >= 3 (else PICHOL_ERR_UNSUPPORTED); the
 * sampled factors and the fit are invalidated (the factor buffer is reused).
 * Errors of the exact factorisations latch as in pichol_eval_holdout_exact
 * (index = 0..2, the position of the lambda in its level); a final range that
 * is not finite latches PICHOL_ERR_INVALID_ARG.
 */
PICHOL_API pichol_status pichol_mchol(pichol_ctx* ctx, double c, double s, double s_min, double* trace_out,
                                      void* stream);

/* Number of levels pichol_mchol runs for (s, s_min): the smallest n >= 1 with
 * s / 2^n <= s_min.  PICHOL_ERR_INVALID_ARG for values out of the ranges of
 * pichol_mchol or more than 64 levels. */
PICHOL_API pichol_status pichol_mchol_levels(double s, double s_min, int32_t* levels);

/* Device copy of the q evaluation lambdas: those of the last
 * pichol_eval_holdout / pichol_eval_holdout_exact call, or the grid of
 * pichol_hessian (MChol's final range after pichol_mchol) before any. */
PICHOL_API pichol_status pichol_get_lambdas(pichol_ctx* ctx, double* lam_out, void* stream);

/* Inspection (for tests): dense double copies of internal results.
 *   factor : L_{f,s} (d x d, upper triangle zero) after pichol_factor_samples; with
 *            warm_samples = g' the folds f > 0 hold s < g' only (the warm-start lambdas)
 *   theta  : Theta_{f,m} for m = 0..r, (r+1) x d x d (upper triangles zero) after pichol_fit
 *   hessian: H_f (d x d, lower triangle mirrored) and B_f (d x c) after pichol_hessian
 * Outputs are device buffers of doubles.  PICHOL_ERR_INVALID_ARG for a null
 * pointer or f, s out of range; PICHOL_ERR_STATE before the step that makes
 * the result (also after a later call that invalidated it, see pichol_mchol
 * and pichol_eval_holdout_exact). */
PICHOL_API pichol_status pichol_export_factor(pichol_ctx* ctx, int32_t f, int32_t s, double* L_out, void* stream);
PICHOL_API pichol_status pichol_export_theta(pichol_ctx* ctx, int32_t f, double* theta_out, void* stream);
PICHOL_API pichol_status pichol_export_hessian(pichol_ctx* ctx, int32_t f, double* H_out, double* B_out, void* stream);

/* Synchronises `stream` and reports the first latched device error. */
PICHOL_API pichol_status pichol_get_info(pichol_ctx* ctx, pichol_info* info, void* stream);

/* Clears the latched device status (enqueued on `stream`). */
PICHOL_API pichol_status pichol_clear_status(pichol_ctx* ctx, void* stream);

/* Exercises the error path of the bounded copy waits: enqueues one wait, with
 * a limit of `cycles` SM clocks (1 .. 2^34), on an mbarrier that nothing
 * completes.  It runs out, latches PICHOL_ERR_TIMEOUT (fold, index and pivot
 * -1) and returns; nothing faults or hangs, and after pichol_clear_status the
 * context is usable as before.  For tests of failure detection. */
PICHOL_API pichol_status pichol_check_timeout(pichol_ctx* ctx, int64_t cycles, void* stream);

/* Exercises the error path of the wavefront solve's waits on blocks solved by
 * other CTAs of the same launch (the few-system interpolated solves, Sec. 3.2
 * and 3.3): enqueues one forward pass over the hold-out gradient's buffers, one
 * system per fold, whose first tile row is never scheduled.  Every CTA waits for
 * block 0 until `cycles` SM clocks (1 .. 2^34) run out, latches
 * PICHOL_ERR_TIMEOUT (fold, the waiting tile row >= 1, pivot 0: the block it
 * waited for), publishes its block as failed and returns; nothing faults or
 * hangs, no result of the context is written, and after pichol_clear_status the
 * context is usable as before.  PICHOL_ERR_UNSUPPORTED where the wavefront does
 * not apply (FP64 mode, r > 3, c > 32, d <= 64, more folds than SMs);
 * PICHOL_ERR_WORKSPACE without a workspace.  For tests of failure detection. */
PICHOL_API pichol_status pichol_check_wave_timeout(pichol_ctx* ctx, int64_t cycles, void* stream);

/* Accuracy check of the double-precision 1/sqrt used for the pivots of the
 * diagonal tiles (a float seed refined by one third-order step, see chol.cu):
 * writes to *max_rel_err (device, one double) the largest relative difference
 * from the library's 1.0 / sqrt(p) over n values p = 2^u, u uniform in
 * [-110, 110) from a splitmix64 stream started at `seed`.  1 <= n <= 2^32.
 * Needs no context.  For tests. */
PICHOL_API pichol_status pichol_check_rsqrt(int64_t n, uint64_t seed, double* max_rel_err, void* stream);

/* Sustained fused multiply-add rate of the current device's FP32 (fp64 = 0) or
 * FP64 (fp64 = 1) pipes, for roofline denominators: 8 CTAs of 256 threads per
 * SM, each thread running eight independent FMA chains of `iters` steps
 * (1 .. 2^24), on the legacy default stream, timed with CUDA events (the
 * second of two runs).  *tflops (host) = 2 x FMAs / seconds / 1e12.  Needs no
 * context; synchronises the device. */
PICHOL_API pichol_status pichol_probe_fma(int32_t fp64, int64_t iters, double* tflops);

/* Issue rate of the tensor cores for tcgen05.mma kind::tf32 with M = 128,
 * K = 8 and N = n_cols (64, 128 or 256), for the roofline of the tcgen05
 * contractions: one CTA per SM issues `iters` MMAs (1 .. 2^22) back to back
 * on zeroed shared-memory operands into tensor memory, on the legacy default
 * stream, timed with CUDA events (the second of two runs).  *tflops (host) =
 * 2 x 128 x n_cols x 8 x MMAs / seconds / 1e12.  PICHOL_ERR_TIMEOUT if the
 * bounded completion wait ran out.  Needs no context; synchronises the device
 * and allocates (and frees) one int of device memory. */
PICHOL_API pichol_status pichol_probe_mma(int32_t n_cols, int64_t iters, double* tflops);

/* Number of kernel launches this context has enqueued since creation. */
PICHOL_API int64_t pichol_launch_count(const pichol_ctx* ctx);

/* Stage timing (for benchmarks): with max_launches > 0 the context records a
 * pair of CUDA events around each of its next max_launches kernel launches on
 * the launching stream; 0 turns timing off and frees the events.  Creating
 * events is the only resource this takes.  The records are external event
 * records, so calls captured into a CUDA graph while timing is on put them in
 * the graph and every replay re-records them (pichol_stage_times then reports
 * the last replay); such a graph must be destroyed before timing is turned
 * off or set again, which frees the events it refers to. */
PICHOL_API pichol_status pichol_set_timing(pichol_ctx* ctx, int32_t max_launches);

/* Synchronises `stream`, then sums the recorded launch durations per stage
 * into ms[i] and counts them in launches[i] for the first n_stages stages, and
 * restarts recording.  Stages, in order: 0 Gram blocks, 1 X^T Y, 2 set-up
 * (grid, V^+), 3 factor input, 4 diagonal-tile Cholesky, 5 panel solve,
 * 6 trailing update, 7 polynomial fit, 8 diagonal inverses, 9 interpolated
 * solve, 10 refinement residual, 11 hold-out score, 12 selection, 13 other.
 * Returns PICHOL_ERR_STATE if timing is off and PICHOL_ERR_WORKSPACE if more
 * launches happened than events were reserved (the sums then cover the first
 * max_launches launches only). */
PICHOL_API pichol_status pichol_stage_times(pichol_ctx* ctx, double* ms, int64_t* launches, int32_t n_stages,
                                            void* stream);

/*
 * Launch shapes of the factorisation and the evaluation that a tuner may change.  Each changes
 * how the work is split into CTAs and scheduled, never the order of any
 * element's arithmetic, so every result is bit-identical under every tuning,
 * except update_engine, which changes the rounding of the trailing updates
 * (fp32-class either way).
 *   update_strip   : output tiles per CTA in the bulk trailing updates, 1..8 (default 4)
 *   diag_threads   : threads of a diagonal-tile CTA, 256 or 512 (default 512)
 *   diag_exclusive : 1 lets each diagonal-tile CTA hold a whole SM (a shared
 *                    memory request no update CTA fits beside) when the k g
 *                    problems fit on half the SMs; 0 never (default 1; batches
 *                    set 0 for their problems)
 *   update_engine  : mixed mode: 1 runs the bulk trailing updates on the CUDA
 *                    cores (fp32 FMA, default), 0 on the tensor cores (split
 *                    TF32: hi*hi + hi*lo + lo*hi).  Measured on GB300 the tensor
 *                    cores are no faster here (each update is bound by reading
 *                    and writing the trailing tiles) and their factors carry
 *                    about ten times the rounding error, which moves hold-out
 *                    errors of ill-conditioned problems past 1e-4, so they are
 *                    an option, not the default
 *   solve_engine   : mixed mode, interpolated solves: 0 on the tensor cores (all
 *                    lambdas of a fold at once, one split-TF32 product per
 *                    coefficient plane: sum_m Theta_m (phi_m Z); each plane is
 *                    read once per block of 64 columns), 1 on the CUDA cores
 *                    (the factor evaluated per lambda in shared memory,
 *                    (sum_m phi_m Theta_m) Z; the planes are read once per two
 *                    lambdas), 2 (default) the tensor cores when one fold's
 *                    coefficient planes exceed 64 MiB (half of the L2 cache),
 *                    else the CUDA cores.  The two round differently (same
 *                    fp32 accuracy class); the choice is per context
 *   eval_overlap   : mixed mode with refinement: 1 splits the lambdas of
 *                    pichol_eval_holdout in two halves, the second run on the
 *                    internal stream from the end of the first half's solve,
 *                    so that its solve overlaps the first half's residual
 *                    passes; 0 runs them as one (default 0)
 * pichol_set_tuning returns PICHOL_ERR_INVALID_ARG for values out of range or
 * nonzero reserved fields and then changes nothing.
 */
typedef struct {
    int32_t update_strip;
    int32_t diag_threads;
    int32_t diag_exclusive;
    int32_t eval_overlap;
    int32_t update_engine;
    int32_t solve_engine;
    int32_t reserved[2];
} pichol_tuning;
PICHOL_API pichol_status pichol_get_tuning(const pichol_ctx* ctx, pichol_tuning* t);
PICHOL_API pichol_status pichol_set_tuning(pichol_ctx* ctx, const pichol_tuning* t);

/*
 * Checkpoint and resume.  Every result of the path (normal-equation blocks,
 * grid, sampled factors, coefficients, status word) lives in the caller's
 * workspace, and nothing in it points into device memory, so a checkpoint is
 * the workspace's bytes plus which results they hold.
 *   pichol_get_state : *state = the results the workspace holds, as bits
 *                      PICHOL_STATE_HESSIAN (pichol_hessian),
 *                      PICHOL_STATE_FACTORS (pichol_factor_samples),
 *                      PICHOL_STATE_FIT (pichol_fit).  Host only.
 *   pichol_resume    : declares that the attached workspace now holds those
 *                      results, its pichol_workspace_size bytes having been
 *                      copied from a context of an identical configuration;
 *                      later calls continue from there (e.g. pichol_eval_holdout
 *                      after PICHOL_STATE_FIT).  Host only; the library cannot
 *                      check the bytes.
 * PICHOL_ERR_INVALID_ARG for a null pointer, unknown bits, or factors or fit
 * without the Hessian; PICHOL_ERR_WORKSPACE from pichol_resume without a
 * workspace.
 */
enum { PICHOL_STATE_HESSIAN = 1, PICHOL_STATE_FACTORS = 2, PICHOL_STATE_FIT = 4 };
PICHOL_API pichol_status pichol_get_state(const pichol_ctx* ctx, int32_t* state);
PICHOL_API pichol_status pichol_resume(pichol_ctx* ctx, int32_t state);

/* Frees the host-side context (and its timing events).  The workspace stays
 * the caller's. */
PICHOL_API void pichol_destroy(pichol_ctx* ctx);

/*
 * Fold right-hand sides with no allocation at all.  The paper has no
 * counterpart to this call; it exists for callers that cannot allocate device
 * memory (a plug-in inside a framework that owns the whole device through its
 * own memory pool, a real-time path that cannot afford cudaMalloc's implicit
 * synchronisation, code that is given only its inputs and outputs).  It
 * computes, for the k contiguous folds f = rows [floor(f n/k), floor((f+1) n/k)),
 *   Bv_out[j] = X_j^T Y_j          and   B_out[f] = sum_{j != f} Bv_out[j],
 * both k x d x c row-major in the mode's type (double for PICHOL_MODE_FP64,
 * float for PICHOL_MODE_MIXED), the same values pichol_hessian forms for B_f.
 * X (n x d) and Y (n x c) are device pointers; the outputs are caller-owned
 * device buffers.  Requires 2 <= k <= 64, n >= k, d >= 1, 1 <= c <= 64.
 *
 * Scratch: the partial sums use a fixed array in the library's device memory
 * (8 MiB, i.e. 2^20 doubles, held by every GPU that loads the library until
 * the process exits); k * 16 * ceil(d/64)*64 * c must not exceed 2^20, else
 * PICHOL_ERR_WORKSPACE is returned and nothing is enqueued.  The array is
 * shared by every call on a device and keeps the last call's contents; every
 * partial a call reads is first written by the same call, so nothing needs to
 * start at zero.  Calls that overlap on the GPU (on different streams, or from
 * several threads) race on the array and give wrong results: serialise them.
 * The first call on each device looks up the array's device address with
 * cudaGetSymbolAddress (with that device current), and looks it up again after
 * the device's context changed (a device reset); make that first call, and the
 * first after a reset, before any stream capture.  The call never calls cudaMalloc, cudaFree or any other
 * allocating routine.  Errors: PICHOL_ERR_INVALID_ARG for bad arguments,
 * PICHOL_ERR_CUDA if a CUDA call fails.
 */
PICHOL_API pichol_status pichol_fold_rhs_noalloc(int32_t mode, const void* X, const void* Y, int64_t n, int64_t d,
                                                 int64_t c, int32_t k, void* Bv_out, void* B_out, void* stream);

/*
 * Batches of independent problems of uneven size (the data-parallel structure
 * of Sec. 1: folds, lambdas and separate problems are independent units).
 * pichol_batch_create makes one context per entry of cfgs[0..nprob) (host
 * memory only); all of them live in one caller-owned workspace of
 * pichol_batch_workspace_size bytes.  pichol_batch_run enqueues, for every
 * problem i, pichol_hessian(X[i], Y[i]), pichol_factor_samples, pichol_fit and
 * pichol_eval_holdout(E_out[i], t_star + i): X, Y, E_out are HOST arrays of
 * DEVICE pointers (problem i's X is n_i x d_i, Y n_i x c_i, E_out[i] k_i * q_i
 * doubles), t_star a device array of nprob int32.  The work forks from
 * `stream` onto `nstreams` internal streams (created on the first run on the
 * current device, most expensive problems first, round robin) and joins back,
 * so everything is ordered after earlier work on `stream` and later work on
 * `stream` waits for it; the whole call can be captured into a CUDA graph
 * (after one uncaptured run, which creates the streams and kernel attributes).
 * The first failing call's status is returned: no later problem is enqueued,
 * and the internal streams are still joined back to `stream`.  Device errors
 * are reported per problem by pichol_batch_get_info.
 * Errors: PICHOL_ERR_INVALID_ARG for a null pointer, nprob outside 1..4096,
 * nstreams outside 1..64, i outside 0..nprob-1, or any config that
 * pichol_create rejects (batch_create then returns that config's status);
 * PICHOL_ERR_WORKSPACE from batch_run before batch_set_workspace, and from
 * batch_set_workspace for a buffer that is too small or not 256-byte aligned.
 * pichol_batch_destroy frees the host side; the workspace stays the caller's.
 */
typedef struct pichol_batch pichol_batch;
PICHOL_API pichol_status pichol_batch_create(const pichol_config* cfgs, int32_t nprob, int32_t nstreams,
                                             pichol_batch** out);
PICHOL_API pichol_status pichol_batch_workspace_size(const pichol_batch* b, size_t* bytes);
PICHOL_API pichol_status pichol_batch_set_workspace(pichol_batch* b, void* workspace, size_t bytes);
/* Changes the number of internal streams (1..64) used by later runs. */
PICHOL_API pichol_status pichol_batch_set_streams(pichol_batch* b, int32_t nstreams);
/* Applies pichol_set_tuning to every problem (all or none on invalid values). */
PICHOL_API pichol_status pichol_batch_set_tuning(pichol_batch* b, const pichol_tuning* t);
PICHOL_API pichol_status pichol_batch_run(pichol_batch* b, const void* const* X, const void* const* Y,
                                          double* const* E_out, int32_t* t_star, void* stream);
PICHOL_API pichol_status pichol_batch_get_info(pichol_batch* b, int32_t i, pichol_info* info, void* stream);
PICHOL_API int64_t pichol_batch_launch_count(const pichol_batch* b);
/* Stage timing of every problem's context (pichol_set_timing on each, same
 * meaning of max_launches), and problem i's per-stage sums
 * (pichol_stage_times).  Each context records on the stream its problem runs
 * on, so with more than one internal stream the recorded durations include
 * time shared with other problems' kernels; time with one stream to get
 * per-kernel durations. */
PICHOL_API pichol_status pichol_batch_set_timing(pichol_batch* b, int32_t max_launches);
PICHOL_API pichol_status pichol_batch_stage_times(pichol_batch* b, int32_t i, double* ms, int64_t* launches,
                                                  int32_t n_stages, void* stream);
PICHOL_API void pichol_batch_destroy(pichol_batch* b);

/* Short text for a status code (static storage). */
PICHOL_API const char* pichol_status_string(pichol_status s);

/* Bounds checking in the debug build (libpichol_debug.so, compiled with
 * -DPICHOL_DEBUG): every workspace section is followed by a 4 KB guard band
 * filled with 0xA5 when the workspace is attached, and pichol_get_info checks
 * the bands first; a changed byte latches PICHOL_ERR_WORKSPACE with index =
 * the band's number and pivot = the byte within it (a kernel wrote past a
 * section's end).  pichol_debug_guards writes up to `capacity` band offsets
 * (bytes from the workspace start) to `offsets` (host) and their number to
 * *count (0 in the regular build).  pichol_debug_build returns 1 in the debug
 * build, else 0. */
PICHOL_API pichol_status pichol_debug_guards(const pichol_ctx* ctx, int64_t* offsets, int32_t capacity,
                                             int32_t* count);
PICHOL_API int32_t pichol_debug_build(void);

/* The interface version the library was built with: 100 * major + minor
 * (compare with PICHOL_VERSION_MAJOR / _MINOR of the header in use). */
PICHOL_API int32_t pichol_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PICHOL_H */
