/*
 * kqr.h -- C ABI of the GB300 (sm_103a) kernel quantile regression library.
 *
 * The library solves the kernel quantile regression problem of Deng, Li and
 * Zhang, "Scalable Kernel Quantile Regression: A Preconditioned Augmented
 * Lagrangian Method" (arxiv 2510.07929):
 *
 *   min_{beta, f in H_k}  sum_i rho_tau(y_i - beta - f(x_i)) + lambda/2 ||f||^2   (eq. (1.1))
 *
 * through its dual (eq. (1.3)):
 *
 *   max_alpha  -alpha^T K alpha / (2 lambda) + y^T alpha,
 *   alpha in [tau - 1, tau]^n,  1^T alpha = 0,
 *
 * with the two-phase method of the paper: inexact ADMM (Alg. 1), then the
 * semismooth Newton augmented Lagrangian method (Alg. 2 and Alg. 3) whose
 * Newton systems (eq. (3.1)) are solved by CG preconditioned with a low-rank
 * RPCholesky factor applied through the Woodbury identity (Lemma 1).  The
 * fitted function is f(x) = beta + (1/lambda) sum_j alpha_j k(x_j, x)
 * (representer form, Sec. 1).
 *
 * Every step of the solve runs in CUDA kernels on the current device.  Kernel
 * matrix entries are formed in tiles inside the Gram-product kernels; the
 * FP32 products inside CG stream a stored copy of K's upper triangle instead
 * when it fits in device memory (options.gram_store), since each entry is
 * then formed once rather than once per product.
 *
 * Conventions for every function below:
 *   - Host pointers ("host") are read or written before the call returns; the
 *     caller owns them.  Device pointers ("device") must point to memory of the
 *     handle's device; the caller owns them.
 *   - Matrices are row-major.  X is n x p; V and U are n x m (m right-hand sides).
 *   - Errors are returned as kqr_status, never thrown; kqr_last_error(h) gives a
 *     one-line description of the last failure on that handle.
 *   - A handle is used by one host thread at a time.  It owns a CUDA stream, or
 *     uses the one given by kqr_set_stream.  The *_dev functions enqueue work
 *     on the given stream (NULL = the handle's stream) and return without
 *     synchronising, except where stated.
 */
#ifndef KQR_H
#define KQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum kqr_status {
  KQR_OK = 0,
  KQR_INVALID_ARG = 1,        /* bad size, pointer, tau, lambda, gamma or non-finite data */
  KQR_OOM = 2,                /* device allocation failed */
  KQR_CUDA_ERROR = 3,         /* a CUDA call or kernel launch failed */
  KQR_NOT_CONVERGED = 4,      /* iteration cap reached; outputs hold the last iterate */
  KQR_BREAKDOWN = 5,          /* CG curvature p^T A p <= 0 or NaN, or a factorisation failed */
  KQR_TIMEOUT = 6,            /* host wall-clock limit (options.time_limit_s) reached */
  KQR_DEVICE_WAIT_TIMEOUT = 7 /* a kernel gave up a bounded wait on a copy and returned */
} kqr_status;

/* Kernel functions of Sec. 1 (text after eq. (1.1)). */
typedef enum kqr_kernel {
  KQR_RBF = 0,       /* k(x, x') = exp(-gamma ||x - x'||_2^2) */
  KQR_LAPLACIAN = 1  /* k(x, x') = exp(-gamma ||x - x'||_1)   */
} kqr_kernel;

/* Arithmetic of a Gram product.
 * KQR_PREC_HIGH: entries and sums accurate to about 1e-13 relative (FP64 class;
 *   Laplacian: exact fixed-point L1 distances plus double-float exp and sums on
 *   the FP32/INT32 pipes; RBF with p <= 40: the same fixed-point scheme on the
 *   squared differences; RBF with p > 40: FP64 arithmetic).  Used for gradients
 *   and KKT residuals, and for CG where FP32 cannot resolve K (options.cg_high).
 * KQR_PREC_FP32: FP32 entries and FP32 partial sums, about 1e-6 relative per
 *   entry.  Used inside CG.  RBF: the cross term x_i . x_j runs on the tcgen05
 *   tensor cores as three TF32 products (hi.hi + hi.lo + lo.hi of a TF32 split
 *   of X), unless options.rbf_tensor_cores = 0 (FP32 CUDA cores).
 * KQR_PREC_TF32: RBF only; one TF32 product on the tensor cores (about 2^-11
 *   relative error in the exponent's cross term).
 * KQR_PREC_BF16: RBF only; coordinates rounded to bf16 and one bf16 product on
 *   the tensor cores (about 2^-8 relative error in the exponent's cross term). */
typedef enum kqr_precision {
  KQR_PREC_HIGH = 0,
  KQR_PREC_FP32 = 1,
  KQR_PREC_TF32 = 2,
  KQR_PREC_BF16 = 3
} kqr_precision;

/* Preconditioner for the linear systems (2.1) and (3.1).
 * KQR_PRECOND_PAPER: P = F F^T + lambda sigma 1 1^T + L (eq. (3.2)).
 * KQR_PRECOND_NYSTROM_DIAG: as PAPER with L replaced by L + max(diag(K - F F^T), nu),
 *   the RPCholesky residual diagonal floored at nu = 0.1 mean(diag(K - F F^T))
 *   (still diagonal plus low rank, so Lemma 1 applies unchanged; the floor keeps
 *   L^{-1} bounded at the pivots, whose residual is 0; not in the paper).
 * KQR_PRECOND_NONE: plain CG (the paper's NALM-KQR ablation, Sec. 4.1). */
typedef enum kqr_precond {
  KQR_PRECOND_NYSTROM_DIAG = 0,
  KQR_PRECOND_PAPER = 1,
  KQR_PRECOND_NONE = 2
} kqr_precond;

/* Algorithm constants.  The paper leaves them open; kqr_default_options fills
 * in the library's readings. */
typedef struct kqr_options {
  /* preconditioner set-up (Sec. 3) */
  int32_t rank0;                 /* initial RPCholesky rank r0; 0 = ceil(sqrt(n)) */
  int32_t adaptive_rank;         /* 1: pick r from the spectrum of F0^T F0 (Sec. 3); 0: r = r0 */
  double xi;                     /* rank threshold: smallest r with xi * lambda_1 >= lambda_r (default 1e-10) */
  uint64_t seed;                 /* pivot stream seed used when pivot_uniforms is NULL */
  const double* pivot_uniforms;  /* host, optional: one uniform [0,1) per pivot step, length >= r0 */
  kqr_precond precond;
  /* Phase I, inexact ADMM (Alg. 1) */
  double sigma0;                 /* initial penalty sigma */
  double gamma_admm;             /* step length in (0, (1 + sqrt 5) / 2) */
  double admm_tol;               /* stop when max(eta_kkt, eta_gap) <= admm_tol (Sec. 4: 1e-3) */
  double admm_cg_rtol;           /* inexactness eps_k = admm_cg_rtol ||b_k|| / (k + 1)^1.5 (summable) */
  int32_t admm_maxit;            /* ... or after admm_maxit iterations (Sec. 4: 100) */
  int32_t balance_every;         /* residual balancing period for sigma */
  double balance_ratio;          /* rebalance when eta_p / eta_d leaves [1/ratio, ratio] */
  double balance_factor;         /* multiply or divide sigma by this */
  /* Phase II, SSN-ALM (Alg. 2, Alg. 3) */
  int32_t alm_maxit;             /* Sec. 4: 1000 */
  double sigma_alm_scale;        /* Phase II sigma_0 = max(final Phase I sigma, sigma_alm_scale / lambda) */
  double sigma_factor;           /* sigma *= sigma_factor when eta_d fails to halve */
  double sigma_max;
  double eta_bar, iota, mu, r_ls, tau1, tau2;   /* Alg. 3 constants */
  int32_t ssn_maxit;             /* Newton steps per ALM subproblem */
  int32_t ls_maxit;              /* backtracking steps per Newton step */
  int32_t pcg_maxit;             /* CG iterations per linear system */
  double core_reuse_rtol;        /* Newton steps keep the Woodbury core while the preconditioner's
                                    diagonal moved by at most this relative amount (0: always rebuild) */
  double time_limit_s;           /* host wall-clock limit per solve; <= 0: none */
  int32_t phase1_only;           /* 1: stop after Phase I (for tests of Alg. 1) */
  int32_t symmetric_gram;        /* 1: single-vector products (FP32, and FP64-class Laplacian) form each off-diagonal tile once and
                                    use it for both K_IJ v_J and K_IJ^T v_I (n(n+1)/2 entries; summation
                                    order not fixed); 0: every entry formed (deterministic) */
  int32_t rbf_tensor_cores;      /* 1: RBF FP32 products on tcgen05 (three TF32 terms); 0: FP32 CUDA cores */
  int32_t cg_tf32;               /* RBF only, 1: CG products in TF32 on tcgen05 (one term), each linear solve
                                    iteratively refined against FP32 residuals to the same tolerance */
  int32_t verbose;               /* 1: one line per outer iteration on stderr */
  int32_t cg_high;               /* CG products: 0 FP32; 1 FP64-class; 2 (default) FP64-class when K is
                                    numerically low-rank at FP32 resolution: from the start when
                                    RPCholesky's mean residual diagonal is below 2^-24 n, and from the
                                    first CG run that stops at a rounding-level curvature on */
  int32_t gram_store;            /* FP32 single-vector products (the CG products) from a stored K:
                                    0 never (entries formed on the fly in tiles every product);
                                    1 always (kqr_create fills the packed upper triangle of K as
                                    128 x 128 FP32 tiles, (T (T + 1) / 2) * 64 KB with T = ceil(n / 128),
                                    and returns KQR_OOM if it does not fit); 2 (default) when those
                                    bytes are at most half the free device memory at kqr_create,
                                    except for RBF kernels with p <= 32 (tensor cores and symmetric
                                    tiles on) once they exceed 64 MB: their on-the-fly tiles are
                                    faster than streaming a stored K */
} kqr_options;

/* Counters and final residuals of a solve (Sec. 4 definitions). */
typedef struct kqr_info {
  int32_t phase1_iters, phase2_iters, newton_steps, pcg_iters;
  int32_t matvecs_fp32, matvecs_high;  /* Gram products by arithmetic, each counted once per RHS */
  int32_t matvecs_low;                 /* TF32 products (options.cg_tf32) */
  int32_t rank;                        /* preconditioner rank r */
  int32_t core_builds;                 /* Woodbury cores built (the rest of the systems reused one) */
  int32_t cg_truncations;              /* CG runs stopped at a non-positive (rounding) curvature */
  double eta_p, eta_d, eta_c, eta_kkt, eta_gap, obj_p, obj_d;
  double sigma_final;
  double seconds;                      /* wall-clock of the solve */
  int32_t gram_stored;                 /* 1: the FP32 products streamed a stored K (options.gram_store) */
  int32_t cg_high_used;                /* 1: the CG products were FP64-class at the end (options.cg_high) */
} kqr_info;

typedef struct kqr_handle kqr_handle;

/* Fills *o with the library's default constants. */
void kqr_default_options(kqr_options* o);

/* Routes the library's device allocations through alloc/free (for example a
 * framework's caching allocator); NULL restores cudaMalloc/cudaFree.  Affects
 * handles created afterwards.  alloc returns NULL on failure. */
void kqr_set_allocator(void* (*alloc)(size_t bytes, void* ctx), void (*free_fn)(void* ptr, void* ctx), void* ctx);

/* Creates a problem on the current device: copies X (host, n x p, row-major)
 * and y (host, n) to the device, prepares the tile layouts of X for the Gram
 * kernels, and builds the RPCholesky factor F (n x r) of K (Sec. 3), which
 * depends only on (X, kernel, gamma) and is reused by every later solve.
 * n >= 2, 1 <= p <= 64, gamma > 0, X and y finite.  opts may be NULL
 * (defaults).  On success *out owns all device memory of the problem. */
kqr_status kqr_create(const double* X, const double* y, int64_t n, int64_t p, kqr_kernel kind,
                      double gamma, const kqr_options* opts, kqr_handle** out);

/* Solves the dual (1.3) for (tau, lambda) to max(eta_kkt, eta_gap) <= tol
 * (Sec. 4 stopping rule), Phase I then Phase II.  0 < tau < 1, lambda > 0,
 * tol > 0.  alpha (host, n) receives the dual solution (also theta of the
 * representer form); *beta the intercept; *kkt = eta_kkt, evaluated with the
 * FP64-class Gram product.  info (nullable) receives counters and residuals.
 * Returns KQR_NOT_CONVERGED (outputs filled with the last iterate) when the
 * iteration caps are reached.  Synchronises. */
kqr_status kqr_solve(kqr_handle* h, double tau, double lambda, double tol,
                     double* alpha, double* beta, double* kkt, kqr_info* info);

/* Solves the dual (1.3) for m pairs (taus[c], lambdas[c]), 1 <= m <= 4096, on
 * the handle's problem, to the tolerance of kqr_solve: a grid of quantile
 * levels and regularisation weights on one data set (Sec. 4.1 fits paths of
 * 50 lambdas).  Every pair runs the two-phase method of kqr_solve on its own
 * state; the pairs' Gram products are taken together, up to 8 right-hand
 * sides per kernel launch (FP32, or FP64-class where options.cg_high says so,
 * and always for gradients and Sec. 4 residuals), so one pass over the kernel
 * matrix serves several pairs; a pair that has converged drops out of the
 * shared products.  alpha (host, n x m column-major: pair c at alpha + c n),
 * beta, kkt and status (host, m each) receive each pair's result as kqr_solve
 * would (status[c] is that pair's kqr_status); info (nullable, m entries) its
 * counters.  Returns KQR_OK when every pair returned KQR_OK, KQR_NOT_CONVERGED
 * or KQR_TIMEOUT (see status), else the first failure.  Uses one host thread
 * per pair; allocates device memory; synchronises. */
kqr_status kqr_solve_grid(kqr_handle* h, int64_t m, const double* taus, const double* lambdas, double tol,
                          double* alpha, double* beta, double* kkt, int32_t* status, kqr_info* info);

/* kqr_solve_grid on B problems (single-problem handles hs[0..B), each created
 * with its own X, y, kernel and gamma; sizes may differ) with the same m pairs,
 * `workers` problems at a time (<= 0: 4), each problem's products on its own
 * stream.  alpha (host): problem b's n_b x m column-major block at
 * alpha + m (n_0 + ... + n_{b-1}); beta, kkt, status (host): B x m, row b for
 * problem b.  Synchronises. */
kqr_status kqr_solve_grid_batch(kqr_handle* const* hs, int64_t B, int64_t m, const double* taus, const double* lambdas,
                                double tol, int32_t workers, double* alpha, double* beta, double* kkt,
                                int32_t* status);

/* After kqr_solve: copies the last iterate's consensus variable v and
 * multiplier z of (1.4)-(1.5) to host arrays of length n (either may be NULL). */
kqr_status kqr_get_state(kqr_handle* h, double* v, double* z);

/* U = K V for host V (n x m, row-major) and host U (n x m); 1 <= m <= 8.
 * Copies V in and U out inside the call.  Synchronises. */
kqr_status kqr_kmatvec(kqr_handle* h, const double* V, double* U, int64_t m, kqr_precision prec);

/* As kqr_kmatvec with device V and U (n x m, row-major, double).  The Gram
 * product of Sec. 1 / Sec. 3, entries formed on the fly in tiles. */
kqr_status kqr_kmatvec_dev(kqr_handle* h, const double* V, double* U, int64_t m, kqr_precision prec,
                           void* stream);

/* FP32 Gram product U = K V (as kqr_kmatvec_dev with KQR_PREC_FP32) that
 * allocates no device memory during the call.  The paper has no counterpart.
 *
 * Some callers cannot allocate device memory at the moment they need a
 * product: a process whose device memory is fully reserved up front by a pool
 * (a further cudaMalloc fails or fragments it), code running inside another
 * framework's allocator or memory-pressure callback (re-entering an allocator
 * there can deadlock), or a latency-critical loop that must not pay the
 * implicit device synchronisation of cudaMalloc and cudaFree.  This entry
 * point keeps its scratch (the FP32 copy of V and per-split partial sums) in a
 * fixed 32 MiB static device array instead; every GPU that loads the library
 * holds that array until the process exits.  The handle itself (kqr_create)
 * is set up beforehand as usual.
 *
 * V and U are device arrays (n x m, row-major, double), 1 <= m <= 8; the
 * handle's device must be the current device.  A problem whose scratch need,
 * ceil256(ldn * M * 4) + splits * ldn * M * 4 bytes (ldn = n rounded up to 128,
 * M = m rounded up to 1, 2, 4 or 8, splits = the column splits of the launch),
 * exceeds 32 MiB is rejected with KQR_INVALID_ARG and a message giving the
 * sizes (about n <= 500000 rows at m = 8).  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  The address is cached per device and CUDA
 * context: after cudaDeviceReset the next call looks it up again (handles
 * created before the reset are invalid anyway).  Every call shares the one
 * array and each call overwrites it completely, so two calls that overlap on
 * the GPU (on different streams, or different handles of the same device) race
 * and both results are undefined: serialise them.  Enqueues on `stream` (NULL:
 * the handle's) and returns without synchronising, so it cannot report a Gram
 * kernel that gave up a bounded wait on a tile copy (U is then incomplete):
 * after synchronising that stream, call kqr_check_device. */
kqr_status kqr_kmatvec_fp32_noalloc_dev(kqr_handle* h, const double* V, double* U, int64_t m, void* stream);

/* Reads the handle's device error word, which a kernel sets when it gives up
 * a bounded wait on a tile copy or an MMA (kqr_status
 * KQR_DEVICE_WAIT_TIMEOUT); the results of that call are then incomplete.
 * The *_dev calls and kqr_kmatvec_fp32_noalloc_dev return without
 * synchronising, so they cannot report this themselves: synchronise the stream
 * they were enqueued on, then call this.  Returns KQR_DEVICE_WAIT_TIMEOUT (and
 * clears the word) if a kernel gave up since the last check, else KQR_OK.
 * Synchronises the device (blocking copy).  No counterpart in the paper. */
kqr_status kqr_check_device(kqr_handle* h);

/* Exercises the timeout path of the kernels' bounded waits: one CTA waits on
 * a barrier that nothing completes, gives up after max_polls polls (1 ..
 * 2^20) and records the timeout in the device error word, exactly as a Gram
 * kernel does when a tile copy never lands; no copy or MMA is in flight.  A
 * following kqr_check_device returns KQR_DEVICE_WAIT_TIMEOUT.  Synchronises.
 * For tests of the error path; no counterpart in the paper. */
kqr_status kqr_test_bounded_wait(kqr_handle* h, uint32_t max_polls);

/* Projection, Jacobian and gradient of the ALM subproblem (eq. (2.3), Sec. 2.2,
 * eq. (3.1)), device vectors of length n:
 *   w = alpha + z / sigma, v = Pi_B(w), S_ii = 1 if tau - 1 < w_i < tau else 0,
 *   grad = Kalpha / lambda - y + beta + sigma 1^T alpha + sigma (w - v),
 *   Ldiag = lambda sigma (1 - S) + lambda eps.
 * Kalpha is K alpha (device).  Any output pointer may be NULL.  *grad_norm2
 * (host, nullable) receives ||grad||^2 (synchronises when non-NULL). */
kqr_status kqr_box_grad_dev(kqr_handle* h, const double* alpha, const double* z, const double* Kalpha,
                            double beta, double sigma, double tau, double lambda, double eps,
                            double* v, double* S, double* grad, double* Ldiag, double* grad_norm2,
                            void* stream);

/* Preconditioner apply of Lemma 1 with the handle's factor F:
 *   out = P^{-1} r,  P = F F^T + gam 1 1^T + diag(Ldiag)  (Ldiag > 0, gam > 0),
 * building the (r+1) x (r+1) core C + U^T L^{-1} U and its Cholesky factor
 * first.  Ldiag, r, out: device, length n.  This applies exactly the given
 * Ldiag (no residual-diagonal correction).  Synchronises. */
kqr_status kqr_precond_apply_dev(kqr_handle* h, const double* Ldiag, double gam, const double* r,
                                 double* out, void* stream);

/* Preconditioned CG (Sec. 3) for (K + gam 1 1^T + diag(Ldiag)) x = b with the
 * handle's preconditioner kind, FP32 Gram products, from x = 0, until the
 * recursive residual satisfies ||r|| <= tol or maxit iterations.  b, x device.
 * *iters (nullable) receives the iteration count.  Returns KQR_NOT_CONVERGED
 * (x holds the last iterate) when CG stopped before meeting tol: at maxit, or
 * at a non-positive curvature p^T A p <= 0 (FP32 rounding on a numerically
 * low-rank K; the message says which).  Synchronises. */
kqr_status kqr_pcg_dev(kqr_handle* h, const double* Ldiag, double gam, const double* b, double* x,
                       double tol, int32_t maxit, int32_t* iters, void* stream);

/* Relative KKT residuals and duality gap of Sec. 4 for host (alpha, v, beta, z)
 * with the FP64-class Gram product: out[0..6] = eta_p, eta_d, eta_c, eta_kkt,
 * eta_gap, obj_p, obj_d.  Synchronises. */
kqr_status kqr_kkt(kqr_handle* h, const double* alpha, const double* v, double beta, const double* z,
                   double tau, double lambda, double* out7);

/* The RPCholesky factor built by kqr_create: F (host, n x rank, column-major,
 * float), pivots (host, int64, rank0 entries: the first-pass pivot sequence),
 * *rank and *rank0.  Any pointer may be NULL. */
kqr_status kqr_get_factor(kqr_handle* h, float* F, int64_t* pivots, int32_t* rank, int32_t* rank0);

/* Rebuilds the RPCholesky factor of Sec. 3 from the device-resident X of the
 * handle (same kernel and gamma), with the pivot uniforms given (host,
 * nullable, length >= r0) or, if NULL, the splitmix64 stream of
 * options.seed.  Used to time the set-up on resident data.  Synchronises. */
kqr_status kqr_refactor(kqr_handle* h, const double* pivot_uniforms);

/* Instrumentation (no counterpart in the paper).  kqr_profile(h, 1) resets
 * and enables CUDA-event timing of the Gram tile kernels on the handle's
 * stream; kqr_profile(h, 0) disables it.  kqr_profile_read returns, for
 * kernel_id 0 (FP32 Gram tiles), 1 (FP64-class Gram tiles) or 2 (stored-K
 * product), the number of launches and their summed device time in
 * milliseconds since the last reset.
 * Reading synchronises the handle's stream. */
kqr_status kqr_profile(kqr_handle* h, int32_t enable);
kqr_status kqr_profile_read(kqr_handle* h, int32_t kernel_id, int64_t* launches, double* total_ms);

/* Held-out check loss of the last solve's fitted function and its gradient
 * (an extension; the paper has no counterpart).  RBF kernel only.  X (host,
 * n x p) must be the training inputs given to kqr_create; Xh (host, nh x p)
 * and yh (host, nh) are held-out points.  With f(x) = beta + (1/lambda)
 * sum_j alpha_j k(x_j, x) (Sec. 1), *loss = sum_h rho_tau(yh_h - f(xh_h)) and
 * the derivatives of that loss with respect to log gamma, log lambda and the
 * training inputs X (dX, host n x p row-major, nullable) are obtained by
 * implicit differentiation through the KKT conditions of Sec. 4 at the
 * solution, holding the elbow set {i : tau - 1 < alpha_i < tau} fixed (the
 * loss is differentiable where no point enters or leaves it and no held-out
 * residual is zero).  The Gram products are recomputed in tiles, FP64-class
 * throughout (the 1/lambda factors amplify product errors); the adjoint solves
 * run CG on the problem's preconditioner, whose core this call replaces.
 * Allocates device memory; synchronises. */
kqr_status kqr_heldout_grad(kqr_handle* h, const double* X, const double* Xh, const double* yh, int64_t nh,
                            double* loss, double* d_loggamma, double* d_loglambda, double* dX);

/* ---- batched multi-right-hand-side products ---------------------------------
 * B independent RBF problems of different sizes (rows offsets[b] .. offsets[b+1]-1
 * of X), each with its own gamma_b, and up to 64 right-hand sides per problem:
 * U_b = K_b V_b with K_b[i][j] = exp(-gamma_b ||x_i - x_j||^2) (Sec. 1).  Fitting a
 * grid of (tau, lambda) pairs on each data set needs products of the same K_b
 * with one vector per pair (the ADMM and Newton systems of Sec. 3), so one
 * pass over each Gram tile serves every pair.  Both contractions (X X^T and
 * K V) run on the tensor cores in TF32 with FP32 accumulation: each entry
 * of U carries a relative error of order 2^-10 of sum_j K_ij |V_jc|.
 *
 * Creates a handle for products only (the single-problem calls reject it;
 * kqr_set_stream, kqr_profile(_read) with kernel id 0, kqr_launch_count,
 * kqr_last_error and kqr_destroy apply).  X: host, offsets[B] x p row-major;
 * offsets: host, B + 1 entries, offsets[0] = 0, strictly increasing;
 * p in [1, 32]; gammas: host, B positive values; flags: 0, or
 * KQR_BATCH_P_IN_SMEM to stage each Gram tile through shared memory instead of
 * tensor memory (the same values; a layout choice kept for comparison).  The
 * handle owns device copies; the caller keeps its arrays.  Synchronises. */
#define KQR_BATCH_P_IN_SMEM 1
kqr_status kqr_batch_create(const double* X, const int64_t* offsets, int64_t B, int64_t p, const double* gammas,
                            int32_t flags, kqr_handle** out);

/* U = blockdiag(K_1 .. K_B) V for V (offsets[B] x m, row-major, rows ordered as
 * X) with m in [1, 64]; U has the same layout.  Host pointers; allocates
 * device staging buffers; synchronises; KQR_DEVICE_WAIT_TIMEOUT if the kernel
 * gave up waiting on a copy. */
kqr_status kqr_batch_kmatmul(kqr_handle* h, const double* V, double* U, int64_t m);

/* As kqr_batch_kmatmul with device pointers, enqueued on the handle's stream;
 * no allocation, no synchronisation.  Calls that overlap on the GPU share the
 * handle's staging copy of V and race. */
kqr_status kqr_batch_kmatmul_dev(kqr_handle* h, const double* V, double* U, int64_t m);

/* Makes the handle enqueue its work on the given cudaStream_t (NULL: its own). */
kqr_status kqr_set_stream(kqr_handle* h, void* stream);

int64_t kqr_n(const kqr_handle* h);
int64_t kqr_p(const kqr_handle* h);

/* Number of kernel launches the handle has issued since creation. */
int64_t kqr_launch_count(const kqr_handle* h);

const char* kqr_last_error(const kqr_handle* h);
const char* kqr_status_string(kqr_status s);

/* Frees every device buffer of the handle.  NULL is ignored. */
void kqr_destroy(kqr_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* KQR_H */
