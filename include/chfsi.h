/*
 * chfsi.h -- C ABI of the GB300 (sm_103a) Chebyshev-filtered subspace iteration library.
 *
 * The library solves sequences of correlated generalized Hermitian eigenproblems
 *     A^(l) x = lambda B^(l) x,   l = 1..N                              (Eq. 1, Section 1)
 * for the nev lowest eigenpairs of each problem, with Chebyshev-filtered subspace
 * iteration with locking (Algorithm 1, Section 3.1), after reduction to standard form
 * B = L L^H, Hs = L^{-1} A L^{-H}, y = L^H x (Section 3.2), each problem warm-started
 * from the Ritz vectors of the previous one (Section 3.2, stages 1-4).
 *
 * Conventions shared by every entry point
 *   - Complex numbers are interleaved complex128 (chfsi_z), matrices column-major with a
 *     leading dimension ld >= rows.  Only the LOWER triangles of A and B are read.
 *   - The caller owns every buffer it passes; the library never frees or keeps caller
 *     memory.  The context owns its device workspace (allocated by chfsi_create).
 *   - The solve entry points accept host or device pointers for A, B, V0, evals and
 *     evecs (the kind is detected per pointer; host data is staged through the
 *     context's workspace on the context's stream).  The step entry points take DEVICE
 *     pointers only.
 *   - Every function returns a status code (chfsi_status); on failure the message is
 *     available from chfsi_last_error(ctx).  No entry point aborts the process.
 *   - One context serves one host thread at a time; all work is queued on the
 *     context's CUDA stream and the solve entry points return after it has finished.
 *
 * Environment variables (read once per process; none is needed for normal use)
 *   CHFSI_OZ_KERNEL=mma            digit products on the mma.sync kernel instead of tcgen05
 *   CHFSI_OZ_GROUPS=0              one slice pair per stage in the tcgen05 kernel (default:
 *                                  slice groups sharing one A tile, blocks <= 96 columns)
 *   CHFSI_OZ_GROUP_MIN_STAGES=k    smallest TMA ring a slice group may leave (default 4)
 *   CHFSI_SLICE_MARGIN_BITS=b      safety margin of the filter's per-loop slice count
 *                                  (default 6 bits)
 */
#ifndef CHFSI_H
#define CHFSI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } chfsi_z;
typedef struct chfsi_ctx chfsi_ctx;

typedef enum {
  CHFSI_OK = 0,
  CHFSI_EINVAL = 1,    /* bad sizes (blk < nev, blk > n, n > n_max, ...), NULL, NaN input */
  CHFSI_ENOTPD = 2,    /* B (or a Gram matrix beyond repair) is not positive definite */
  CHFSI_ENOCONV = 3,   /* not converged within max_loops, or residual check failed (see solve) */
  CHFSI_ECUDA = 4,     /* a CUDA runtime call failed */
  CHFSI_ETIMEOUT = 5,  /* a bounded device-side wait expired (kernel returned early) */
  CHFSI_ENOMEM = 6     /* workspace allocation failed */
} chfsi_status;

/* Solver options.  Defaults (chfsi_default_opts) follow Table 3 of the paper for ChFSI:
 * polynomial degree 25, TOL 1e-10; lanczos-iter 10 (warm) / 40 (cold) within the
 * table's range "10 : 3 x blk". */
typedef struct {
  int32_t deg_min;          /* adaptive degree range (deg == 0 in a solve call) */
  int32_t deg_max;
  int32_t max_loops;        /* filter loops per problem before CHFSI_ENOCONV (default 50) */
  int32_t lanczos_k_warm;   /* Lanczos steps for the spectral upper bound, warm start */
  int32_t lanczos_k_cold;   /* ... cold start */
  int32_t reuse_factor;     /* 1: reuse L when B is bitwise equal to the previous B */
  int32_t precision;        /* 0 = FP64 throughout; 1 (default) = mixed: the filter products
                               as split-BF16 tensor-core digit products with an accuracy
                               chosen per loop, the other large products (reduction,
                               Rayleigh-Ritz, re-orthonormalisation, back-transform) as
                               digit products with FP64-level results, the small
                               eigensolver, residuals and small products in FP64 */
  int32_t slices_max;       /* most digit slices per operand in mixed mode (2..8, default 7) */
  uint64_t seed;            /* SplitMix64 seed of the Lanczos start vector / cold block */
  void* cuda_stream;        /* cudaStream_t to run on (cudaStreamLegacy for the legacy default
                               stream); NULL = a stream created and owned by the context */
} chfsi_opts;

/* Per-problem statistics (Table 4 of the paper reports loops and filtered vectors). */
typedef struct {
  int32_t loops;             /* filter loops (outer repeat of Algorithm 1) */
  int32_t filtered_vectors;  /* sum over loops of the active block width */
  int32_t converged;         /* locked pairs returned */
  int32_t accept_rounds;     /* times the locking threshold was tightened */
  int64_t matvecs;           /* column products Hs*y (filter + Rayleigh-Ritz + Lanczos) */
  int64_t filter_matvecs;    /* column products Hs*y inside the Chebyshev filter only */
  int64_t launches;          /* CUDA kernels launched by the library for this problem */
  int64_t filter_matvecs_fp64; /* filter column products done with FP64 arithmetic */
  double tensor_flops;       /* tensor-core flops of the split-BF16 filter products, counted on the
                                unpadded operands: 2 * pairs * (2n) * m * (2n) per product */
  double max_resid;          /* max_i ||A x_i - lambda_i B x_i|| / (||A||_est ||x_i||) */
  double lanczos_upper;      /* spectral upper bound b used by the filter */
  double t_reduce_ms, t_lanczos_ms, t_filter_ms, t_qr_ms, t_rr_ms, t_resid_ms, t_total_ms;
  double t_filter_gemm_ms;   /* device time of the filter's product kernels alone */
  double t_small_ms;         /* Cholesky QR factorisations of the Gram matrices (within t_qr) */
  double t_eig_ms;           /* Rayleigh-Ritz eigensolver (within t_rr) */
  int64_t filter_products;   /* split-BF16 product launches of the filter */
  double filter_slice_bytes; /* bytes of the Hs digit slices those launches stream (S * Mp * Kp * 2
                                each): the launches' minimum DRAM traffic */
} chfsi_stats;

/* ---------------------------------------------------------------- context */
void chfsi_default_opts(chfsi_opts* opts);

/* Create a context able to solve problems with n <= n_max and blk <= blk_max; allocates
 * all device workspace: six n_max x n_max complex matrices, bf16 digit-slice buffers (two
 * of 8 slices of the 2 n_max x 2 n_max real embedding, one of 8 slices of up to n_max
 * columns, or the Gauss form's three parts), split-K partials and about 12 n_max
 * max(blk_max, 128) complex entries: about 2.3 GB at n_max = 2600, blk_max = 130, and 26.5
 * GB (measured) at n_max = 9300, blk_max = 320.
 * opts may be NULL (defaults).  Errors: EINVAL, ENOMEM, ECUDA. */
int chfsi_create(chfsi_ctx** out, int64_t n_max, int32_t blk_max, const chfsi_opts* opts);
void chfsi_destroy(chfsi_ctx* ctx);
const char* chfsi_last_error(const chfsi_ctx* ctx);
/* Drop the carried Ritz vectors and the cached factor of B: the next solve starts cold. */
int chfsi_reset_warm_state(chfsi_ctx* ctx);

/* Checkpoint and resume of the warm state (Section 3.2, stage 3: the eigenvectors of problem
 * l seed problem l + 1), so that a sequence can continue in another context or process.
 * The state is the last solve's blk Ritz vectors in x-coordinates (B-orthonormal, n x blk)
 * and their Ritz values; the factor of B is not part of it (the next solve factors its B).
 * chfsi_get_state: *n and *blk receive the state's sizes (both 0 when the context has no
 * warm state: after a cold context, chfsi_reset_warm_state or a solve that did not converge);
 * X (n x blk complex, column-major, ld n; host or device) and lam (blk doubles, host) are
 * filled when not NULL (query the sizes first with both NULL).  The call synchronises the
 * context's stream.
 * chfsi_set_state: installs n x blk vectors X (ld ldx >= n; host or device) and blk values
 * lam (host, ascending) as the warm state; the next solve with this n and blk starts from
 * them.  Copies before returning (the caller may free X and lam).  n = 0 clears the state.
 * Errors: EINVAL (NULL context, n > n_max, blk > blk_max, blk < 1 or NULL arrays with
 * n > 0, ldx < n), ECUDA. */
int chfsi_get_state(chfsi_ctx* ctx, int64_t* n, int32_t* blk, chfsi_z* X, double* lam);
int chfsi_set_state(chfsi_ctx* ctx, int64_t n, int32_t blk, const chfsi_z* X, int64_t ldx,
                    const double* lam);

/* ---------------------------------------------------------------- solves */
/* Solve one problem of the sequence (Algorithm 1 with the reduction of Section 3.2).
 *   A, B   n x n (lower triangles read), leading dimensions lda, ldb.
 *   V0     optional n x blk start block (ld n) used when the context has no warm state;
 *          NULL = SplitMix64 complex Gaussian block.  Ignored when warm state exists.
 *   deg    > 0: fixed filter degree; 0: adaptive per-vector degree in [deg_min, deg_max].
 *   tol    residual tolerance (paper: 1e-10).
 *   evals  nev ascending eigenvalues (host or device, double).
 *   evecs  n x nev B-orthonormal eigenvectors, ld n (host or device), may be NULL.
 *   st     optional statistics (host).
 * The Ritz vectors (all blk of them, in x-coordinates) and the bounds are kept in the
 * context as the warm start of the next call.
 * Errors: EINVAL, ENOTPD, ECUDA, ETIMEOUT, and ENOCONV in two cases: max_loops reached
 *         with fewer than nev pairs locked (evals of the locked prefix, the rest NaN;
 *         st->max_resid NaN), or all nev pairs locked but their generalized residual
 *         st->max_resid still above tol after three tightenings of the locking threshold
 *         (all nev evals and evecs returned).  In both cases the context's warm state is
 *         updated from the returned vectors and the context stays usable. */
int chfsi_solve_next(chfsi_ctx* ctx, int64_t n, const chfsi_z* A, int64_t lda,
                     const chfsi_z* B, int64_t ldb, const chfsi_z* V0, int32_t nev,
                     int32_t blk, int32_t deg, double tol, double* evals, chfsi_z* evecs,
                     chfsi_stats* st);

/* Solve N problems in order, problem l warm-started from problem l-1 (Section 3.2,
 * stages 1-4).  A[l], B[l]: pointers to the l-th matrices (ld = ld).  V0 as above for
 * the first problem.  evals: N x nev (row l at evals + l*nev).  evecs: N pointers to
 * n x nev outputs, or NULL.  st: N entries or NULL.  Starts from the context's warm
 * state if it has one (call chfsi_reset_warm_state first for a cold first problem). */
int chfsi_solve_sequence(chfsi_ctx* ctx, int32_t N, int64_t n, const chfsi_z* const* A,
                         const chfsi_z* const* B, int64_t ld, const chfsi_z* V0,
                         int32_t nev, int32_t blk, int32_t deg, double tol, double* evals,
                         chfsi_z* const* evecs, chfsi_stats* st);

/* ---------------------------------------------------------------- steps (device pointers)
 * Each step of the hot path is also exposed on its own, for testing and for callers that
 * assemble their own loop.  All run on the context's stream and synchronise it before
 * returning.  Workspace limits of the context apply (n <= n_max, m <= blk_max). */

/* B = L L^H (Section 3.2).  L receives the lower factor, its strict upper part zeroed.
 * Errors: ENOTPD (message names the failing pivot), EINVAL. */
int chfsi_cholesky(chfsi_ctx* ctx, int64_t n, const chfsi_z* B, int64_t ldb, chfsi_z* L,
                   int64_t ldl);

/* Hs = L^{-1} A L^{-H}, exactly Hermitian in full storage (Section 3.2).  L lower.  With
 * precision 1 the two products run as 8-slice split-BF16 tensor-core products (error about
 * 1e-17 relative to the operands' row and column scales, below the FP64 GEMM bound); with
 * precision 0 in FP64. */
int chfsi_reduce(chfsi_ctx* ctx, int64_t n, const chfsi_z* A, int64_t lda, const chfsi_z* L,
                 int64_t ldl, chfsi_z* Hs, int64_t ldh);

/* k-step Lanczos with full re-orthogonalisation on the Hermitian H (full storage),
 * starting from v0 (device, n) or, if v0 is NULL, from the SplitMix64 start vector of
 * the context seed (Algorithm 1, first step).  upper = max eig(T_k) + |beta_k|,
 * theta_min = min eig(T_k), theta_max = max eig(T_k) (host doubles).  With precision 1 the
 * products H v use FP32 multiply-adds on the FP64 data (relative error ~1e-7, ample for a
 * spectral bound); with precision 0 FP64. */
int chfsi_lanczos(chfsi_ctx* ctx, int64_t n, const chfsi_z* H, int64_t ldh, int32_t k,
                  const chfsi_z* v0, double* upper, double* theta_min, double* theta_max);

/* Chebyshev filter in place on the n x m block Y (Algorithm 1, filtering step): column i
 * becomes T_{d_i}((H - c)/e) y_i / T_{d_i}((a0 - c)/e), e = (b-a)/2, c = (b+a)/2, by the
 * scaled three-term recurrence.  degrees: HOST array of m non-negative degrees. */
int chfsi_filter(chfsi_ctx* ctx, int64_t n, int32_t m, const chfsi_z* H, int64_t ldh,
                 chfsi_z* Y, int64_t ldy, const int32_t* degrees, double a0, double a,
                 double b);

/* The same filter with split-BF16 tensor-core products (mixed-precision filter): every
 * product Hs*Y is computed from `slices` 7-bit digit slices of each FP64 operand (power-of-
 * two scales per row of H and per column of Y), exact in FP32 per 960-term chunk, combined
 * in double-float; relative error about 2^(-7 slices) of the operands' scales.
 * slices in [1, 8].  H must be Hermitian (full storage). */
int chfsi_filter_split(chfsi_ctx* ctx, int64_t n, int32_t m, const chfsi_z* H, int64_t ldh,
                       chfsi_z* Y, int64_t ldy, const int32_t* degrees, double a0, double a,
                       double b, int32_t slices);

/* Re-orthonormalisation (Algorithm 1): Y <- orthonormal basis of (I - YL YL^H) Y, by two
 * passes of classical Gram-Schmidt against the k locked columns YL (may be 0), then with
 * precision 1 FP32 Cholesky QR steps and FP64 first-order Loewdin steps chosen from the
 * Gram matrix on the device (orthonormal to about 1e-15), with precision 0 Cholesky QR
 * twice (three times, shifted, on breakdown).  In place, n x m. */
int chfsi_orthonormalize(chfsi_ctx* ctx, int64_t n, int32_t m, chfsi_z* Y, int64_t ldy,
                         int32_t k, const chfsi_z* YL, int64_t ldyl);

/* Rayleigh-Ritz (Algorithm 1): G = Y^H H Y, G w = theta w (ascending), Y <- Y W,
 * W_out <- H Y (the new Ritz vectors' products).  theta: device, m doubles.  H Hermitian;
 * with precision 1 the product H Y uses 7-slice split-BF16 products (FP64-level). */
int chfsi_rayleigh_ritz(chfsi_ctx* ctx, int64_t n, int32_t m, const chfsi_z* H, int64_t ldh,
                        chfsi_z* Y, int64_t ldy, chfsi_z* HY, int64_t ldhy, double* theta);

/* Residual norms of the locking test (Algorithm 1): r_i = ||HY_i - theta_i Y_i|| / ||Y_i||.
 * theta, r: device, m doubles. */
int chfsi_residuals(chfsi_ctx* ctx, int64_t n, int32_t m, const chfsi_z* HY, int64_t ldhy,
                    const chfsi_z* Y, int64_t ldy, const double* theta, double* r);

/* Deviation angles between eigenvectors of adjacent problems of a sequence (Section 2.2:
 * the scalar products <x_i^(l) x_j^(l+1)> of eigenvectors of neighbouring pencils and the
 * angles theta_i^(l) plotted in Fig. 1).  With a common overlap matrix B (lower triangle
 * read) the paper's product c^(l)H L L^H c^(l+1) is the B-inner product, so
 * M = X_prev^H B X_cur (k x k).  Previous vector i is associated with current vector
 * assoc[i] by repeatedly taking the largest |M_ij| over unassigned rows and columns (ties:
 * smallest row, then smallest column), the one-to-one matching the paper bases on the
 * diagonal dominance of M; theta_i = asin(min(1, ||r_i||_B)) with
 * r_i = u_c - u_p (u_p^H B u_c), u_p and u_c the B-normalised x_prev_i and x_cur_assoc[i]
 * (full relative accuracy for small angles).  X_prev, X_cur: device, n x k; B: device,
 * n x n; theta: device, k doubles; assoc: device, k int32.  k <= blk_max, n <= n_max.
 * Uses the context's scratch buffers; the warm state and the stored factor of B are kept. */
int chfsi_deviation_angles(chfsi_ctx* ctx, int64_t n, int32_t k, const chfsi_z* X_prev, int64_t ldp,
                           const chfsi_z* X_cur, int64_t ldc, const chfsi_z* B, int64_t ldb,
                           double* theta, int32_t* assoc);

/* Closed-form per-vector degrees (not in the paper; the adaptive mode):
 * d_i = clamp(ceil(ln(r_i/tau)/ln rho_i), dmin, dmax), rho_i = |t_i| + sqrt(t_i^2-1),
 * t_i = (theta_i - c)/e; d_i = dmin when r_i <= tau, dmax when |t_i| <= 1; columns
 * i >= n_wanted take the largest degree of the first n_wanted.  theta, r device;
 * degrees: device, m int32.  With a model installed by chfsi_set_degree_model the learned
 * rate replaces ln rho_i (see below). */
int chfsi_degrees(chfsi_ctx* ctx, int32_t m, const double* theta, const double* r, double a,
                  double b, double tau, int32_t dmin, int32_t dmax, int32_t n_wanted,
                  int32_t* degrees);

/* Eigen-decomposition of the m x m Hermitian matrix G (full storage, device): ascending
 * eigenvalues w (device) and orthonormal eigenvectors V (device, ld ldv), by cyclic
 * parallel Jacobi.  G is not modified. */
int chfsi_heev(chfsi_ctx* ctx, int32_t m, const chfsi_z* G, int64_t ldg, double* w,
               chfsi_z* V, int64_t ldv);

/* The same decomposition (Rayleigh-Ritz step of Algorithm 1) as the mixed-precision solve
 * runs it on wide blocks: the matrix and the eigenvector rows held as double-float pairs
 * (hi + lo FP32 numbers, about 48 significand bits) and rotated with FP32 instructions, the
 * rotations computed in FP64; eigenvalue and orthogonality errors about 2^-46 ||G||_F.
 * Below 64 columns it is chfsi_heev.  Arguments, layout and errors as chfsi_heev
 * (EINVAL for bad sizes or NULL; ETIMEOUT; ENOCONV after 40 sweeps). */
int chfsi_heev_df(chfsi_ctx* ctx, int32_t m, const chfsi_z* G, int64_t ldg, double* w,
                  chfsi_z* V, int64_t ldv);

/* ---------------------------------------------------------------- allocation-free variant
 * The paper has no counterpart to this entry point; it serves callers that cannot call
 * cudaMalloc (an application whose pool allocator owns all device memory, or a
 * latency-critical path that must not trigger the implicit synchronisation of
 * cudaMalloc/cudaFree) and therefore cannot create a context.
 * Same computation as chfsi_heev (ascending eigenvalues w and orthonormal eigenvectors V of
 * the m x m Hermitian G, device pointers) with no context and no allocation: the scratch is
 * a fixed file-scope device array of 786,688 bytes that every GPU loading the library holds
 * until the process exits, so m is limited to CHFSI_HEEV_NOALLOC_MAX.
 *   cuda_stream  cudaStream_t to run on (NULL = the legacy default stream); the call
 *                synchronises it before returning.
 * All calls share the one array, which keeps the last call's contents (each call clears
 * what must start at zero): calls that overlap on the GPU (several streams or host
 * threads at once) race and must be serialised by the caller.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress, with that device
 * current) and keeps it for that device's context; the first call after the context was
 * reset (cudaDeviceReset) looks it up again.  Make the first call on a device before any
 * stream capture.  Works on the current device; G, w and V must live on it.
 * Errors: EINVAL (m > CHFSI_HEEV_NOALLOC_MAX, m <= 0, NULL, ld < m), ECUDA, ETIMEOUT,
 *         ENOCONV. */
#define CHFSI_HEEV_NOALLOC_MAX 128
int chfsi_heev_noalloc(int32_t m, const chfsi_z* G, int64_t ldg, double* w, chfsi_z* V,
                       int64_t ldv, void* cuda_stream);

/* Bound on the device-side waits of this context's kernels, in polls: the grid barriers of
 * the Rayleigh-Ritz eigensolver and the mbarrier waits of the split-BF16 product kernel
 * (not in the paper).  Every such wait is bounded; one that runs out sets a status flag,
 * the kernel unwinds (letting its own copies and tensor-core operations finish first) and
 * returns, and the call reports CHFSI_ETIMEOUT with the context still usable.  0 (the
 * default) means a few seconds of polling, far above any normal wait; a small bound makes
 * the waits run out, which is how the timeout path is exercised.  Errors: EINVAL. */
int chfsi_set_wait_limit(chfsi_ctx* ctx, int64_t polls);

/* Complex FP64 GEMM used by every dense step, exposed for testing:
 * C <- alpha op(A) op(B) + beta C, op = 'N' (as stored) or 'C' (conjugate transpose);
 * C is M x N, op(A) M x K, op(B) K x N.  alpha, beta real. */
int chfsi_zgemm(chfsi_ctx* ctx, char opa, char opb, int32_t M, int32_t N, int32_t K,
                double alpha, const chfsi_z* A, int64_t lda, const chfsi_z* B, int64_t ldb,
                double beta, chfsi_z* C, int64_t ldc);

/* ---------------------------------------------------------------- batched sequences */
/* Independent sequences solved concurrently on one GPU: the k-points of one
 * self-consistent cycle each give their own sequence of pencils (Section 1), with uneven
 * sizes.  A batch owns `workers` contexts (each with its own stream and the workspace of
 * chfsi_create(n_max, blk_max)) and solves with one host thread per context; whole
 * sequences are handed to the workers in order, so one sequence's host synchronisations
 * and latency-bound kernels overlap another's products.  opts: as chfsi_create, except
 * cuda_stream, which is ignored.  Errors of create: as chfsi_create. */
typedef struct chfsi_batch chfsi_batch;
int chfsi_batch_create(chfsi_batch** out, int32_t workers, int64_t n_max, int32_t blk_max,
                       const chfsi_opts* opts);
void chfsi_batch_destroy(chfsi_batch* batch);
const char* chfsi_batch_last_error(const chfsi_batch* batch);

/* K sequences of N problems each; sequence s has size n[s], nev[s], blk[s] (each within
 * the batch's n_max, blk_max), its problems at A[s*N + l], B[s*N + l] (lower triangles,
 * leading dimension ld[s], host or device as in chfsi_solve_next), outputs evals[s]
 * (N x nev[s], host), evecs[s*N + l] (n[s] x nev[s], or evecs == NULL) and st[s*N + l] (or
 * st == NULL).  Every sequence starts cold (each worker resets its warm state) and
 * problem l of a sequence is warm-started from problem l-1 (Section 3.2).  deg, tol as in
 * chfsi_solve_next.  Returns the first failing sequence's status (message in
 * chfsi_batch_last_error); sequences not yet started are then skipped. */
int chfsi_batch_solve(chfsi_batch* batch, int32_t K, int32_t N, const int64_t* n, const int32_t* nev,
                      const int32_t* blk, int32_t deg, double tol, const chfsi_z* const* A,
                      const chfsi_z* const* B, const int64_t* ld, double* const* evals,
                      chfsi_z* const* evecs, chfsi_stats* st);

/* ---------------------------------------------------------------- learned degree model */
/* Not in the paper: a learned form of the adaptive per-vector degree (the degree / block
 * size trade-off of Section 3.1).  The closed-form rule assumes a degree-d filter reduces the
 * residual of Ritz vector i by rho_i^d, rho_i = exp(acosh|t_i|), t_i = (theta_i - c)/e.  The
 * model predicts a correction g(x) of that rate, rate_i = ln(rho_i) exp(g(x_i)), and the
 * degree is d_i = clamp(ceil(ln(r_i/tau) / rate_i), deg_min, deg_max) (g clamped to [-3, 3];
 * the closed form wherever the result is not finite or no model is installed), from the
 * CHFSI_MLP_IN inputs of vector i in loop k of a problem:
 *   x0..x2  log10(r/tau) of the vector now and after the two previous loops (the residual
 *           history over the last three loops; a missing loop repeats the later value),
 *   x3, x4  the degrees it was filtered with in the two previous loops (0 where missing),
 *   x5      its normalised Ritz-value position t_i = (theta_i - c)/e,
 *   x6      the position t_0 = (a0 - c)/e of the smallest Ritz value a0 of the block,
 *   x7      the filter-bound ratio (a - a0)/(b - a0),
 * normalised as (x - mean) * scale, through a perceptron with three hidden layers of
 * CHFSI_MLP_HID tanh units and a linear output.  "The same vector" in consecutive loops is the
 * one with the same global index (locked count + active index; locking removes a prefix).
 * The solver evaluates it with FP16 weights; an untrained model (zero output layer) gives the
 * closed form exactly. */
#define CHFSI_MLP_IN 8
#define CHFSI_MLP_HID 64
/* trainable parameters (w1 .. b4): 8961 */
#define CHFSI_MLP_NPARAM                                                                   \
  (CHFSI_MLP_HID * CHFSI_MLP_IN + CHFSI_MLP_HID + 2 * (CHFSI_MLP_HID * CHFSI_MLP_HID +     \
   CHFSI_MLP_HID) + CHFSI_MLP_HID + 1)
typedef struct {
  float w1[CHFSI_MLP_HID * CHFSI_MLP_IN];  /* row j: weights of hidden unit j of layer 1 */
  float b1[CHFSI_MLP_HID];
  float w2[CHFSI_MLP_HID * CHFSI_MLP_HID]; /* row j: weights of hidden unit j of layer 2 */
  float b2[CHFSI_MLP_HID];
  float w3[CHFSI_MLP_HID * CHFSI_MLP_HID]; /* row j: weights of hidden unit j of layer 3 */
  float b3[CHFSI_MLP_HID];
  float w4[CHFSI_MLP_HID];                 /* output weights */
  float b4;
  float mean[CHFSI_MLP_IN], scale[CHFSI_MLP_IN];
} chfsi_mlp;

/* Uniform (Glorot) hidden weights from SplitMix64(seed), zero biases and output layer (the
 * untrained model predicts g = 0, i.e. the closed form), mean 0, scale 1. */
void chfsi_mlp_init(chfsi_mlp* model, uint64_t seed);
/* Training: sets mean/scale from X, then `epochs` epochs of Adam (lr, minibatches of
 * `batch`, order shuffled by SplitMix64(seed)) on L = 1/(2n) sum (g(x_k) - z_k)^2, in place
 * on *model.  X: host, n x CHFSI_MLP_IN (row-major), z: host, n.  *loss: mean loss of the last
 * epoch. */
int chfsi_mlp_train(chfsi_ctx* ctx, chfsi_mlp* model, const float* X, const float* z, int64_t n,
                    int32_t epochs, int32_t batch, float lr, uint64_t seed, float* loss);
/* One epoch of Adam (beta1 0.9, beta2 0.999, eps 1e-8) over the samples in the caller's order
 * (order: n indices into X, z), minibatches of `batch`, each on the gradient of its own mean
 * squared error; model (its mean/scale kept), moments m1, m2 (CHFSI_MLP_NPARAM floats each) and
 * the step counter updated in place (host); *loss = 1/(2n) sum of the epoch's squared errors. */
int chfsi_mlp_adam_epoch(chfsi_ctx* ctx, chfsi_mlp* model, float* m1, float* m2, int32_t* step,
                         const float* X, const float* z, const int32_t* order, int64_t n, int32_t batch,
                         float lr, float* loss);
/* dL/dparameters over all n samples (host, CHFSI_MLP_NPARAM floats in the order of chfsi_mlp's
 * fields w1 .. b4) and L, for the given model and its mean/scale. */
int chfsi_mlp_gradient(chfsi_ctx* ctx, const chfsi_mlp* model, const float* X, const float* z,
                       int64_t n, float* grad, float* loss);
/* g(x_k) for n host samples (FP32 weights). */
int chfsi_mlp_predict(chfsi_ctx* ctx, const chfsi_mlp* model, const float* X, int64_t n, float* y);
/* Install the model for the context's adaptive degrees (NULL: the closed form).  The step
 * entry point chfsi_degrees evaluates it without residual history (as in a first loop). */
int chfsi_set_degree_model(chfsi_ctx* ctx, const chfsi_mlp* model);

/* Degree log: from now on, every adaptive filter loop appends one record of
 * CHFSI_DEGREE_LOG_FIELDS doubles per active column, [problem, loop, g, i, m, theta, r, tau, d,
 * c, e, r_next, x0 .. x7]: problem counts solves of the context, g = locked count + i, d the
 * degree the column was filtered with, r_next its residual after the loop's filter and
 * Rayleigh-Ritz (so that vectors that lock in that loop are logged too), x the model inputs as
 * the solver computed them; up to `capacity` records; capacity 0 stops logging and clears it. */
#define CHFSI_DEGREE_LOG_FIELDS 20
int chfsi_degree_log_start(chfsi_ctx* ctx, int64_t capacity);
/* Copies up to cap records to out (host) and returns the number of records logged. */
int64_t chfsi_degree_log_read(chfsi_ctx* ctx, double* out, int64_t cap);

#ifdef __cplusplus
}
#endif
#endif /* CHFSI_H */
