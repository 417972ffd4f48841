// Internal declarations of the ChFSI library (kernels, workspace, engine).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>

#include <cuda_fp16.h>

#include "chfsi.h"

typedef double2 zd;  // complex double: x = real part, y = imaginary part

// Kernels launched by this library on the calling host thread (statistics only).
extern thread_local long long g_kernel_launches;
#define CHFSI_COUNT_LAUNCH() (++g_kernel_launches)

#define CHFSI_HD __host__ __device__ __forceinline__

CHFSI_HD zd zmk(double r, double i) { return make_double2(r, i); }
CHFSI_HD zd zadd(zd a, zd b) { return make_double2(a.x + b.x, a.y + b.y); }
CHFSI_HD zd zsub(zd a, zd b) { return make_double2(a.x - b.x, a.y - b.y); }
CHFSI_HD zd zscale(zd a, double s) { return make_double2(a.x * s, a.y * s); }
CHFSI_HD zd zconj(zd a) { return make_double2(a.x, -a.y); }
CHFSI_HD zd zmul(zd a, zd b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// c + a * b
CHFSI_HD zd zfma(zd a, zd b, zd c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// c + conj(a) * b
CHFSI_HD zd zfma_cj(zd a, zd b, zd c) {
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}
CHFSI_HD double zabs2(zd a) { return a.x * a.x + a.y * a.y; }

// Status flags written by kernels into the context's device status word.
enum : int {
  DEV_OK = 0,
  DEV_NOTPD = 1,       // non-positive pivot in a Cholesky factorisation
  DEV_TIMEOUT = 2,     // a bounded grid barrier gave up
  DEV_NOCONV = 4,      // Jacobi reached its sweep limit
  DEV_NAN = 8,         // non-finite value met
};

// ------------------------------------------------------------------ GEMM
enum { OPN = 0, OPC = 1 };

struct GemmDesc {
  int M = 0, N = 0, K = 0;
  const zd* A = nullptr; int64_t lda = 0; int opA = OPN;
  const zd* B = nullptr; int64_t ldb = 0; int opB = OPN;
  zd* C = nullptr; int64_t ldc = 0;
  double alpha = 1.0;
  double beta = 0.0; const zd* Cin = nullptr; int64_t ldcin = 0;   // + beta * Cin (may alias C)
  double gamma = 0.0; const zd* D = nullptr; int64_t ldd = 0;      // + gamma * D (may alias C)
  int triA = 0;   // 1: op(A)(i,k) == 0 for k > i (lower); 2: == 0 for k < i (upper)
  int triB = 0;   // 1: op(B)(k,j) == 0 for k > j (upper); 2: == 0 for k < j (lower)
  int lowerC = 0; // 1: only C(i,j) with i >= j is computed and written
};

struct Workspace;
// Queue one GEMM on `stream`.  Uses ws's split-K buffer.  Returns cudaError_t.
cudaError_t zgemm_run(const GemmDesc& g, Workspace& ws, cudaStream_t stream);
// Number of SMs of the current device (cached).
int sm_count();

// ------------------------------------------------------------------ small dense kernels
// Cholesky of an m x m Hermitian block (lower triangle read), in place: lower factor,
// strict upper zeroed.  scale: first scale to unit diagonal (D G D, dscale[i] = 1/sqrt(G_ii)).
// shift_on_fail: retry a failed factorisation on G + s I, s = shift_base * trace (shifted
// Cholesky QR); backup is an m x m scratch for the retry.  On failure sets DEV_NOTPD in
// status and atomically lowers *info to info_base + the failing pivot.  One CTA.
cudaError_t small_cholesky(zd* G, int64_t ldg, int m, int scale, int shift_on_fail,
                           double shift_base, double* dscale, zd* backup, int* status, int* info,
                           int info_base, cudaStream_t s, int* shift_flag = nullptr);
// X = L^{-1} for an m x m lower-triangular L (strict upper of X zeroed).  X != L.
cudaError_t trinv_lower(const zd* L, int64_t ldl, zd* X, int64_t ldx, int m, cudaStream_t s);
// One pass of the mixed-precision re-orthonormalisation (Y <- Y T) from G = Y^H Y (lower):
// a first-order Loewdin step in FP64 when ||G - I||_F <= 1e-3 (flags[0] = 1 once that norm
// is <= 1e-8), else an FP32 Cholesky QR step on the scaled Gram (shift on breakdown), whose
// T applies to Y scaled by dscale (flags[3] = 1).  T is m x m (full).  scratch: m*m + 32*m
// float2, or m*m float2 + one double per SM + 4 ints for the many-CTA pass (used when m > 144;
// barrier: 4 words for that pass's grid barrier, nullptr keeps the one-CTA pass; spin_limit:
// polls before a barrier wait gives up, 0 for the default).  flags: 4 ints.
cudaError_t qr_pass(const zd* G, int64_t ldg, int m, zd* T, int64_t ldt, double* dscale, void* scratch,
                    int* flags, int* status, cudaStream_t s, unsigned* barrier = nullptr,
                    long long spin_limit = 0);
// Y[:, j] *= d[j] when *flag (device) is set; no-op otherwise.
cudaError_t scale_cols_flag(zd* Y, int64_t ldy, int n, int m, const double* d, const int* flag, cudaStream_t s);
// T = D X^H (upper triangular, zero below): the right factor of Cholesky QR, Q = Y T.
cudaError_t cholqr_T(const zd* X, int64_t ldx, int m, const double* dscale, zd* T, int64_t ldt,
                     cudaStream_t s);
// Jacobi eigensolver (cooperative multi-CTA).  G not modified.  work: 3*m'*m' (m' = m
// rounded up to even), barrier: 4 words.  spin_limit: polls of a grid-barrier wait before it
// gives up (0: the default of a few seconds).
cudaError_t jacobi_heev(const zd* G, int64_t ldg, int m, double* w, zd* V, int64_t ldv,
                        zd* work, unsigned* barrier, int* status, cudaStream_t s,
                        long long spin_limit = 0);
// The same decomposition with the rotations applied in double-float arithmetic (about 48
// significand bits; FP32 instructions instead of the FP64 pipe): the mixed-precision path's
// solver for wide blocks.  Same arguments and work area; below 64 columns the FP64 solver.
cudaError_t jacobi_heev_df(const zd* G, int64_t ldg, int m, double* w, zd* V, int64_t ldv,
                           zd* work, unsigned* barrier, int* status, cudaStream_t s,
                           long long spin_limit = 0);

// Deviation angles (Section 2.2, Fig. 1): B-norms of columns from W = B X; greedy
// one-to-one association from |M|; the B-orthogonal parts R of the associated current
// vectors; theta_i = asin(min(1, ||r_i||_B)) from BR = B R.
cudaError_t bnorms(const zd* X, int64_t ldx, const zd* W, int64_t ldw, int n, int k, double* nrm,
                   cudaStream_t s);
cudaError_t associate(const zd* M, int64_t ldm, int k, int* assoc, cudaStream_t s);
cudaError_t deviation_residual(const zd* Xp, int64_t ldp, const zd* Xc, int64_t ldc, const zd* M,
                               int64_t ldm, const double* np_, const double* nc_, const int* assoc,
                               int n, int k, zd* R, int64_t ldr, cudaStream_t s);
cudaError_t deviation_theta(const zd* R, int64_t ldr, const zd* BR, int64_t ldbr, int n, int k,
                            double* theta, cudaStream_t s);

// ------------------------------------------------------------------ vector kernels
cudaError_t herm_from_lower(const zd* src, int64_t lds, zd* dst, int64_t ldd, int n,
                            int* status, cudaStream_t s);
cudaError_t mirror_lower(zd* H, int64_t ldh, int n, cudaStream_t s);
cudaError_t zero_upper(zd* L, int64_t ldl, int n, cudaStream_t s);
// H <- H + H^H in place (full storage), exactly Hermitian.
cudaError_t herm_sum(zd* H, int64_t ldh, int n, cudaStream_t s);
// out2 = [max_i |L_ii|^2, min_i |L_ii|^2] (device): their ratio bounds cond(L L^H) from below.
cudaError_t diag_ratio(const zd* L, int64_t ldl, int n, double* out2, cudaStream_t s);
cudaError_t copy_cols(const zd* src, int64_t lds, zd* dst, int64_t ldd, int n, int m,
                      cudaStream_t s);
cudaError_t compare_equal(const zd* a, int64_t lda, const zd* b, int64_t ldb, int n, int m,
                          int* diff_flag, cudaStream_t s);
cudaError_t gather_cols(const zd* src, int64_t lds, zd* dst, int64_t ldd, int n, int m,
                        const int* perm, cudaStream_t s);
cudaError_t select_cols(const zd* src1, int64_t ld1, zd* dst, int64_t ldd, int n, int m,
                        const int* flag, cudaStream_t s);
cudaError_t column_residuals(const zd* HY, int64_t ldhy, const zd* Y, int64_t ldy,
                             const double* theta, int n, int m, double* r, cudaStream_t s);
cudaError_t rayleigh_quotients(const zd* HY, int64_t ldhy, const zd* Y, int64_t ldy, int n, int m,
                               double* theta, cudaStream_t s);
cudaError_t generalized_residuals(const zd* AX, int64_t ldax, const zd* BX, int64_t ldbx,
                                  const zd* X, int64_t ldx, const double* lam, int n, int m,
                                  const double* a_norm, double* r, cudaStream_t s);
cudaError_t splitmix_start_vector(zd* v, int n, uint64_t seed, cudaStream_t s);
cudaError_t splitmix_gaussian_block(zd* Y, int64_t ldy, int n, int m, uint64_t seed,
                                    cudaStream_t s);
// Per-column degrees (closed-form rule; gcorr: the learned rate correction per column, or
// nullptr).  With rh1 != nullptr the column's residual and degree are pushed into the
// per-vector history (rh1/dh1: last loop, rh2/dh2: the loop before; global index g0 + i).
cudaError_t degrees_kernel_run(const double* theta, const double* r, int m, double a, double b,
                               double tau, int dmin, int dmax, int n_wanted, int* deg,
                               int* perm_desc, int* deg_sorted, cudaStream_t s, const float* gcorr = nullptr,
                               int g0 = 0, double* rh1 = nullptr, double* rh2 = nullptr,
                               int* dh1 = nullptr, int* dh2 = nullptr);
// Model inputs X (m x CHFSI_MLP_IN floats, row per column) from the block and the history
// (null history: none), and the model's g per column (FP16 weights as laid out by mlp_to_half).
cudaError_t degree_features(const double* theta, const double* r, int m, double a, double b, double tau,
                            int g0, const double* rh1, const double* rh2, const int* dh1, const int* dh2,
                            float* X, cudaStream_t s);
cudaError_t degree_model_eval(const __half* mlp, const float* X, int m, float* g, cudaStream_t s);
// learned degree model (mlp.cu)
int mlp_param_count();
cudaError_t mlp_to_half(const chfsi_mlp* m, __half* dst_dev, cudaStream_t s);
cudaError_t mlp_train(chfsi_mlp* m, const float* X, const float* z, int64_t n, int epochs, int batch,
                      float lr, uint64_t seed, float* loss_out, cudaStream_t s);
cudaError_t mlp_gradient(const chfsi_mlp* m, const float* X, const float* z, int64_t n, float* grad,
                         float* loss_out, cudaStream_t s);
cudaError_t mlp_predict(const chfsi_mlp* m, const float* X, int64_t n, float* y, cudaStream_t s);
cudaError_t mlp_adam_epoch(chfsi_mlp* m, float* m1, float* m2, int* step, const float* X, const float* z,
                           const int* order, int64_t n, int batch, float lr, float* loss_out, cudaStream_t s);
cudaError_t lock_scan(const double* r, int m, double tau, int max_lock, int* nlock,
                      cudaStream_t s);
cudaError_t fill_nan(double* x, int m, cudaStream_t s);

// Lanczos pieces
// w = H v for Hermitian H (row i read as column i); f32: FP32 multiply-adds (bound estimates).
cudaError_t hemv_rows(const zd* H, int64_t ldh, const zd* v, zd* w, int n, cudaStream_t s, bool f32 = false);
// Host-side set-up of the FP32 product for size n (kernel attribute, CTAs per SM with v in
// shared memory; 0 when v stays in global memory), cached per host thread: called before a
// stream capture so that none of it happens inside one.
cudaError_t hemv_rows_prepare(int n, int* per_sm);
cudaError_t block_dots(const zd* V, int64_t ldv, int j, const zd* w, int n, zd* c,
                       cudaStream_t s);
cudaError_t block_update(const zd* V, int64_t ldv, int j, const zd* c, zd* w, int n,
                         cudaStream_t s);
cudaError_t vec_norm(const zd* w, int n, double* out, cudaStream_t s);
cudaError_t vec_scale_into(const zd* w, int n, const double* nrm, zd* dst, cudaStream_t s);
cudaError_t lanczos_record(const zd* c, int j, const double* nrm, double* alpha, double* beta,
                           cudaStream_t s);
cudaError_t tridiag_extremes(const double* alpha, const double* beta, int k, double* out3,
                             cudaStream_t s);

// ------------------------------------------------------------------ split-BF16 products
struct OzA {                        // A operand: S digit slices of op(A) (M x K complex)
  struct __nv_bfloat16* ptr = nullptr;
  int* e = nullptr;                 // power-of-two scale per complex row
  int S = 0, M = 0, K = 0, Mp = 0, Kp = 0;
  int64_t slice = 0;
  int S_max = 0, Mp_max = 0, Kp_max = 0;
  int nz = 1;                       // 1: real embedding; 3: Gauss form (Hr, Hi, Hr + Hi)
};
struct OzB {                        // B operand: S digit slices of op(B) (K x N complex)
  struct __nv_bfloat16* ptr = nullptr;
  int* e = nullptr;                 // power-of-two scale per column
  int S = 0, N = 0, Np = 0, Kp = 0;
  int64_t slice = 0;
  int S_max = 0, Np_max = 0, Kp_max = 0;
  int64_t elems = 0;                // bf16 entries allocated
  int nz = 1;                       // 1: real embedding; 3: Gauss form (Yr, Yi, Yr + Yi)
};
struct OzWorkspace {
  OzA H;                            // slices of the problem's Hs (kept for the whole solve)
  OzA X;                            // scratch A operand of general products
  OzB B;                            // scratch B operand
  double* part = nullptr;           // split-K partial sums
  size_t part_elems = 0;
  int* status = nullptr;            // device status word for bounded-wait timeouts
  long long wait_limit = 0;         // polls of a first-level mbarrier wait (0: the default)
  int gauss = 1;                    // the Gauss form is allowed for the current products
};
bool oz_use_tcgen05();
int oz_padded_k(int n);
int oz_padded_m(int n);
int oz_padded_n(int m);
int64_t oz_pair_count(int S);
cudaError_t oz_alloc(OzWorkspace& oz, int n_max, int blk_max, int S_max);
void oz_free(OzWorkspace& oz);
// Digit slices of op(A) = X (op N: rows of X, M x K) or X^H (op C: conj columns of X, K x M).
cudaError_t oz_slice_a(OzA& a, int op, const zd* X, int64_t ldx, int M, int K, int S, cudaStream_t s);
// Digit slices of op(B) = X (op N: columns, K x N) or X^H (op C: conj rows of X, N x K).
cudaError_t oz_slice_b(OzB& b, int op, const zd* X, int64_t ldx, int K, int N, int S, int Kp,
                       cudaStream_t s, int lower_half = 0);
cudaError_t oz_product(const OzA& a, const OzB& b, int S, double alpha, double beta, const zd* Cin,
                       int64_t ldcin, double gamma, const zd* D, int64_t ldd, zd* out, int64_t ldo,
                       int a_lower, int c_lower, OzWorkspace& oz, cudaStream_t s,
                       cudaEvent_t ev_gemm_begin = nullptr, cudaEvent_t ev_gemm_end = nullptr, int b_tri = 0);
// Slices of the Hermitian Hs into oz.H (once per problem).
cudaError_t oz_slice_hermitian(const zd* Hs, int64_t ldh, int n, int S, OzWorkspace& oz,
                               cudaStream_t s);
// out = alpha Hs Y + beta Cin + gamma D with S-slice split-BF16 products (Hs from oz.H).
cudaError_t oz_filter_product(const zd* Y, int64_t ldy, int n, int m, int S, double alpha,
                              double beta, const zd* Cin, int64_t ldcin, double gamma, const zd* D,
                              int64_t ldd, zd* out, int64_t ldo, OzWorkspace& oz, cudaStream_t s,
                              cudaEvent_t ev_gemm_begin = nullptr, cudaEvent_t ev_gemm_end = nullptr);
// General split product on the scratch operands.
cudaError_t oz_gemm(int opA, const zd* A, int64_t lda, int opB, const zd* B, int64_t ldb, int M, int N,
                    int K, int S, double alpha, double beta, const zd* Cin, int64_t ldcin, double gamma,
                    const zd* D, int64_t ldd, zd* C, int64_t ldc, int a_lower, int c_lower,
                    OzWorkspace& oz, cudaStream_t s, int b_tri = 0,
                    int b_lower_half = 0);

// ------------------------------------------------------------------ workspace
struct Workspace {
  int dev = 0;
  int64_t n_max = 0;
  int blk_max = 0;
  // n x n buffers
  zd *Af = nullptr, *Bf = nullptr, *Lf = nullptr, *Linv = nullptr, *Hs = nullptr, *T = nullptr;
  // n x blk buffers
  zd *Y0 = nullptr, *Y1 = nullptr, *F = nullptr, *W = nullptr, *YL = nullptr, *Xw = nullptr,
     *Z = nullptr;
  // m x m buffers
  zd *G = nullptr, *V = nullptr, *Rt = nullptr, *jac = nullptr;
  // vectors
  zd *lv = nullptr, *lw = nullptr, *lV = nullptr, *lc = nullptr;  // Lanczos: n, n, n*(kmax+1), kmax+1
  int lanczos_kmax = 0;
  double *theta = nullptr, *theta2 = nullptr, *resid = nullptr, *resid2 = nullptr;
  double *lamL = nullptr, *residL = nullptr, *gres = nullptr;
  double *dscale = nullptr, *scal = nullptr, *lal = nullptr, *lbe = nullptr;
  int *deg = nullptr, *perm = nullptr, *degs = nullptr, *flag = nullptr, *ilist = nullptr;
  // learned degree: per-vector residual/degree history (global column index), model inputs
  // and outputs of the current loop
  double *hist_r1 = nullptr, *hist_r2 = nullptr;
  int *hist_d1 = nullptr, *hist_d2 = nullptr;
  float *feat = nullptr, *gcorr = nullptr;
  int* status = nullptr;  // [0]: DEV_* flags, [1]: first failing pivot
  int* shiftflag = nullptr;  // set when a Cholesky QR pass needed the shifted retry
  long long wait_limit = 0;  // polls of the eigensolver's grid-barrier waits (0: the default)
  unsigned* barrier = nullptr;
  // split-K partials
  zd* splitk = nullptr;
  size_t splitk_elems = 0;
  OzWorkspace oz;
  // pinned host mirror for small read-backs
  void* host_pinned = nullptr;
  size_t host_pinned_bytes = 0;
};

cudaError_t workspace_alloc(Workspace& ws, int64_t n_max, int blk_max, int lanczos_kmax);
void workspace_free(Workspace& ws);
