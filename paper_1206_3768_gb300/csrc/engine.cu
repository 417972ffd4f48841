// ChFSI engine and C ABI: context and workspace, reduction to standard form, Lanczos
// bound, Chebyshev filter, re-orthonormalisation, Rayleigh-Ritz, locking, and the
// sequence driver with warm starts (Algorithm 1 of Di Napoli & Berljafa, arXiv:1206.3768,
// with the reduction of Section 3.2).
//
// All arithmetic runs in the kernels of gemm.cu, small.cu and vec.cu on the context's
// stream.  The host only sequences launches and reads back, once per filter loop, the
// locked count and the Ritz values and residuals of the active block (a few KB), from
// which it sets the filter bounds and the per-step active widths.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "internal.cuh"

thread_local long long g_kernel_launches = 0;

struct chfsi_ctx {
  Workspace ws;
  chfsi_opts opts;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  // warm state: Ritz vectors (x-coordinates) in ws.Xw and their values
  bool has_warm = false;
  int64_t warm_n = 0;
  int warm_blk = 0;
  std::vector<double> warm_lam;
  // factor of B kept in ws.Lf / ws.Linv for ws.Bf
  bool has_factor = false;
  int64_t factor_n = 0;
  double factor_cond_lb = INFINITY;  // max/min squared pivot of that factor (cond(B) >= it)
  // phase timing
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct Mark { int phase; cudaEvent_t a, b; };
  std::vector<Mark> marks;
  // learned degree model (FP16 weights on the device) and the degree log
  __half* mlp_dev = nullptr;
  bool mlp_on = false;
  std::vector<double> deglog;
  int64_t deglog_cap = 0;
  int64_t problems_solved = 0;
  // staging of host inputs in chfsi_solve_sequence: problem l + 1's A and B are copied on
  // their own stream into the other of two buffer pairs while problem l solves
  cudaStream_t copy_stream = nullptr;
  zd* stage[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  cudaEvent_t staged[2] = {nullptr, nullptr};
  // Lanczos runs captured as CUDA graphs (their launch sequence depends only on the matrix,
  // its size, the step count, the seed and the precision), replayed on the context's stream
  struct LanczosGraph {
    const void* H; int64_t ldh; int n, k; uint64_t seed; int f32; const double* out;
    cudaGraphExec_t exec; long long kernels;
  };
  std::vector<LanczosGraph> lanczos_graphs;
  cudaStream_t capture_stream = nullptr;
  bool graphs_off = false;
};

namespace {

enum Phase { PH_REDUCE = 0, PH_LANCZOS, PH_FILTER, PH_QR, PH_RR, PH_RESID, PH_FGEMM, PH_SMALL, PH_EIG, PH_N };

int set_err(chfsi_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

#define CK(expr)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return set_err(ctx, CHFSI_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));   \
  } while (0)

#define CKS(expr)                \
  do {                           \
    int s_ = (expr);             \
    if (s_ != CHFSI_OK) return s_; \
  } while (0)

inline zd* Z(const chfsi_z* p) { return reinterpret_cast<zd*>(const_cast<chfsi_z*>(p)); }

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

cudaEvent_t next_event(chfsi_ctx* ctx) {
  if (ctx->ev_used == ctx->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    ctx->ev_pool.push_back(e);
  }
  return ctx->ev_pool[ctx->ev_used++];
}

struct PhaseScope {
  chfsi_ctx* ctx;
  int phase;
  cudaEvent_t a;
  PhaseScope(chfsi_ctx* c, int ph) : ctx(c), phase(ph) {
    a = next_event(c);
    cudaEventRecord(a, c->stream);
  }
  ~PhaseScope() {
    cudaEvent_t b = next_event(ctx);
    cudaEventRecord(b, ctx->stream);
    ctx->marks.push_back({phase, a, b});
  }
};

void collect_times(chfsi_ctx* ctx, double* t) {
  for (int i = 0; i < PH_N; ++i) t[i] = 0.0;
  for (auto& m : ctx->marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) t[m.phase] += ms;
    else cudaGetLastError();
  }
  ctx->marks.clear();
  ctx->ev_used = 0;
}

template <class T>
int read_back(chfsi_ctx* ctx, T* host, const T* dev, size_t count) {
  if (count == 0) return CHFSI_OK;
  CK(cudaMemcpyAsync(host, dev, count * sizeof(T), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CHFSI_OK;
}

int reset_status(chfsi_ctx* ctx) {
  const int init[2] = {0, 0x7fffffff};
  CK(cudaMemcpyAsync(ctx->ws.status, init, sizeof init, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CHFSI_OK;
}

// Translate the device status word into a return code (and clear it).
int check_status(chfsi_ctx* ctx, const char* where) {
  int st[2];
  CKS(read_back(ctx, st, ctx->ws.status, 2));
  if (st[0] == DEV_OK) return CHFSI_OK;
  const int info = st[1];
  CKS(reset_status(ctx));
  if (st[0] & DEV_TIMEOUT)
    return set_err(ctx, CHFSI_ETIMEOUT, "%s: a bounded device wait expired", where);
  if (st[0] & DEV_NAN) return set_err(ctx, CHFSI_EINVAL, "%s: non-finite input", where);
  if (st[0] & DEV_NOTPD)
    return set_err(ctx, CHFSI_ENOTPD, "%s: matrix not positive definite (pivot %d)", where, info);
  if (st[0] & DEV_NOCONV)
    return set_err(ctx, CHFSI_ENOCONV, "%s: Jacobi eigensolver reached its sweep limit", where);
  return set_err(ctx, CHFSI_ECUDA, "%s: device status %d", where, st[0]);
}

// Every public entry point starts by clearing the runtime's last-error slot, so that a
// non-sticky error left by an earlier, unrelated call is not reported as this call's
// failure.  With CHFSI_DEBUG set, such stale errors are printed to stderr.
void entry_guard(const char* fn) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess && std::getenv("CHFSI_DEBUG"))
    std::fprintf(stderr, "[chfsi] stale CUDA error '%s' at entry of %s\n", cudaGetErrorString(e), fn);
}

int gemm(chfsi_ctx* ctx, const GemmDesc& g) {
  CK(zgemm_run(g, ctx->ws, ctx->stream));
  return CHFSI_OK;
}

// A dense product in the context's precision: in mixed mode, products large enough to
// amortise the slicing run as 7-slice split-BF16 tensor-core products (error ~2e-15 relative
// to the operands' row and column scales; triangular operands are used with their exact
// zeros), the rest as FP64 GEMMs.
constexpr int kGemmSlices = 7;
int gemm_auto(chfsi_ctx* ctx, const GemmDesc& g) {
  const double work = (double)g.M * g.N * g.K;
  const bool square_c = !g.lowerC || g.M == g.N;
  if (ctx->opts.precision == 1 && work >= 16777216.0 && square_c) {
    CK(oz_gemm(g.opA, g.A, g.lda, g.opB, g.B, g.ldb, g.M, g.N, g.K, kGemmSlices, g.alpha, g.beta, g.Cin,
               g.ldcin, g.gamma, g.D, g.ldd, g.C, g.ldc, g.triA == 1, g.lowerC, ctx->ws.oz,
               ctx->stream, g.triB));
    return CHFSI_OK;
  }
  return gemm(ctx, g);
}

// A product of the factorisation of B and of its inverse (blocked Cholesky and triangular
// inverse): in mixed mode the large ones run as 8-slice digit products (error about 2^-56 of
// the operands' row and column scales, below the FP64 GEMM bound; the zero k-blocks of a
// triangular left or right operand are skipped), the rest in FP64.
int gemm_factor(chfsi_ctx* ctx, const GemmDesc& g) {
  const double work = (double)g.M * g.N * g.K;
  const bool square_c = !g.lowerC || g.M == g.N;
  if (ctx->opts.precision == 1 && work >= 16777216.0 && square_c) {
    CK(oz_gemm(g.opA, g.A, g.lda, g.opB, g.B, g.ldb, g.M, g.N, g.K, 8, g.alpha, g.beta, g.Cin, g.ldcin,
               g.gamma, g.D, g.ldd, g.C, g.ldc, g.triA == 1, g.lowerC, ctx->ws.oz, ctx->stream, g.triB));
    return CHFSI_OK;
  }
  return gemm(ctx, g);
}

// C(MxN) = alpha op(A) op(B) [+ beta Cin]
GemmDesc gd(int M, int N, int K, const zd* A, int64_t lda, int opA, const zd* B, int64_t ldb,
            int opB, zd* C, int64_t ldc, double alpha = 1.0) {
  GemmDesc g;
  g.M = M; g.N = N; g.K = K;
  g.A = A; g.lda = lda; g.opA = opA;
  g.B = B; g.ldb = ldb; g.opB = opB;
  g.C = C; g.ldc = ldc;
  g.alpha = alpha;
  return g;
}

// Panel width of the blocked factorisations (measured: 256-column panels made the n = 9300
// workload's reduction phase slower, 2.90 s against 2.81 s per 20-problem step).
constexpr int NB = 128;
// Digit slices of the FP64-level products in mixed mode (reduction, Rayleigh-Ritz, Gram and
// rotation products, back-transforms): 7 slices leave an error of about 2^-49 (2e-15)
// relative to the row and column scales, four orders of magnitude below the 1e-10 bar.
constexpr int kProductSlices = 7;

// Restores the workspace's Gauss-form permission on leaving a scope that changed it.
struct GaussScope {
  OzWorkspace& oz;
  int saved;
  GaussScope(OzWorkspace& o, int allow) : oz(o), saved(o.gauss) { oz.gauss = allow; }
  ~GaussScope() { oz.gauss = saved; }
};

// In-place blocked right-looking Cholesky on the lower triangle of L (n x n).  Its digit
// products keep the real embedding (the factor's errors reach every later step).
int blocked_cholesky(chfsi_ctx* ctx, zd* L, int64_t ld, int n, int nb = NB) {
  Workspace& ws = ctx->ws;
  GaussScope gs(ws.oz, 0);
  for (int k0 = 0; k0 < n; k0 += nb) {
    const int kb = std::min(nb, n - k0);
    zd* L11 = L + k0 + (int64_t)k0 * ld;
    CK(small_cholesky(L11, ld, kb, 0, 0, 0.0, nullptr, nullptr, ws.status, ws.status + 1, k0,
                      ctx->stream));
    const int r = n - k0 - kb;
    if (r <= 0) break;
    // L21 = A21 L11^{-H}
    CK(trinv_lower(L11, ld, ws.Rt, ws.blk_max, kb, ctx->stream));
    zd* A21 = L + (k0 + kb) + (int64_t)k0 * ld;
    GemmDesc g = gd(r, kb, kb, A21, ld, OPN, ws.Rt, ws.blk_max, OPC, ws.Z, r);
    g.triB = 1;
    CKS(gemm_factor(ctx, g));
    CK(cudaMemcpy2DAsync(A21, ld * sizeof(zd), ws.Z, r * sizeof(zd), r * sizeof(zd), kb,
                         cudaMemcpyDeviceToDevice, ctx->stream));
    // A22 -= L21 L21^H (lower)
    zd* A22 = L + (k0 + kb) + (int64_t)(k0 + kb) * ld;
    GemmDesc h = gd(r, r, kb, A21, ld, OPN, A21, ld, OPC, A22, ld, -1.0);
    h.beta = 1.0; h.Cin = A22; h.ldcin = ld; h.lowerC = 1;
    CKS(gemm_factor(ctx, h));
  }
  CK(zero_upper(L, ld, n, ctx->stream));
  return CHFSI_OK;
}

// X = L^{-1} (n x n, lower) by block rows: X_II = inv(L_II),
// X[I, 0:I] = -X_II (L[I, 0:I] X[0:I, 0:I]).
int blocked_trinv(chfsi_ctx* ctx, const zd* L, int64_t ld, zd* X, int64_t ldx, int n, int nb = NB) {
  Workspace& ws = ctx->ws;
  GaussScope gs(ws.oz, 0);  // the embedding, as in blocked_cholesky
  CK(cudaMemset2DAsync(X, ldx * sizeof(zd), 0, n * sizeof(zd), n, ctx->stream));
  for (int k0 = 0; k0 < n; k0 += nb) {
    const int kb = std::min(nb, n - k0);
    CK(trinv_lower(L + k0 + (int64_t)k0 * ld, ld, X + k0 + (int64_t)k0 * ldx, ldx, kb, ctx->stream));
    if (k0 == 0) continue;
    // Zt = L[I, 0:k0] X[0:k0, 0:k0]  (kb x k0), X lower => op(B)(k, j) = 0 for k < j
    GemmDesc g = gd(kb, k0, k0, L + k0, ld, OPN, X, ldx, OPN, ws.Z, kb);
    g.triB = 2;
    CKS(gemm_factor(ctx, g));
    // X[I, 0:k0] = -X_II Zt, X_II lower
    GemmDesc h = gd(kb, k0, kb, X + k0 + (int64_t)k0 * ldx, ldx, OPN, ws.Z, kb, OPN, X + k0, ldx, -1.0);
    h.triA = 1;
    CKS(gemm_factor(ctx, h));
  }
  return CHFSI_OK;
}

// Hs = Linv Af Linv^H.  split: the two products use split-BF16 tensor-core products
// (FP64-level accuracy) on the lower part A_h of Af (strict lower triangle plus half the
// diagonal, Af = A_h + A_h^H): P = Linv A_h is lower triangular (only k-blocks between the
// two triangles and the lower tiles are computed), Q = P Linv^H takes only k <= min(i, j),
// and Hs = Q + Q^H.  That is n^3/6 + n^3/3 complex multiply-adds against n^3/2 + n^3/3 for
// T = Linv Af, Hs = Linv T^H.  Otherwise (FP64): T = Linv Af, lower of T Linv^H, mirrored.
// Slices: the row scales of L^{-1} grow like sqrt(cond(B)), and its two products carry that
// growth into Hs; 8 slices (2^-56) keep the eigenvalue error at the FP64 level for cond(B)
// 1e4, 7 slices (2^-49) do so for a well-conditioned B (squared pivots within a factor 10;
// that ratio is a lower bound of cond(B) — 58.6 for a random B of condition 1e4 at n = 2600
// — so an ill-conditioned B may still take 7 only if its pivots hide it, which the
// generalized-residual acceptance then still checks).
int reduce_to_standard(chfsi_ctx* ctx, const zd* Af, int64_t lda, const zd* Linv, int64_t ldl,
                       zd* Hs, int64_t ldh, int n, bool split = false, double cond_lb = INFINITY) {
  Workspace& ws = ctx->ws;
  if (split) {
    const int S = cond_lb < 10.0 ? 7 : 8;
    // P = Linv A_h: lower x lower, lower tiles only (B zero for k < j)
    CK(oz_gemm(OPN, Linv, ldl, OPN, Af, lda, n, n, n, S, 1.0, 0.0, nullptr, 0, 0.0, nullptr, 0, ws.T,
               ws.n_max, 1, 1, ws.oz, ctx->stream, /*b_tri=*/2, /*b_lower_half=*/1));
    CK(zero_upper(ws.T, ws.n_max, n, ctx->stream));
    // Q = P Linv^H: lower x upper (B zero for k > j), full result
    CK(oz_gemm(OPN, ws.T, ws.n_max, OPC, Linv, ldl, n, n, n, S, 1.0, 0.0, nullptr, 0, 0.0, nullptr, 0,
               Hs, ldh, 1, 0, ws.oz, ctx->stream, /*b_tri=*/1));
    CK(herm_sum(Hs, ldh, n, ctx->stream));
    return CHFSI_OK;
  }
  GemmDesc g = gd(n, n, n, Linv, ldl, OPN, Af, lda, OPN, ws.T, ws.n_max);
  g.triA = 1;
  CKS(gemm(ctx, g));
  GemmDesc h = gd(n, n, n, ws.T, ws.n_max, OPN, Linv, ldl, OPC, Hs, ldh);
  h.triB = 1;
  h.lowerC = 1;
  CKS(gemm(ctx, h));
  CK(mirror_lower(Hs, ldh, n, ctx->stream));
  return CHFSI_OK;
}

// k-step Lanczos with full re-orthogonalisation (two classical Gram-Schmidt passes).  In
// mixed precision the products H v use FP32 multiply-adds on the FP64 data (a bound of the
// spectrum and a norm estimate need no more); the vectors and T_k stay FP64.
// v0: device start vector or nullptr (SplitMix64 with `seed`).  out3 (device):
// [theta_min, theta_max, theta_max + |beta_k|].
int lanczos_issue(chfsi_ctx* ctx, cudaStream_t st, const zd* H, int64_t ldh, int n, int k, const zd* v0,
                  uint64_t seed, double* out3);

// The launch-bound Lanczos loop (seven small kernels per step) is captured once per
// (matrix, size, steps, seed, precision) on a private stream and replayed as a CUDA graph on
// the context's stream; a caller start vector v0, or a failed capture, issues it directly.
int lanczos_run(chfsi_ctx* ctx, const zd* H, int64_t ldh, int n, int k, const zd* v0,
                uint64_t seed, double* out3) {
  const int f32 = ctx->opts.precision == 1;
  if (v0 || ctx->graphs_off) return lanczos_issue(ctx, ctx->stream, H, ldh, n, k, v0, seed, out3);
  k = std::min(std::min(k, n), ctx->ws.lanczos_kmax);
  for (auto& g : ctx->lanczos_graphs)
    if (g.H == H && g.ldh == ldh && g.n == n && g.k == k && g.seed == seed && g.f32 == f32 && g.out == out3) {
      CK(cudaGraphLaunch(g.exec, ctx->stream));
      g_kernel_launches += g.kernels;
      return CHFSI_OK;
    }
  if (!ctx->capture_stream) CK(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
  CK(hemv_rows_prepare(n, nullptr));
  cudaGraph_t graph = nullptr;
  const long long before = g_kernel_launches;
  cudaError_t e = cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const int rc = lanczos_issue(ctx, ctx->capture_stream, H, ldh, n, k, nullptr, seed, out3);
    e = cudaStreamEndCapture(ctx->capture_stream, &graph);
    if (rc != CHFSI_OK && e == cudaSuccess) e = cudaErrorUnknown;
  }
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  const long long kernels = g_kernel_launches - before;
  g_kernel_launches = before;
  if (e != cudaSuccess) {  // no graphs on this context: issue directly from now on
    cudaGetLastError();
    ctx->graphs_off = true;
    return lanczos_issue(ctx, ctx->stream, H, ldh, n, k, nullptr, seed, out3);
  }
  ctx->lanczos_graphs.push_back({H, ldh, n, k, seed, f32, out3, exec, kernels});
  CK(cudaGraphLaunch(exec, ctx->stream));
  g_kernel_launches += kernels;
  return CHFSI_OK;
}

int lanczos_issue(chfsi_ctx* ctx, cudaStream_t st, const zd* H, int64_t ldh, int n, int k, const zd* v0,
                  uint64_t seed, double* out3) {
  Workspace& ws = ctx->ws;
  k = std::min(k, n);
  k = std::min(k, ws.lanczos_kmax);
  if (k <= 0) return set_err(ctx, CHFSI_EINVAL, "lanczos: k must be positive");
  const int64_t ldv = ws.n_max;
  zd* V = ws.lV;
  if (v0) CK(cudaMemcpyAsync(ws.lw, v0, n * sizeof(zd), cudaMemcpyDeviceToDevice, st));
  else CK(splitmix_start_vector(ws.lw, n, seed, st));
  double* nrm = ws.scal + 8;
  CK(vec_norm(ws.lw, n, nrm, st));
  CK(vec_scale_into(ws.lw, n, nrm, V, st));
  for (int j = 0; j < k; ++j) {
    CK(hemv_rows(H, ldh, V + (int64_t)j * ldv, ws.lw, n, st, ctx->opts.precision == 1));
    CK(block_dots(V, ldv, j, ws.lw, n, ws.lc, st));
    CK(block_update(V, ldv, j, ws.lc, ws.lw, n, st));
    CK(block_dots(V, ldv, j, ws.lw, n, ws.lc + (ws.lanczos_kmax + 1), st));
    CK(block_update(V, ldv, j, ws.lc + (ws.lanczos_kmax + 1), ws.lw, n, st));
    CK(vec_norm(ws.lw, n, nrm, st));
    CK(lanczos_record(ws.lc, j, nrm, ws.lal, ws.lbe, st));
    if (j + 1 < k) CK(vec_scale_into(ws.lw, n, nrm, V + (int64_t)(j + 1) * ldv, st));
  }
  CK(tridiag_extremes(ws.lal, ws.lbe, k, out3, st));
  return CHFSI_OK;
}

// Chebyshev filter on the first m columns of *Ya (ld n_max) with per-column degrees.
// degs_sorted: host, descending; perm_dev: device permutation (column r of the permuted
// block is column perm[r] of the input) or nullptr when all degrees are equal.  The result
// (in permuted order) is left in *Ya.
int filter_block(chfsi_ctx* ctx, const zd* H, int64_t ldh, int n, int m, zd** Ya, zd** Yb,
                 zd** Yf, const std::vector<int>& degs_sorted, const int* perm_dev, double a0,
                 double a, double b, int64_t* matvecs, int slices = 0, chfsi_stats* st = nullptr) {
  Workspace& ws = ctx->ws;
  const int64_t ld = ws.n_max;
  if (m <= 0 || degs_sorted.empty()) return CHFSI_OK;
  const int dmax = degs_sorted[0];
  if (dmax <= 0) return CHFSI_OK;
  if (perm_dev) {
    CK(gather_cols(*Ya, ld, *Yb, ld, n, m, perm_dev, ctx->stream));
    std::swap(*Ya, *Yb);
  }
  const double e = 0.5 * (b - a), c = 0.5 * (b + a);
  const double s1 = e / (a0 - c);
  double s = s1;
  zd* buf[2] = {*Ya, *Yf};
  int mk = m;
  for (int k = 1; k <= dmax; ++k) {
    while (mk > 0 && degs_sorted[mk - 1] < k) --mk;
    if (mk <= 0) break;
    double al, be, ga;
    if (k == 1) {
      al = s1 / e; be = -al * c; ga = 0.0;
    } else {
      const double sn = 1.0 / (2.0 / s1 - s);
      al = 2.0 * sn / e; be = -al * c; ga = -s * sn;
      s = sn;
    }
    zd* cur = buf[(k - 1) & 1];
    zd* out = buf[k & 1];
    cudaEvent_t gb = nullptr, ge = nullptr;
    if (st) {
      gb = next_event(ctx);
      ge = next_event(ctx);
    }
    if (slices > 0) {
      // split-BF16 tensor-core product with the same fused recurrence epilogue
      CK(oz_filter_product(cur, ld, n, mk, slices, al, be, cur, ld, k >= 2 ? ga : 0.0, out, ld, out,
                           ld, ws.oz, ctx->stream, gb, ge));
      if (st) {
        // slice-pair flops the kernel issues: the 2n x 2n real embedding, or the Gauss form's
        // three real n x n products
        const double pairs = (double)oz_pair_count(slices);
        st->tensor_flops += ws.oz.H.nz == 3 ? 3.0 * 2.0 * pairs * n * (double)mk * n
                                            : 2.0 * pairs * (2.0 * n) * (double)mk * (2.0 * n);
        st->filter_products += 1;
        st->filter_slice_bytes += 2.0 * (double)slices * ws.oz.H.nz * ws.oz.H.Mp * (double)ws.oz.H.Kp;
      }
    } else {
      GemmDesc g = gd(n, mk, n, H, ldh, OPN, cur, ld, OPN, out, ld, al);
      g.beta = be; g.Cin = cur; g.ldcin = ld;
      if (k >= 2) { g.gamma = ga; g.D = out; g.ldd = ld; }
      if (gb) cudaEventRecord(gb, ctx->stream);
      CKS(gemm(ctx, g));
      if (ge) cudaEventRecord(ge, ctx->stream);
      if (st) st->filter_matvecs_fp64 += mk;
    }
    if (st) ctx->marks.push_back({PH_FGEMM, gb, ge});
    if (matvecs) *matvecs += mk;
  }
  // columns with odd degree ended in buf[1]
  std::vector<int> odd(m);
  int nodd = 0;
  for (int j = 0; j < m; ++j) { odd[j] = degs_sorted[j] & 1; nodd += odd[j]; }
  if (nodd == m) {
    std::swap(*Ya, *Yf);
  } else if (nodd > 0) {
    CK(cudaMemcpyAsync(ws.flag, odd.data(), m * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CK(select_cols(*Yf, ld, *Ya, ld, n, m, ws.flag, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));  // odd[] lives on the host stack
  }
  return CHFSI_OK;
}

// Digit slices for the next filter loop of the mixed-precision mode: the products must be
// accurate well below the residual the loop can reach, target = max(tau, r_min / (10 T)),
// T = |T_dmax(t0)| the largest amplification of one loop; about 2^(-7 S) relative error
// per product with S slices.
int slices_for_loop(double hs_norm, double tau, double r_min, double a0, double a, double b,
                    int dmax, int s_max) {
  if (!(r_min > 0.0) || !std::isfinite(r_min)) return s_max;
  const double e = 0.5 * (b - a), c = 0.5 * (b + a);
  const double t0 = std::fabs((a0 - c) / e);
  double T = 1.0;
  if (t0 > 1.0) T = std::cosh(dmax * std::acosh(t0));
  if (!std::isfinite(T)) T = 1e300;
  const double target = std::max(tau, r_min / (10.0 * T));
  static const double margin = [] {
    const char* v = std::getenv("CHFSI_SLICE_MARGIN_BITS");
    return v ? std::atof(v) : 6.0;
  }();
  const double bits = std::log2(hs_norm / target) + margin;
  const int S = (int)std::ceil(bits / 7.0);
  return std::min(s_max, std::max(2, S));
}

// CGS2 against YL (k columns), then re-orthonormalisation: in mixed precision FP32 Cholesky QR
// steps and FP64 Loewdin steps chosen on the device (qr_pass); in FP64 Cholesky QR twice, three
// times when the first pass needed the shifted retry.
int orthonormalize_block(chfsi_ctx* ctx, int n, int m, zd** Ya, zd** Yb, const zd* YL, int64_t ldyl,
                         int k) {
  Workspace& ws = ctx->ws;
  const int64_t ld = ws.n_max;
  const int64_t ldm = ws.blk_max;
  if (m <= 0) return CHFSI_OK;
  if (k > 0) {
    for (int pass = 0; pass < 2; ++pass) {
      CKS(gemm_auto(ctx, gd(k, m, n, YL, ldyl, OPC, *Ya, ld, OPN, ws.G, ldm)));
      GemmDesc g = gd(n, m, k, YL, ldyl, OPN, ws.G, ldm, OPN, *Ya, ld, -1.0);
      g.beta = 1.0; g.Cin = *Ya; g.ldcin = ld;
      CKS(gemm_auto(ctx, g));
    }
  }
  if (ctx->opts.precision == 1) {
    // Mixed precision: FP32 Cholesky QR steps until the Gram matrix is within 1e-3 of the
    // identity, then FP64 first-order Loewdin steps (T = I - (G - I)/2) until it is within
    // 1e-8, which leaves an orthonormality error of about 1e-16.  The device chooses the
    // step from G; the host reads the "finished" flag from the third pass on.
    CK(cudaMemsetAsync(ws.shiftflag, 0, 4 * sizeof(int), ctx->stream));
    for (int pass = 0; pass < 12; ++pass) {
      GemmDesc g = gd(m, m, n, *Ya, ld, OPC, *Ya, ld, OPN, ws.G, ldm);
      g.lowerC = 1;
      CKS(gemm_auto(ctx, g));
      {
        PhaseScope ps(ctx, PH_SMALL);
        CK(qr_pass(ws.G, ldm, m, ws.V, ldm, ws.dscale, ws.jac, ws.shiftflag, ws.status, ctx->stream,
                   ws.barrier, ws.wait_limit));
        CK(scale_cols_flag(*Ya, ld, n, m, ws.dscale, ws.shiftflag + 3, ctx->stream));
      }
      CKS(gemm_auto(ctx, gd(n, m, m, *Ya, ld, OPN, ws.V, ldm, OPN, *Yb, ld)));
      std::swap(*Ya, *Yb);
      if (pass >= 2) {
        int done = 0;
        CKS(read_back(ctx, &done, ws.shiftflag, 1));
        if (done) return CHFSI_OK;
      }
    }
    // not finished (a numerically rank-deficient block): finish with FP64 shifted Cholesky QR
  }
  const double u = 1.1102230246251565e-16;
  const double shift_base = 11.0 * ((double)n * m + (double)m * (m + 1)) * u;
  // Cholesky QR twice; a third pass only when the first one needed the shifted retry
  // (shifted Cholesky QR3), which the device reports in ws.shiftflag.
  CK(cudaMemsetAsync(ws.shiftflag, 0, sizeof(int), ctx->stream));
  for (int pass = 0; pass < 3; ++pass) {
    if (pass == 2) {
      int shifted = 1;
      CKS(read_back(ctx, &shifted, ws.shiftflag, 1));
      if (!shifted) break;
    }
    GemmDesc g = gd(m, m, n, *Ya, ld, OPC, *Ya, ld, OPN, ws.G, ldm);
    g.lowerC = 1;
    CKS(gemm_auto(ctx, g));
    {
      PhaseScope ps(ctx, PH_SMALL);
      CK(small_cholesky(ws.G, ldm, m, 1, 1, shift_base, ws.dscale, ws.jac, ws.status, ws.status + 1, 0,
                        ctx->stream, pass == 0 ? ws.shiftflag : nullptr));
      CK(trinv_lower(ws.G, ldm, ws.Rt, ldm, m, ctx->stream));
      CK(cholqr_T(ws.Rt, ldm, m, ws.dscale, ws.V, ldm, ctx->stream));
    }
    GemmDesc h = gd(n, m, m, *Ya, ld, OPN, ws.V, ldm, OPN, *Yb, ld);
    h.triB = 1;
    CKS(gemm_auto(ctx, h));
    std::swap(*Ya, *Yb);
  }
  return CHFSI_OK;
}

// Narrowest Rayleigh-Ritz block whose eigensolver runs in double-float arithmetic in mixed
// precision: environment variable CHFSI_JACOBI_DF_MIN (default 384 columns).
int jacobi_df_min() {
  static const int v = [] {
    const char* e = std::getenv("CHFSI_JACOBI_DF_MIN");
    return e ? std::atoi(e) : 384;
  }();
  return v;
}

// Rayleigh-Ritz on the m columns of *Ya: theta (device), *Ya <- Ritz vectors, *W <- H *Ya.
int rayleigh_ritz_block(chfsi_ctx* ctx, const zd* H, int64_t ldh, int n, int m, zd** Ya, zd** Yb,
                        zd** W, zd** Zb, double* theta, int rr_slices = 0) {
  Workspace& ws = ctx->ws;
  const int64_t ld = ws.n_max;
  const int64_t ldm = ws.blk_max;
  if (rr_slices > 0) {
    // FP64-level product from 7 digit slices per operand (error ~2e-15 of the scales)
    CK(oz_filter_product(*Ya, ld, n, m, rr_slices, 1.0, 0.0, nullptr, 0, 0.0, nullptr, 0, *W, ld,
                         ws.oz, ctx->stream));
  } else {
    CKS(gemm(ctx, gd(n, m, n, H, ldh, OPN, *Ya, ld, OPN, *W, ld)));
  }
  GemmDesc g = gd(m, m, n, *Ya, ld, OPC, *W, ld, OPN, ws.G, ldm);
  g.lowerC = 1;
  CKS(gemm_auto(ctx, g));
  CK(mirror_lower(ws.G, ldm, m, ctx->stream));
  {
    PhaseScope ps(ctx, PH_EIG);
    if (ctx->opts.precision == 1 && m >= jacobi_df_min())
      CK(jacobi_heev_df(ws.G, ldm, m, theta, ws.V, ldm, ws.jac, ws.barrier, ws.status, ctx->stream,
                        ws.wait_limit));
    else
      CK(jacobi_heev(ws.G, ldm, m, theta, ws.V, ldm, ws.jac, ws.barrier, ws.status, ctx->stream,
                     ws.wait_limit));
  }
  CKS(gemm_auto(ctx, gd(n, m, m, *Ya, ld, OPN, ws.V, ldm, OPN, *Yb, ld)));
  CKS(gemm_auto(ctx, gd(n, m, m, *W, ld, OPN, ws.V, ldm, OPN, *Zb, ld)));
  std::swap(*Ya, *Yb);
  std::swap(*W, *Zb);
  return CHFSI_OK;
}

int validate_sizes(chfsi_ctx* ctx, int64_t n, int32_t nev, int32_t blk) {
  if (!ctx) return CHFSI_EINVAL;
  if (n <= 0 || n > ctx->ws.n_max)
    return set_err(ctx, CHFSI_EINVAL, "n=%lld outside (0, n_max=%lld]", (long long)n,
                   (long long)ctx->ws.n_max);
  if (nev <= 0 || blk < nev || blk > n || blk > ctx->ws.blk_max)
    return set_err(ctx, CHFSI_EINVAL, "need 0 < nev <= blk <= min(n, blk_max): nev=%d blk=%d",
                   nev, blk);
  return CHFSI_OK;
}

// Stage an n x cols matrix (host or device, leading dimension ld) into a device buffer
// (ld_dst) or return the device pointer itself when no copy is needed.
int stage_in(chfsi_ctx* ctx, const chfsi_z* src, int64_t ld, int n, int cols, zd* staging,
             int64_t ld_dst, const zd** out) {
  if (is_device_ptr(src)) {
    *out = Z(src);
    return CHFSI_OK;
  }
  CK(cudaMemcpy2DAsync(staging, ld_dst * sizeof(zd), src, ld * sizeof(zd), n * sizeof(zd), cols,
                       cudaMemcpyHostToDevice, ctx->stream));
  *out = staging;
  return CHFSI_OK;
}

struct SolveArgs {
  int n, nev, blk, deg;
  double tol;
  const chfsi_z *A, *B, *V0;
  int64_t lda, ldb;
  double* evals;
  chfsi_z* evecs;
  chfsi_stats* st;
};

int solve_one(chfsi_ctx* ctx, const SolveArgs& S) {
  Workspace& ws = ctx->ws;
  const int n = S.n, nev = S.nev, blk = S.blk;
  const int64_t ld = ws.n_max, ldm = ws.blk_max;
  chfsi_stats st{};
  double tph[PH_N];
  const chfsi_opts& o = ctx->opts;
  const bool adaptive = S.deg <= 0;
  if (adaptive && (o.deg_min < 1 || o.deg_max < o.deg_min))
    return set_err(ctx, CHFSI_EINVAL, "bad adaptive degree range [%d, %d]", o.deg_min, o.deg_max);
  if (!(S.tol > 0.0)) return set_err(ctx, CHFSI_EINVAL, "tol must be positive");
  CKS(reset_status(ctx));
  const long long launches0 = g_kernel_launches;
  cudaEvent_t t_start = next_event(ctx), t_end = next_event(ctx);
  CK(cudaEventRecord(t_start, ctx->stream));

  // ---------------------------------------------------------------- a1, a2: reduction
  {
    PhaseScope ps(ctx, PH_REDUCE);
    const zd* Bsrc = nullptr;
    CKS(stage_in(ctx, S.B, S.ldb, n, n, ws.Hs, ld, &Bsrc));
    bool refactor = true;
    if (o.reuse_factor && ctx->has_factor && ctx->factor_n == n) {
      CK(cudaMemsetAsync(ws.flag, 0, sizeof(int), ctx->stream));
      CK(compare_equal(Bsrc, Bsrc == ws.Hs ? ld : S.ldb, ws.Bf, ld, n, n, ws.flag, ctx->stream));
      int diff = 1;
      CKS(read_back(ctx, &diff, ws.flag, 1));
      refactor = diff != 0;
    }
    if (refactor) {
      ctx->has_factor = false;
      CK(herm_from_lower(Bsrc, Bsrc == ws.Hs ? ld : S.ldb, ws.Bf, ld, n, ws.status, ctx->stream));
      CK(cudaMemcpy2DAsync(ws.Lf, ld * sizeof(zd), ws.Bf, ld * sizeof(zd), n * sizeof(zd), n,
                           cudaMemcpyDeviceToDevice, ctx->stream));
      CKS(blocked_cholesky(ctx, ws.Lf, ld, n));
      CKS(check_status(ctx, "Cholesky of B"));
      CK(diag_ratio(ws.Lf, ld, n, ws.scal + 12, ctx->stream));
      double piv[2];
      CKS(read_back(ctx, piv, ws.scal + 12, 2));
      ctx->factor_cond_lb = piv[1] > 0.0 ? piv[0] / piv[1] : INFINITY;
      // Gauss form of the problem's complex products only for a well-conditioned B (squared
      // pivots within a factor 10; the pivot ratio is a lower bound of cond(B), 58.6 for a
      // random B of condition 1e4 at n = 2600 and about 1 for B = I + 0.1 G^H G / n): with
      // cond(B) ~ 1e4 the filter needs accuracy at the edge of 7 slices, and the Gauss
      // form's errors are up to a few times the embedding's (three products' bounds)
      ws.oz.gauss = ctx->factor_cond_lb < 10.0 ? 1 : 0;
      CKS(blocked_trinv(ctx, ws.Lf, ld, ws.Linv, ld, n));
      ctx->has_factor = true;
      ctx->factor_n = n;
    }
    const zd* Asrc = nullptr;
    CKS(stage_in(ctx, S.A, S.lda, n, n, ws.Hs, ld, &Asrc));
    CK(herm_from_lower(Asrc, Asrc == ws.Hs ? ld : S.lda, ws.Af, ld, n, ws.status, ctx->stream));
    CKS(reduce_to_standard(ctx, ws.Af, ld, ws.Linv, ld, ws.Hs, ld, n, o.precision == 1,
                           ctx->factor_cond_lb));
    if (o.precision == 1) CK(oz_slice_hermitian(ws.Hs, ld, n, kProductSlices, ws.oz, ctx->stream));
  }
  CKS(check_status(ctx, "input"));

  const int rr_slices = o.precision == 1 ? kProductSlices : 0;

  // ---------------------------------------------------------------- a3: Lanczos bounds
  const bool warm = ctx->has_warm && ctx->warm_n == n && ctx->warm_blk == blk;
  double lz[3], an[3];
  {
    PhaseScope ps(ctx, PH_LANCZOS);
    const int k = warm ? o.lanczos_k_warm : o.lanczos_k_cold;
    CKS(lanczos_run(ctx, ws.Hs, ld, n, k, nullptr, o.seed, ws.scal));
    CKS(lanczos_run(ctx, ws.Af, ld, n, 20, nullptr, o.seed ^ 0x5A5A5A5Aull, ws.scal + 3));
    st.matvecs += std::min(k, n);
  }
  CKS(read_back(ctx, lz, ws.scal, 3));
  CKS(read_back(ctx, an, ws.scal + 3, 3));
  const double b_up = lz[2];
  const double a_norm = std::max(std::fabs(an[0]), std::fabs(an[1]));
  CK(cudaMemcpyAsync(ws.scal + 6, &a_norm, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  st.lanczos_upper = b_up;

  // ---------------------------------------------------------------- start block
  zd *Ya = ws.Y0, *Yb = ws.Y1, *Yf = ws.F, *W = ws.W, *Zb = ws.Z;
  if (warm) {
    GemmDesc g = gd(n, blk, n, ws.Lf, ld, OPC, ws.Xw, ld, OPN, Ya, ld);
    g.triA = 2;
    CKS(gemm_auto(ctx, g));
  } else if (S.V0) {
    const zd* v0 = nullptr;
    CKS(stage_in(ctx, S.V0, n, n, blk, Yb, ld, &v0));
    CK(cudaMemcpy2DAsync(Ya, ld * sizeof(zd), v0, (v0 == Yb ? ld : n) * sizeof(zd), n * sizeof(zd),
                         blk, cudaMemcpyDeviceToDevice, ctx->stream));
  } else {
    CK(splitmix_gaussian_block(Ya, ld, n, blk, o.seed + 1, ctx->stream));
  }

  std::vector<double> th(blk), rr(blk), lamL;
  std::vector<double> rL;
  double a0, a;
  double* theta = ws.theta;
  double* theta_alt = ws.theta2;
  double* resid = ws.resid;
  double* resid_alt = ws.resid2;
  bool have_r = false;
  if (warm && adaptive) {
    // adaptive degrees need residuals before the first loop: for a warm start they are the
    // residuals of the carried vectors at their Rayleigh quotients (one product H Y, no
    // re-orthonormalisation or Rayleigh-Ritz); the bounds come from the carried Ritz values
    {
      PhaseScope ps(ctx, PH_RESID);
      if (rr_slices > 0)
        CK(oz_filter_product(Ya, ld, n, blk, rr_slices, 1.0, 0.0, nullptr, 0, 0.0, nullptr, 0, W, ld, ws.oz,
                             ctx->stream));
      else
        CKS(gemm(ctx, gd(n, blk, n, ws.Hs, ld, OPN, Ya, ld, OPN, W, ld)));
      CK(rayleigh_quotients(W, ld, Ya, ld, n, blk, theta, ctx->stream));
      CK(column_residuals(W, ld, Ya, ld, theta, n, blk, resid, ctx->stream));
    }
    st.matvecs += blk;
    CKS(read_back(ctx, th.data(), theta, blk));
    CKS(read_back(ctx, rr.data(), resid, blk));
    have_r = true;
    a0 = ctx->warm_lam[0];
    a = ctx->warm_lam[blk - 1];
  } else if (!warm) {
    {
      PhaseScope ps(ctx, PH_QR);
      CKS(orthonormalize_block(ctx, n, blk, &Ya, &Yb, nullptr, 0, 0));
    }
    {
      PhaseScope ps(ctx, PH_RR);
      CKS(rayleigh_ritz_block(ctx, ws.Hs, ld, n, blk, &Ya, &Yb, &W, &Zb, theta, rr_slices));
    }
    {
      PhaseScope ps(ctx, PH_RESID);
      CK(column_residuals(W, ld, Ya, ld, theta, n, blk, resid, ctx->stream));
    }
    st.matvecs += blk;
    CKS(read_back(ctx, th.data(), theta, blk));
    CKS(read_back(ctx, rr.data(), resid, blk));
    CKS(check_status(ctx, "initial Rayleigh-Ritz"));
    have_r = true;
    a0 = th[0];
    a = a0 + (b_up - a0) * (double)blk / (double)n;
  } else {
    th = ctx->warm_lam;
    a0 = th[0];
    a = th[blk - 1];
  }
  double tau = 0.25 * S.tol * std::max(std::fabs(a0), std::fabs(b_up));

  int conv = 0;
  int status = CHFSI_OK;
  std::vector<int> degs;
  std::vector<double> pending_log;  // degree-log records of the current loop
  if (adaptive) {
    // the learned degree's per-vector history starts empty for every problem
    CK(cudaMemsetAsync(ws.hist_r1, 0, 2 * sizeof(double) * ws.blk_max, ctx->stream));
    CK(cudaMemsetAsync(ws.hist_d1, 0, 2 * sizeof(int) * ws.blk_max, ctx->stream));
  }
  double max_gres = NAN;
  const double hs_norm = std::max(std::fabs(a0), std::fabs(b_up));
  bool mixed = o.precision == 1;
  int slice_boost = 0;        // extra slices after a loop that stalled on product precision
  double front_before = NAN;  // residual of the first active (next to lock) column
  for (int accept = 0; accept < 4; ++accept) {
    while (conv < nev && st.loops < o.max_loops) {
      const int m = blk - conv;
      // ---- a8: degrees
      const int* perm_dev = nullptr;
      degs.assign(m, S.deg);
      pending_log.clear();
      if (adaptive) {
        if (!have_r) return set_err(ctx, CHFSI_ECUDA, "internal: residuals missing");
        const bool logging = ctx->deglog_cap > 0 && (int)th.size() == m &&
                             (int64_t)ctx->deglog.size() / CHFSI_DEGREE_LOG_FIELDS < ctx->deglog_cap;
        const float* gcorr = nullptr;
        if (ctx->mlp_on || logging) {
          CK(degree_features(theta, resid, m, a, b_up, tau, conv, ws.hist_r1, ws.hist_r2, ws.hist_d1,
                             ws.hist_d2, ws.feat, ctx->stream));
          if (ctx->mlp_on) {
            CK(degree_model_eval(ctx->mlp_dev, ws.feat, m, ws.gcorr, ctx->stream));
            gcorr = ws.gcorr;
          }
        }
        if (logging) {
          std::vector<float> feat((size_t)m * CHFSI_MLP_IN);
          CKS(read_back(ctx, feat.data(), ws.feat, feat.size()));
          const double c = 0.5 * (a + b_up), e = 0.5 * (b_up - a);
          pending_log.resize((size_t)m * CHFSI_DEGREE_LOG_FIELDS);
          for (int i = 0; i < m; ++i) {
            double* rec = pending_log.data() + (size_t)i * CHFSI_DEGREE_LOG_FIELDS;
            const double head[12] = {(double)ctx->problems_solved, (double)st.loops, (double)(conv + i),
                                     (double)i, (double)m, th[i], rr[i], tau, 0.0, c, e, NAN};
            std::copy(head, head + 12, rec);
            for (int f = 0; f < CHFSI_MLP_IN; ++f) rec[12 + f] = feat[(size_t)i * CHFSI_MLP_IN + f];
          }
        }
        CK(degrees_kernel_run(theta, resid, m, a, b_up, tau, o.deg_min, o.deg_max, nev - conv,
                              ws.deg, ws.perm, ws.degs, ctx->stream, gcorr, conv, ws.hist_r1, ws.hist_r2,
                              ws.hist_d1, ws.hist_d2));
        CKS(read_back(ctx, degs.data(), ws.degs, m));
        perm_dev = ws.perm;
        if (logging) {
          // degrees per column (degs holds them in descending order): read them unsorted
          std::vector<int> dcol(m);
          CKS(read_back(ctx, dcol.data(), ws.deg, m));
          for (int i = 0; i < m; ++i) pending_log[(size_t)i * CHFSI_DEGREE_LOG_FIELDS + 8] = dcol[i];
        }
      }
      // ---- a4: filter (split-BF16 tensor-core products in mixed mode)
      int slices = 0;
      // smallest residual among the wanted active columns that still need filtering
      double rneed = INFINITY;
      if (have_r)
        for (int i = 0; i < std::min(nev - conv, (int)rr.size()); ++i)
          if (rr[i] >= tau) rneed = std::min(rneed, rr[i]);
      front_before = (have_r && !rr.empty()) ? rr[0] : NAN;
      if (mixed) {
        const int dmax_loop = degs.empty() ? 0 : *std::max_element(degs.begin(), degs.end());
        slices = slices_for_loop(hs_norm, tau, have_r ? rneed : NAN, a0, a, b_up, dmax_loop,
                                 o.slices_max);
        slices = std::min(o.slices_max, slices + slice_boost);
      }
      {
        PhaseScope ps(ctx, PH_FILTER);
        CKS(filter_block(ctx, ws.Hs, ld, n, m, &Ya, &Yb, &Yf, degs, perm_dev, a0, a, b_up,
                         &st.filter_matvecs, slices, &st));
      }
      st.filtered_vectors += m;
      // ---- a5: deflation + Cholesky QR
      {
        PhaseScope ps(ctx, PH_QR);
        CKS(orthonormalize_block(ctx, n, m, &Ya, &Yb, ws.YL, ld, conv));
      }
      // ---- a6: Rayleigh-Ritz
      {
        PhaseScope ps(ctx, PH_RR);
        CKS(rayleigh_ritz_block(ctx, ws.Hs, ld, n, m, &Ya, &Yb, &W, &Zb, theta, rr_slices));
      }
      st.matvecs += m;
      // ---- a7: residuals and locking
      {
        PhaseScope ps(ctx, PH_RESID);
        CK(column_residuals(W, ld, Ya, ld, theta, n, m, resid, ctx->stream));
        CK(lock_scan(resid, m, tau, nev - conv, ws.ilist, ctx->stream));
      }
      // one synchronisation for the loop's read-back: status, locked count, theta, r
      int nlock = 0;
      {
        int* h_int = static_cast<int*>(ws.host_pinned);
        double* h_th = reinterpret_cast<double*>(static_cast<char*>(ws.host_pinned) + 16);
        double* h_r = h_th + ws.blk_max;
        CK(cudaMemcpyAsync(h_int, ws.status, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(h_int + 2, ws.ilist, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(h_th, theta, m * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(h_r, resid, m * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        nlock = h_int[2];
        std::copy(h_th, h_th + m, th.begin());
        std::copy(h_r, h_r + m, rr.begin());
        if (h_int[0] != DEV_OK) CKS(check_status(ctx, "filter loop"));
      }
      have_r = true;
      st.loops++;
      if (!pending_log.empty()) {
        // the residual each logged column reached after this loop's filter and Rayleigh-Ritz
        for (int i = 0; i < m; ++i) pending_log[(size_t)i * CHFSI_DEGREE_LOG_FIELDS + 11] = rr[i];
        const int64_t room = ctx->deglog_cap - (int64_t)ctx->deglog.size() / CHFSI_DEGREE_LOG_FIELDS;
        const int64_t cnt = std::min<int64_t>(room, m);
        ctx->deglog.insert(ctx->deglog.end(), pending_log.begin(),
                           pending_log.begin() + cnt * CHFSI_DEGREE_LOG_FIELDS);
        pending_log.clear();
      }
      if (nlock > 0) {
        CK(copy_cols(Ya, ld, ws.YL + (int64_t)conv * ld, ld, n, nlock, ctx->stream));
        CK(cudaMemcpyAsync(ws.lamL + conv, theta, nlock * sizeof(double), cudaMemcpyDeviceToDevice,
                           ctx->stream));
        CK(cudaMemcpyAsync(ws.residL + conv, resid, nlock * sizeof(double),
                           cudaMemcpyDeviceToDevice, ctx->stream));
        lamL.insert(lamL.end(), th.begin(), th.begin() + nlock);
        rL.insert(rL.end(), rr.begin(), rr.begin() + nlock);
        const int rem = m - nlock;
        CK(copy_cols(Ya + (int64_t)nlock * ld, ld, Yb, ld, n, rem, ctx->stream));
        std::swap(Ya, Yb);
        CK(cudaMemcpyAsync(theta_alt, theta + nlock, rem * sizeof(double), cudaMemcpyDeviceToDevice,
                           ctx->stream));
        CK(cudaMemcpyAsync(resid_alt, resid + nlock, rem * sizeof(double), cudaMemcpyDeviceToDevice,
                           ctx->stream));
        std::swap(theta, theta_alt);
        std::swap(resid, resid_alt);
        th.erase(th.begin(), th.begin() + nlock);
        rr.erase(rr.begin(), rr.begin() + nlock);
        conv += nlock;
      }
      th.resize(blk - conv);
      rr.resize(blk - conv);
      a0 = th[0];
      a = th[blk - conv - 1];
      // A mixed-precision loop that locked nothing and did not halve the residual of the
      // column blocking the locked prefix has met the precision floor of its products:
      // add two slices, and once the maximum is in use finish with FP64 filters.
      if (mixed && nlock == 0 && !rr.empty() && std::isfinite(front_before) &&
          rr[0] > 0.5 * front_before) {
        if (slices >= o.slices_max) mixed = false;
        else slice_boost += 2;
      }
    }
    if (conv < nev) {
      status = set_err(ctx, CHFSI_ENOCONV, "%d of %d pairs converged after %d loops", conv, nev,
                       st.loops);
      break;
    }
    // ---- a9: back-transform and acceptance on the generalized residual
    {
      PhaseScope ps(ctx, PH_RESID);
      GemmDesc g1 = gd(n, conv, n, ws.Linv, ld, OPC, ws.YL, ld, OPN, ws.Xw, ld);
      g1.triA = 2;
      CKS(gemm_auto(ctx, g1));
      CKS(gemm_auto(ctx, gd(n, nev, n, ws.Af, ld, OPN, ws.Xw, ld, OPN, W, ld)));
      CKS(gemm_auto(ctx, gd(n, nev, n, ws.Bf, ld, OPN, ws.Xw, ld, OPN, Zb, ld)));
      CK(generalized_residuals(W, ld, Zb, ld, ws.Xw, ld, ws.lamL, n, nev, ws.scal + 6, ws.gres,
                               ctx->stream));
    }
    std::vector<double> gr(nev);
    CKS(read_back(ctx, gr.data(), ws.gres, nev));
    max_gres = *std::max_element(gr.begin(), gr.end());
    if (max_gres <= S.tol) break;
    if (accept == 3) {
      // every wanted pair is locked, but the generalized residual stays above tol after the
      // last tightening of the locking threshold: the pairs are returned, flagged
      status = set_err(ctx, CHFSI_ENOCONV,
                       "generalized residual %.3e above tol %.3e after %d tightened locking rounds",
                       max_gres, S.tol, st.accept_rounds);
      break;
    }
    // Tighten the locking threshold and iterate again on all blk columns.
    st.accept_rounds++;
    tau /= 10.0;
    CK(copy_cols(ws.YL, ld, Yb, ld, n, conv, ctx->stream));
    CK(copy_cols(Ya, ld, Yb + (int64_t)conv * ld, ld, n, blk - conv, ctx->stream));
    std::swap(Ya, Yb);
    std::vector<double> th2(lamL);
    th2.insert(th2.end(), th.begin(), th.end());
    std::vector<double> r2(rL);
    r2.insert(r2.end(), rr.begin(), rr.end());
    th = th2;
    rr = r2;
    CK(cudaMemcpyAsync(theta, th.data(), blk * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(resid, rr.data(), blk * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    lamL.clear();
    rL.clear();
    conv = 0;
    a0 = th[0];
    a = th[blk - 1];
  }

  // ---- outputs and warm state: X = L^{-H} [YL, Y_active]
  {
    GemmDesc g1 = gd(n, conv, n, ws.Linv, ld, OPC, ws.YL, ld, OPN, ws.Xw, ld);
    g1.triA = 2;
    CKS(gemm_auto(ctx, g1));
    GemmDesc g2 = gd(n, blk - conv, n, ws.Linv, ld, OPC, Ya, ld, OPN, ws.Xw + (int64_t)conv * ld, ld);
    g2.triA = 2;
    CKS(gemm_auto(ctx, g2));
  }
  std::vector<double> lam_out(nev, NAN);
  for (int i = 0; i < std::min(conv, nev); ++i) lam_out[i] = lamL[i];
  if (S.evals) {
    if (is_device_ptr(S.evals))
      CK(cudaMemcpyAsync(S.evals, lam_out.data(), nev * sizeof(double), cudaMemcpyHostToDevice,
                         ctx->stream));
    else
      std::memcpy(S.evals, lam_out.data(), nev * sizeof(double));
  }
  if (S.evecs) {
    const cudaMemcpyKind kind =
        is_device_ptr(S.evecs) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpy2DAsync(S.evecs, n * sizeof(zd), ws.Xw, ld * sizeof(zd), n * sizeof(zd), nev, kind,
                         ctx->stream));
  }
  ctx->warm_lam = lamL;
  ctx->warm_lam.insert(ctx->warm_lam.end(), th.begin(), th.end());
  ctx->warm_lam.resize(blk);
  ctx->has_warm = (conv == nev);
  ctx->warm_n = n;
  ctx->warm_blk = blk;
  ctx->problems_solved++;
  CK(cudaEventRecord(t_end, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  float tot = 0.f;
  cudaEventElapsedTime(&tot, t_start, t_end);
  collect_times(ctx, tph);
  st.converged = conv;
  st.matvecs += st.filter_matvecs;
  st.launches = g_kernel_launches - launches0;
  st.max_resid = max_gres;
  st.t_reduce_ms = tph[PH_REDUCE];
  st.t_lanczos_ms = tph[PH_LANCZOS];
  st.t_filter_ms = tph[PH_FILTER];
  st.t_qr_ms = tph[PH_QR];
  st.t_rr_ms = tph[PH_RR];
  st.t_resid_ms = tph[PH_RESID];
  st.t_filter_gemm_ms = tph[PH_FGEMM];
  st.t_small_ms = tph[PH_SMALL];
  st.t_eig_ms = tph[PH_EIG];
  st.t_total_ms = tot;
  if (S.st) *S.st = st;
  return status;
}

void debug_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess && std::getenv("CHFSI_DEBUG"))
    std::fprintf(stderr, "[chfsi] %s: %s\n", what, cudaGetErrorString(e));
}

void release_stream(chfsi_ctx* ctx) {
  if (ctx->own_stream && ctx->stream) debug_check(cudaStreamDestroy(ctx->stream), "cudaStreamDestroy");
  ctx->stream = nullptr;
}

// Buffers and stream for staging host inputs ahead of the solve (allocated on first use).
int prefetch_resources(chfsi_ctx* ctx) {
  if (ctx->copy_stream) return CHFSI_OK;
  const size_t bytes = sizeof(zd) * (size_t)ctx->ws.n_max * (size_t)ctx->ws.n_max;
  for (int k = 0; k < 2; ++k)
    for (int j = 0; j < 2; ++j) {
      cudaError_t e = cudaMalloc((void**)&ctx->stage[k][j], bytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, e == cudaErrorMemoryAllocation ? CHFSI_ENOMEM : CHFSI_ECUDA,
                       "staging buffers for host inputs: %s", cudaGetErrorString(e));
      }
    }
  for (int k = 0; k < 2; ++k) CK(cudaEventCreateWithFlags(&ctx->staged[k], cudaEventDisableTiming));
  CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  return CHFSI_OK;
}

void release_prefetch(chfsi_ctx* ctx) {
  if (ctx->copy_stream) debug_check(cudaStreamSynchronize(ctx->copy_stream), "cudaStreamSynchronize");
  for (int k = 0; k < 2; ++k) {
    for (int j = 0; j < 2; ++j)
      if (ctx->stage[k][j]) debug_check(cudaFree(ctx->stage[k][j]), "cudaFree");
    if (ctx->staged[k]) debug_check(cudaEventDestroy(ctx->staged[k]), "cudaEventDestroy");
  }
  if (ctx->copy_stream) debug_check(cudaStreamDestroy(ctx->copy_stream), "cudaStreamDestroy");
  ctx->copy_stream = nullptr;
}

}  // namespace

// ====================================================================== workspace
cudaError_t workspace_alloc(Workspace& ws, int64_t n_max, int blk_max, int lanczos_kmax) {
  ws.n_max = n_max;
  ws.blk_max = std::max(blk_max, NB);
  ws.lanczos_kmax = lanczos_kmax;
  const int64_t nn = n_max * n_max;
  const int64_t nb = n_max * (int64_t)std::max(blk_max, NB);
  const int64_t mm = (int64_t)ws.blk_max * ws.blk_max;
  const int64_t mp = (int64_t)(ws.blk_max + 1);
  cudaError_t e;
#define AL(ptr, count)                                                      \
  do {                                                                      \
    e = cudaMalloc((void**)&(ptr), sizeof(*(ptr)) * (size_t)(count));       \
    if (e != cudaSuccess) return e;                                         \
  } while (0)
  AL(ws.Af, nn); AL(ws.Bf, nn); AL(ws.Lf, nn); AL(ws.Linv, nn); AL(ws.Hs, nn); AL(ws.T, nn);
  AL(ws.Y0, nb); AL(ws.Y1, nb); AL(ws.F, nb); AL(ws.W, nb); AL(ws.YL, nb); AL(ws.Xw, nb); AL(ws.Z, nb);
  AL(ws.G, mm); AL(ws.V, mm); AL(ws.Rt, mm); AL(ws.jac, 3 * mp * mp);
  AL(ws.lv, n_max); AL(ws.lw, n_max); AL(ws.lV, n_max * (lanczos_kmax + 1));
  AL(ws.lc, 2 * (lanczos_kmax + 1));
  AL(ws.theta, ws.blk_max); AL(ws.theta2, ws.blk_max); AL(ws.resid, ws.blk_max);
  AL(ws.resid2, ws.blk_max); AL(ws.lamL, ws.blk_max); AL(ws.residL, ws.blk_max);
  AL(ws.gres, ws.blk_max); AL(ws.dscale, ws.blk_max); AL(ws.scal, 64);
  AL(ws.lal, lanczos_kmax + 1); AL(ws.lbe, lanczos_kmax + 1);
  AL(ws.deg, ws.blk_max); AL(ws.perm, ws.blk_max); AL(ws.degs, ws.blk_max);
  AL(ws.hist_r1, 2 * ws.blk_max); ws.hist_r2 = ws.hist_r1 + ws.blk_max;
  AL(ws.hist_d1, 2 * ws.blk_max); ws.hist_d2 = ws.hist_d1 + ws.blk_max;
  AL(ws.feat, (int64_t)CHFSI_MLP_IN * ws.blk_max); AL(ws.gcorr, ws.blk_max);
  AL(ws.flag, ws.blk_max + 64); AL(ws.ilist, 64);
  AL(ws.status, 2); AL(ws.barrier, 4); AL(ws.shiftflag, 4);
  ws.splitk_elems = (size_t)std::max<int64_t>(8 * nb, 48 * mm);
  AL(ws.splitk, ws.splitk_elems);
#undef AL
  e = oz_alloc(ws.oz, (int)n_max, ws.blk_max, 8);
  if (e != cudaSuccess) return e;
  ws.oz.status = ws.status;
  // pinned mirror for the per-loop read-back: status (2 ints), locked count, theta, r
  ws.host_pinned_bytes = 16 + 2 * sizeof(double) * (size_t)ws.blk_max;
  e = cudaMallocHost(&ws.host_pinned, ws.host_pinned_bytes);
  if (e != cudaSuccess) return e;
  e = cudaMemset(ws.status, 0, 2 * sizeof(int));
  if (e != cudaSuccess) return e;
  const int big = 0x7fffffff;
  e = cudaMemcpy(ws.status + 1, &big, sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  return cudaSuccess;
}

void workspace_free(Workspace& ws) {
  void* ptrs[] = {ws.Af, ws.Bf, ws.Lf, ws.Linv, ws.Hs, ws.T, ws.Y0, ws.Y1, ws.F, ws.W, ws.YL,
                  ws.Xw, ws.Z, ws.G, ws.V, ws.Rt, ws.jac, ws.lv, ws.lw, ws.lV, ws.lc, ws.theta,
                  ws.theta2, ws.resid, ws.resid2, ws.lamL, ws.residL, ws.gres, ws.dscale,
                  ws.scal, ws.lal, ws.lbe, ws.deg, ws.perm, ws.degs, ws.hist_r1, ws.hist_d1,
                  ws.feat, ws.gcorr, ws.flag, ws.ilist,
                  ws.status, ws.shiftflag, ws.barrier, ws.splitk};
  for (void* p : ptrs)
    if (p) debug_check(cudaFree(p), "cudaFree");
  oz_free(ws.oz);
  if (ws.host_pinned) debug_check(cudaFreeHost(ws.host_pinned), "cudaFreeHost");
  ws = Workspace{};
}

// ====================================================================== C ABI
extern "C" {

void chfsi_default_opts(chfsi_opts* o) {
  if (!o) return;
  o->deg_min = 8;
  o->deg_max = 25;
  o->max_loops = 50;
  o->lanczos_k_warm = 10;
  o->lanczos_k_cold = 40;
  o->reuse_factor = 1;
  o->precision = 1;
  o->slices_max = 7;
  o->seed = 12063768ull;
  o->cuda_stream = nullptr;
}

int chfsi_create(chfsi_ctx** out, int64_t n_max, int32_t blk_max, const chfsi_opts* opts) {
  if (!out) return CHFSI_EINVAL;
  *out = nullptr;
  if (n_max <= 0 || blk_max <= 0 || blk_max > n_max || n_max > (int64_t)1 << 30)
    return CHFSI_EINVAL;
  entry_guard("chfsi_create");
  if (opts && (opts->precision < 0 || opts->precision > 1 || opts->slices_max < 1 ||
               opts->slices_max > 8))
    return CHFSI_EINVAL;
  chfsi_ctx* ctx = new chfsi_ctx;
  chfsi_default_opts(&ctx->opts);
  if (opts) ctx->opts = *opts;
  if (cudaGetDevice(&ctx->ws.dev) != cudaSuccess) {
    delete ctx;
    return CHFSI_ECUDA;
  }
  if (ctx->opts.cuda_stream) {
    ctx->stream = (cudaStream_t)ctx->opts.cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return CHFSI_ECUDA;
    }
    ctx->own_stream = true;
  }
  const int kmax = std::max({ctx->opts.lanczos_k_warm, ctx->opts.lanczos_k_cold, 20, 1});
  cudaError_t e = workspace_alloc(ctx->ws, n_max, blk_max, kmax);
  if (e != cudaSuccess) {
    cudaGetLastError();
    workspace_free(ctx->ws);
    release_stream(ctx);
    delete ctx;
    return e == cudaErrorMemoryAllocation ? CHFSI_ENOMEM : CHFSI_ECUDA;
  }
  *out = ctx;
  return CHFSI_OK;
}

void chfsi_destroy(chfsi_ctx* ctx) {
  entry_guard("chfsi_destroy");
  if (!ctx) return;
  debug_check(cudaSetDevice(ctx->ws.dev), "cudaSetDevice");
  if (ctx->stream) debug_check(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  for (auto e : ctx->ev_pool) debug_check(cudaEventDestroy(e), "cudaEventDestroy");
  if (ctx->mlp_dev) debug_check(cudaFree(ctx->mlp_dev), "cudaFree");
  release_prefetch(ctx);
  for (auto& g : ctx->lanczos_graphs) debug_check(cudaGraphExecDestroy(g.exec), "cudaGraphExecDestroy");
  if (ctx->capture_stream) debug_check(cudaStreamDestroy(ctx->capture_stream), "cudaStreamDestroy");
  workspace_free(ctx->ws);
  release_stream(ctx);
  delete ctx;
  cudaGetLastError();
}

const char* chfsi_last_error(const chfsi_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int chfsi_reset_warm_state(chfsi_ctx* ctx) {
  if (!ctx) return CHFSI_EINVAL;
  ctx->has_warm = false;
  ctx->has_factor = false;
  ctx->warm_lam.clear();
  return CHFSI_OK;
}

int chfsi_get_state(chfsi_ctx* ctx, int64_t* n, int32_t* blk, chfsi_z* X, double* lam) {
  entry_guard("chfsi_get_state");
  if (!ctx || !n || !blk) return set_err(ctx, CHFSI_EINVAL, "bad args");
  const bool have = ctx->has_warm && (int)ctx->warm_lam.size() == ctx->warm_blk;
  *n = have ? ctx->warm_n : 0;
  *blk = have ? ctx->warm_blk : 0;
  if (!have) return CHFSI_OK;
  cudaSetDevice(ctx->ws.dev);
  if (X)
    CK(cudaMemcpy2DAsync(X, (size_t)ctx->warm_n * sizeof(zd), ctx->ws.Xw, (size_t)ctx->ws.n_max * sizeof(zd),
                         (size_t)ctx->warm_n * sizeof(zd), (size_t)ctx->warm_blk, cudaMemcpyDefault,
                         ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (lam) std::copy(ctx->warm_lam.begin(), ctx->warm_lam.end(), lam);
  return CHFSI_OK;
}

int chfsi_set_state(chfsi_ctx* ctx, int64_t n, int32_t blk, const chfsi_z* X, int64_t ldx,
                    const double* lam) {
  entry_guard("chfsi_set_state");
  if (!ctx) return CHFSI_EINVAL;
  if (n == 0) {
    ctx->has_warm = false;
    ctx->warm_lam.clear();
    return CHFSI_OK;
  }
  if (n < 0 || n > ctx->ws.n_max || blk < 1 || blk > ctx->ws.blk_max || blk > n || !X || !lam || ldx < n)
    return set_err(ctx, CHFSI_EINVAL, "bad state: n=%lld blk=%d ldx=%lld", (long long)n, blk,
                   (long long)ldx);
  cudaSetDevice(ctx->ws.dev);
  CK(cudaMemcpy2DAsync(ctx->ws.Xw, (size_t)ctx->ws.n_max * sizeof(zd), X, (size_t)ldx * sizeof(zd),
                       (size_t)n * sizeof(zd), (size_t)blk, cudaMemcpyDefault, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->warm_lam.assign(lam, lam + blk);
  ctx->warm_n = n;
  ctx->warm_blk = blk;
  ctx->has_warm = true;
  return CHFSI_OK;
}

int chfsi_solve_next(chfsi_ctx* ctx, int64_t n, const chfsi_z* A, int64_t lda, const chfsi_z* B,
                     int64_t ldb, const chfsi_z* V0, int32_t nev, int32_t blk, int32_t deg,
                     double tol, double* evals, chfsi_z* evecs, chfsi_stats* st) {
  entry_guard("chfsi_solve_next");
  CKS(validate_sizes(ctx, n, nev, blk));
  if (!A || !B || lda < n || ldb < n) return set_err(ctx, CHFSI_EINVAL, "bad A/B arguments");
  if (deg < 0) return set_err(ctx, CHFSI_EINVAL, "deg must be >= 0");
  cudaSetDevice(ctx->ws.dev);
  SolveArgs S{(int)n, nev, blk, deg, tol, A, B, V0, lda, ldb, evals, evecs, st};
  return solve_one(ctx, S);
}

int chfsi_solve_sequence(chfsi_ctx* ctx, int32_t N, int64_t n, const chfsi_z* const* A,
                         const chfsi_z* const* B, int64_t ld, const chfsi_z* V0, int32_t nev,
                         int32_t blk, int32_t deg, double tol, double* evals,
                         chfsi_z* const* evecs, chfsi_stats* st) {
  CKS(validate_sizes(ctx, n, nev, blk));
  if (N <= 0 || !A || !B || !evals) return set_err(ctx, CHFSI_EINVAL, "bad sequence arguments");
  if (ld < n) return set_err(ctx, CHFSI_EINVAL, "ld < n");
  entry_guard("chfsi_solve_sequence");
  cudaSetDevice(ctx->ws.dev);
  bool host_in = false;
  for (int l = 0; l < N && !host_in; ++l) host_in = !is_device_ptr(A[l]) || !is_device_ptr(B[l]);
  if (host_in) CKS(prefetch_resources(ctx));
  const int64_t lds = ctx->ws.n_max;
  // queue the copies of problem l's host matrices into buffer pair l & 1
  auto stage = [&](int l) -> int {
    const int k = l & 1;
    const chfsi_z* src[2] = {A[l], B[l]};
    for (int j = 0; j < 2; ++j)
      if (!is_device_ptr(src[j]))
        CK(cudaMemcpy2DAsync(ctx->stage[k][j], lds * sizeof(zd), src[j], ld * sizeof(zd), n * sizeof(zd), n,
                             cudaMemcpyHostToDevice, ctx->copy_stream));
    CK(cudaEventRecord(ctx->staged[k], ctx->copy_stream));
    return CHFSI_OK;
  };
  if (host_in) CKS(stage(0));
  for (int l = 0; l < N; ++l) {
    const chfsi_z* Al = A[l];
    const chfsi_z* Bl = B[l];
    int64_t lda = ld, ldb = ld;
    if (host_in) {
      // buffer pair (l + 1) & 1 was read by problem l - 1, which has finished
      if (l + 1 < N) CKS(stage(l + 1));
      const int k = l & 1;
      CK(cudaStreamWaitEvent(ctx->stream, ctx->staged[k], 0));
      if (!is_device_ptr(Al)) { Al = reinterpret_cast<const chfsi_z*>(ctx->stage[k][0]); lda = lds; }
      if (!is_device_ptr(Bl)) { Bl = reinterpret_cast<const chfsi_z*>(ctx->stage[k][1]); ldb = lds; }
    }
    const int rc = chfsi_solve_next(ctx, n, Al, lda, Bl, ldb, l == 0 ? V0 : nullptr, nev, blk,
                                    deg, tol, evals + (int64_t)l * nev,
                                    evecs ? evecs[l] : nullptr, st ? st + l : nullptr);
    if (rc != CHFSI_OK) {
      if (host_in) debug_check(cudaStreamSynchronize(ctx->copy_stream), "cudaStreamSynchronize");
      return rc;
    }
  }
  return CHFSI_OK;
}

// ---------------------------------------------------------------- step entry points
int chfsi_cholesky(chfsi_ctx* ctx, int64_t n, const chfsi_z* B, int64_t ldb, chfsi_z* L,
                   int64_t ldl) {
  entry_guard("chfsi_cholesky");
  if (!ctx || !B || !L || n <= 0 || ldb < n || ldl < n) return set_err(ctx, CHFSI_EINVAL, "bad args");
  if (n > ctx->ws.n_max) return set_err(ctx, CHFSI_EINVAL, "n > n_max");
  cudaSetDevice(ctx->ws.dev);
  CKS(reset_status(ctx));
  CK(cudaMemcpy2DAsync(L, ldl * sizeof(zd), B, ldb * sizeof(zd), n * sizeof(zd), n,
                       cudaMemcpyDeviceToDevice, ctx->stream));
  CKS(blocked_cholesky(ctx, Z(L), ldl, (int)n));
  CK(cudaStreamSynchronize(ctx->stream));
  return check_status(ctx, "chfsi_cholesky");
}

int chfsi_reduce(chfsi_ctx* ctx, int64_t n, const chfsi_z* A, int64_t lda, const chfsi_z* L,
                 int64_t ldl, chfsi_z* Hs, int64_t ldh) {
  entry_guard("chfsi_reduce");
  if (!ctx || !A || !L || !Hs || n <= 0 || lda < n || ldl < n || ldh < n)
    return set_err(ctx, CHFSI_EINVAL, "bad args");
  if (n > ctx->ws.n_max) return set_err(ctx, CHFSI_EINVAL, "n > n_max");
  cudaSetDevice(ctx->ws.dev);
  CKS(reset_status(ctx));
  Workspace& ws = ctx->ws;
  CKS(blocked_trinv(ctx, Z(L), ldl, ws.Linv, ws.n_max, (int)n));
  CK(herm_from_lower(Z(A), lda, ws.Af, ws.n_max, (int)n, ws.status, ctx->stream));
  CKS(reduce_to_standard(ctx, ws.Af, ws.n_max, ws.Linv, ws.n_max, Z(Hs), ldh, (int)n,
                         ctx->opts.precision == 1));
  ctx->has_factor = false;  // ws.Linv no longer matches ws.Bf
  CK(cudaStreamSynchronize(ctx->stream));
  return check_status(ctx, "chfsi_reduce");
}

int chfsi_lanczos(chfsi_ctx* ctx, int64_t n, const chfsi_z* H, int64_t ldh, int32_t k,
                  const chfsi_z* v0, double* upper, double* theta_min, double* theta_max) {
  entry_guard("chfsi_lanczos");
  if (!ctx || !H || n <= 0 || ldh < n || k <= 0) return set_err(ctx, CHFSI_EINVAL, "bad args");
  if (n > ctx->ws.n_max) return set_err(ctx, CHFSI_EINVAL, "n > n_max");
  if (k > ctx->ws.lanczos_kmax)
    return set_err(ctx, CHFSI_EINVAL, "k=%d above the context's Lanczos limit %d", k,
                   ctx->ws.lanczos_kmax);
  cudaSetDevice(ctx->ws.dev);
  double out[3];
  CKS(lanczos_issue(ctx, ctx->stream, Z(H), ldh, (int)n, k, Z(v0), ctx->opts.seed, ctx->ws.scal));
  CKS(read_back(ctx, out, ctx->ws.scal, 3));
  if (theta_min) *theta_min = out[0];
  if (theta_max) *theta_max = out[1];
  if (upper) *upper = out[2];
  return CHFSI_OK;
}

int chfsi_filter(chfsi_ctx* ctx, int64_t n, int32_t m, const chfsi_z* H, int64_t ldh, chfsi_z* Y,
                 int64_t ldy, const int32_t* degrees, double a0, double a, double b) {
  entry_guard("chfsi_filter");
  if (!ctx || !H || !Y || !degrees || n <= 0 || m <= 0 || ldh < n || ldy < n)
    return set_err(ctx, CHFSI_EINVAL, "bad args");
  if (n > ctx->ws.n_max || m > ctx->ws.blk_max) return set_err(ctx, CHFSI_EINVAL, "size > workspace");
  if (!(b > a)) return set_err(ctx, CHFSI_EINVAL, "need b > a");
  cudaSetDevice(ctx->ws.dev);
  Workspace& ws = ctx->ws;
  const int64_t ld = ws.n_max;
  std::vector<int> idx(m);
  std::iota(idx.begin(), idx.end(), 0);
  for (int j = 0; j < m; ++j)
    if (degrees[j] < 0) return set_err(ctx, CHFSI_EINVAL, "negative degree");
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return degrees[x] > degrees[y]; });
  std::vector<int> ds(m), inv(m);
  for (int r = 0; r < m; ++r) { ds[r] = degrees[idx[r]]; inv[idx[r]] = r; }
  CK(cudaMemcpy2DAsync(ws.Y0, ld * sizeof(zd), Y, ldy * sizeof(zd), n * sizeof(zd), m,
                       cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ws.perm, idx.data(), m * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  zd *Ya = ws.Y0, *Yb = ws.Y1, *Yf = ws.F;
  CKS(filter_block(ctx, Z(H), ldh, (int)n, m, &Ya, &Yb, &Yf, ds, ws.perm, a0, a, b, nullptr));
  // undo the permutation: Y[:, j] = Ya[:, inv[j]]
  CK(cudaMemcpyAsync(ws.deg, inv.data(), m * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  CK(gather_cols(Ya, ld, Yb, ld, (int)n, m, ws.deg, ctx->stream));
  CK(cudaMemcpy2DAsync(Y, ldy * sizeof(zd), Yb, ld * sizeof(zd), n * sizeof(zd), m,
                       cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CHFSI_OK;
}

int chfsi_filter_split(chfsi_ctx* ctx, int64_t n, int32_t m, const chfsi_z* H, int64_t ldh,
                       chfsi_z* Y, int64_t ldy, const int32_t* degrees, double a0, double a,
                       double b, int32_t slices) {
  entry_guard("chfsi_filter_split");
  if (!ctx || !H || !Y || !degrees || n <= 0 || m <= 0 || ldh < n || ldy < n || slices < 1 ||
      slices > 8)
    return set_err(ctx, CHFSI_EINVAL, "bad args");
  if (n > ctx->ws.n_max || m > ctx->ws.blk_max) return set_err(ctx, CHFSI_EINVAL, "size > workspace");
  if (!(b > a)) return set_err(ctx, CHFSI_EINVAL, "need b > a");
  cudaSetDevice(ctx->ws.dev);
  Workspace& ws = ctx->ws;
  const int64_t ld = ws.n_max;
  std::vector<int> idx(m);
  std::iota(idx.begin(), idx.end(), 0);
  for (int j = 0; j < m; ++j)
    if (degrees[j] < 0) return set_err(ctx, CHFSI_EINVAL, "negative degree");
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return degrees[x] > degrees[y]; });
  std::vector<int> ds(m), inv(m);
  for (int r = 0; r < m; ++r) { ds[r] = degrees[idx[r]]; inv[idx[r]] = r; }
  CKS(reset_status(ctx));
  CK(oz_slice_hermitian(Z(H), ldh, (int)n, slices, ws.oz, ctx->stream));
  CK(cudaMemcpy2DAsync(ws.Y0, ld * sizeof(zd), Y, ldy * sizeof(zd), n * sizeof(zd), m,
                       cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ws.perm, idx.data(), m * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  zd *Ya = ws.Y0, *Yb = ws.Y1, *Yf = ws.F;
  CKS(filter_block(ctx, Z(H), ldh, (int)n, m, &Ya, &Yb, &Yf, ds, ws.perm, a0, a, b, nullptr, slices));
  CK(cudaMemcpyAsync(ws.deg, inv.data(), m * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  CK(gather_cols(Ya, ld, Yb, ld, (int)n, m, ws.deg, ctx->stream));
  CK(cudaMemcpy2DAsync(Y, ldy * sizeof(zd), Yb, ld * sizeof(zd), n * sizeof(zd), m,
                       cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return check_status(ctx, "chfsi_filter_split");
}

int chfsi_set_wait_limit(chfsi_ctx* ctx, int64_t polls) {
  if (!ctx || polls < 0) return set_err(ctx, CHFSI_EINVAL, "polls must be >= 0");
  ctx->ws.wait_limit = polls;
  ctx->ws.oz.wait_limit = polls;
  return CHFSI_OK;
}

int chfsi_orthonormalize(chfsi_ctx* ctx, int64_t n, int32_t m, chfsi_z* Y, int64_t ldy, int32_t k,
                         const chfsi_z* YL, int64_t ldyl) {
  entry_guard("chfsi_orthonormalize");
  if (!ctx || !Y || n <= 0 || m <= 0 || ldy < n || k < 0 || (k > 0 && (!YL || ldyl < n)))
    return set_err(ctx, CHFSI_EINVAL, "bad args");
  if (n > ctx->ws.n_max || m > ctx->ws.blk_max || k > ctx->ws.blk_max || m + k > n)
    return set_err(ctx, CHFSI_EINVAL, "size > workspace");
  cudaSetDevice(ctx->ws.dev);
  CKS(reset_status(ctx));
  Workspace& ws = ctx->ws;
  const int64_t ld = ws.n_max;
  CK(cudaMemcpy2DAsync(ws.Y0, ld * sizeof(zd), Y, ldy * sizeof(zd), n * sizeof(zd), m,
                       cudaMemcpyDeviceToDevice, ctx->stream));
  zd *Ya = ws.Y0, *Yb = ws.Y1;
  CKS(orthonormalize_block(ctx, (int)n, m, &Ya, &Yb, Z(YL), ldyl, k));
  CK(cudaMemcpy2DAsync(Y, ldy * sizeof(zd), Ya, ld * sizeof(zd), n * sizeof(zd), m,
                       cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return check_status(ctx, "chfsi_orthonormalize");
}

int chfsi_rayleigh_ritz(chfsi_ctx* ctx, int64_t n, int32_t m, const chfsi_z* H, int64_t ldh,
                        chfsi_z* Y, int64_t ldy, chfsi_z* HY, int64_t ldhy, double* theta) {
  entry_guard("chfsi_rayleigh_ritz");
  if (!ctx || !H || !Y || !HY || !theta || n <= 0 || m <= 0 || ldh < n || ldy < n || ldhy < n)
    return set_err(ctx, CHFSI_EINVAL, "bad args");
  if (n > ctx->ws.n_max || m > ctx->ws.blk_max) return set_err(ctx, CHFSI_EINVAL, "size > workspace");
  cudaSetDevice(ctx->ws.dev);
  CKS(reset_status(ctx));
  Workspace& ws = ctx->ws;
  const int64_t ld = ws.n_max;
  CK(cudaMemcpy2DAsync(ws.Y0, ld * sizeof(zd), Y, ldy * sizeof(zd), n * sizeof(zd), m,
                       cudaMemcpyDeviceToDevice, ctx->stream));
  zd *Ya = ws.Y0, *Yb = ws.Y1, *W = ws.W, *Zb = ws.Z;
  int rr_slices = 0;
  if (ctx->opts.precision == 1) {
    rr_slices = kProductSlices;
    CK(oz_slice_hermitian(Z(H), ldh, (int)n, rr_slices, ws.oz, ctx->stream));
  }
  CKS(rayleigh_ritz_block(ctx, Z(H), ldh, (int)n, m, &Ya, &Yb, &W, &Zb, theta, rr_slices));
  CK(cudaMemcpy2DAsync(Y, ldy * sizeof(zd), Ya, ld * sizeof(zd), n * sizeof(zd), m,
                       cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaMemcpy2DAsync(HY, ldhy * sizeof(zd), W, ld * sizeof(zd), n * sizeof(zd), m,
                       cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return check_status(ctx, "chfsi_rayleigh_ritz");
}

int chfsi_residuals(chfsi_ctx* ctx, int64_t n, int32_t m, const chfsi_z* HY, int64_t ldhy,
                    const chfsi_z* Y, int64_t ldy, const double* theta, double* r) {
  entry_guard("chfsi_residuals");
  if (!ctx || !HY || !Y || !theta || !r || n <= 0 || m <= 0 || ldhy < n || ldy < n)
    return set_err(ctx, CHFSI_EINVAL, "bad args");
  cudaSetDevice(ctx->ws.dev);
  CK(column_residuals(Z(HY), ldhy, Z(Y), ldy, theta, (int)n, m, r, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CHFSI_OK;
}

int chfsi_degrees(chfsi_ctx* ctx, int32_t m, const double* theta, const double* r, double a,
                  double b, double tau, int32_t dmin, int32_t dmax, int32_t n_wanted,
                  int32_t* degrees) {
  entry_guard("chfsi_degrees");
  if (!ctx || !theta || !r || !degrees || m <= 0 || dmin < 0 || dmax < dmin || !(b > a) || n_wanted < 0)
    return set_err(ctx, CHFSI_EINVAL, "bad args");
  if (m > ctx->ws.blk_max) return set_err(ctx, CHFSI_EINVAL, "m > blk_max");
  cudaSetDevice(ctx->ws.dev);
  const float* gcorr = nullptr;
  if (ctx->mlp_on) {
    // the model without residual history (as in the first loop of a problem)
    CK(degree_features(theta, r, m, a, b, tau, 0, nullptr, nullptr, nullptr, nullptr, ctx->ws.feat,
                       ctx->stream));
    CK(degree_model_eval(ctx->mlp_dev, ctx->ws.feat, m, ctx->ws.gcorr, ctx->stream));
    gcorr = ctx->ws.gcorr;
  }
  CK(degrees_kernel_run(theta, r, m, a, b, tau, dmin, dmax, n_wanted, degrees, ctx->ws.perm,
                        ctx->ws.degs, ctx->stream, gcorr));
  CK(cudaStreamSynchronize(ctx->stream));
  return CHFSI_OK;
}

int chfsi_mlp_train(chfsi_ctx* ctx, chfsi_mlp* model, const float* X, const float* z, int64_t n,
                    int32_t epochs, int32_t batch, float lr, uint64_t seed, float* loss) {
  entry_guard("chfsi_mlp_train");
  if (!ctx || !model || !X || !z || n <= 0 || n > (int64_t)1 << 30 || epochs < 0 || batch < 1 || !(lr > 0.f))
    return set_err(ctx, CHFSI_EINVAL, "bad args");
  cudaSetDevice(ctx->ws.dev);
  CK(mlp_train(model, X, z, n, epochs, batch, lr, seed, loss, ctx->stream));
  return CHFSI_OK;
}

int chfsi_mlp_gradient(chfsi_ctx* ctx, const chfsi_mlp* model, const float* X, const float* z,
                       int64_t n, float* grad, float* loss) {
  entry_guard("chfsi_mlp_gradient");
  if (!ctx || !model || !X || !z || !grad || !loss || n <= 0 || n > (int64_t)1 << 30)
    return set_err(ctx, CHFSI_EINVAL, "bad args");
  cudaSetDevice(ctx->ws.dev);
  CK(mlp_gradient(model, X, z, n, grad, loss, ctx->stream));
  return CHFSI_OK;
}

int chfsi_mlp_predict(chfsi_ctx* ctx, const chfsi_mlp* model, const float* X, int64_t n, float* y) {
  entry_guard("chfsi_mlp_predict");
  if (!ctx || !model || !X || !y || n <= 0 || n > (int64_t)1 << 30) return set_err(ctx, CHFSI_EINVAL, "bad args");
  cudaSetDevice(ctx->ws.dev);
  CK(mlp_predict(model, X, n, y, ctx->stream));
  return CHFSI_OK;
}

int chfsi_mlp_adam_epoch(chfsi_ctx* ctx, chfsi_mlp* model, float* m1, float* m2, int32_t* step,
                         const float* X, const float* z, const int32_t* order, int64_t n, int32_t batch,
                         float lr, float* loss) {
  entry_guard("chfsi_mlp_adam_epoch");
  if (!ctx || !model || !m1 || !m2 || !step || !X || !z || !order || !loss || n <= 0 ||
      n > (int64_t)1 << 30 || batch < 1 || !(lr >= 0.f))
    return set_err(ctx, CHFSI_EINVAL, "bad args");
  for (int64_t i = 0; i < n; ++i)
    if (order[i] < 0 || order[i] >= n) return set_err(ctx, CHFSI_EINVAL, "order out of range");
  cudaSetDevice(ctx->ws.dev);
  CK(mlp_adam_epoch(model, m1, m2, step, X, z, order, n, batch, lr, loss, ctx->stream));
  return CHFSI_OK;
}

int chfsi_set_degree_model(chfsi_ctx* ctx, const chfsi_mlp* model) {
  entry_guard("chfsi_set_degree_model");
  if (!ctx) return CHFSI_EINVAL;
  cudaSetDevice(ctx->ws.dev);
  if (!model) {
    ctx->mlp_on = false;
    return CHFSI_OK;
  }
  if (!ctx->mlp_dev) CK(cudaMalloc((void**)&ctx->mlp_dev, sizeof(__half) * (mlp_param_count() + 2 * CHFSI_MLP_IN)));
  CK(mlp_to_half(model, ctx->mlp_dev, ctx->stream));
  ctx->mlp_on = true;
  return CHFSI_OK;
}

int chfsi_degree_log_start(chfsi_ctx* ctx, int64_t capacity) {
  if (!ctx || capacity < 0) return CHFSI_EINVAL;
  ctx->deglog.clear();
  ctx->deglog_cap = capacity;
  return CHFSI_OK;
}

int64_t chfsi_degree_log_read(chfsi_ctx* ctx, double* out, int64_t cap) {
  if (!ctx) return -1;
  const int64_t cnt = (int64_t)ctx->deglog.size() / CHFSI_DEGREE_LOG_FIELDS;
  if (out && cap > 0)
    std::memcpy(out, ctx->deglog.data(), sizeof(double) * CHFSI_DEGREE_LOG_FIELDS * std::min(cap, cnt));
  return cnt;
}

int chfsi_deviation_angles(chfsi_ctx* ctx, int64_t n, int32_t k, const chfsi_z* X_prev, int64_t ldp,
                           const chfsi_z* X_cur, int64_t ldc, const chfsi_z* B, int64_t ldb,
                           double* theta, int32_t* assoc) {
  entry_guard("chfsi_deviation_angles");
  if (!ctx || !X_prev || !X_cur || !B || !theta || !assoc || n <= 0 || k <= 0 || k > n || ldp < n ||
      ldc < n || ldb < n)
    return set_err(ctx, CHFSI_EINVAL, "bad args");
  Workspace& ws = ctx->ws;
  if (n > ws.n_max || k > ws.blk_max) return set_err(ctx, CHFSI_EINVAL, "n > n_max or k > blk_max");
  cudaSetDevice(ws.dev);
  CKS(reset_status(ctx));
  const int64_t ld = ws.n_max, ldm = ws.blk_max;
  const int ni = (int)n;
  // Hermitian completion of B in the product scratch (not ws.Bf, which keys the reuse of L)
  CK(herm_from_lower(Z(B), ldb, ws.T, ld, ni, ws.status, ctx->stream));
  CKS(gemm_auto(ctx, gd(ni, k, ni, ws.T, ld, OPN, Z(X_cur), ldc, OPN, ws.W, ld)));
  CKS(gemm_auto(ctx, gd(ni, k, ni, ws.T, ld, OPN, Z(X_prev), ldp, OPN, ws.Z, ld)));
  CKS(gemm_auto(ctx, gd(k, k, ni, Z(X_prev), ldp, OPC, ws.W, ld, OPN, ws.G, ldm)));
  CK(bnorms(Z(X_prev), ldp, ws.Z, ld, ni, k, ws.resid, ctx->stream));
  CK(bnorms(Z(X_cur), ldc, ws.W, ld, ni, k, ws.resid2, ctx->stream));
  CK(associate(ws.G, ldm, k, assoc, ctx->stream));
  CK(deviation_residual(Z(X_prev), ldp, Z(X_cur), ldc, ws.G, ldm, ws.resid, ws.resid2, assoc, ni, k,
                        ws.F, ld, ctx->stream));
  CKS(gemm_auto(ctx, gd(ni, k, ni, ws.T, ld, OPN, ws.F, ld, OPN, ws.Y0, ld)));
  CK(deviation_theta(ws.F, ld, ws.Y0, ld, ni, k, theta, ctx->stream));
  return check_status(ctx, "chfsi_deviation_angles");
}

int chfsi_heev(chfsi_ctx* ctx, int32_t m, const chfsi_z* G, int64_t ldg, double* w, chfsi_z* V,
               int64_t ldv) {
  entry_guard("chfsi_heev");
  if (!ctx || !G || !w || !V || m <= 0 || ldg < m || ldv < m) return set_err(ctx, CHFSI_EINVAL, "bad args");
  if (m > ctx->ws.blk_max) return set_err(ctx, CHFSI_EINVAL, "m > blk_max");
  cudaSetDevice(ctx->ws.dev);
  CKS(reset_status(ctx));
  CK(jacobi_heev(Z(G), ldg, m, w, Z(V), ldv, ctx->ws.jac, ctx->ws.barrier, ctx->ws.status,
                 ctx->stream, ctx->ws.wait_limit));
  CK(cudaStreamSynchronize(ctx->stream));
  return check_status(ctx, "chfsi_heev");
}

int chfsi_heev_df(chfsi_ctx* ctx, int32_t m, const chfsi_z* G, int64_t ldg, double* w, chfsi_z* V,
                  int64_t ldv) {
  entry_guard("chfsi_heev_df");
  if (!ctx || !G || !w || !V || m <= 0 || ldg < m || ldv < m) return set_err(ctx, CHFSI_EINVAL, "bad args");
  if (m > ctx->ws.blk_max) return set_err(ctx, CHFSI_EINVAL, "m > blk_max");
  cudaSetDevice(ctx->ws.dev);
  CKS(reset_status(ctx));
  CK(jacobi_heev_df(Z(G), ldg, m, w, Z(V), ldv, ctx->ws.jac, ctx->ws.barrier, ctx->ws.status,
                    ctx->stream, ctx->ws.wait_limit));
  CK(cudaStreamSynchronize(ctx->stream));
  return check_status(ctx, "chfsi_heev_df");
}

int chfsi_zgemm(chfsi_ctx* ctx, char opa, char opb, int32_t M, int32_t N, int32_t K, double alpha,
                const chfsi_z* A, int64_t lda, const chfsi_z* B, int64_t ldb, double beta,
                chfsi_z* C, int64_t ldc) {
  entry_guard("chfsi_zgemm");
  if (!ctx || !C || M < 0 || N < 0 || K < 0 || (K > 0 && (!A || !B)))
    return set_err(ctx, CHFSI_EINVAL, "bad args");
  const int oA = (opa == 'C' || opa == 'c') ? OPC : OPN;
  const int oB = (opb == 'C' || opb == 'c') ? OPC : OPN;
  if ((oA == OPN && lda < M) || (oA == OPC && lda < K) || (oB == OPN && ldb < K) ||
      (oB == OPC && ldb < N) || ldc < M)
    return set_err(ctx, CHFSI_EINVAL, "bad leading dimension");
  cudaSetDevice(ctx->ws.dev);
  GemmDesc g = gd(M, N, K, Z(A), lda, oA, Z(B), ldb, oB, Z(C), ldc, alpha);
  if (beta != 0.0) { g.beta = beta; g.Cin = Z(C); g.ldcin = ldc; }
  CKS(gemm(ctx, g));
  CK(cudaStreamSynchronize(ctx->stream));
  return CHFSI_OK;
}

}  // extern "C"
