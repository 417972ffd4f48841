// Bandwidth-bound and bookkeeping kernels of the solver: Hermitian completion of the
// lower-triangle inputs, column copies and gathers, residual norms of the locking test,
// locking prefix scan, per-vector degrees, the SplitMix64 start vectors, and the pieces
// of the Lanczos bound (row-dot Hermitian matrix-vector product, block dot products,
// tridiagonal extreme eigenvalues by Sturm bisection).
#include <algorithm>
#include <cmath>

#include "internal.cuh"

namespace {

constexpr int TILE = 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum (blockDim.x a multiple of 32, <= 1024).  All threads get the result.
__device__ double block_sum(double v) {
  __shared__ double sh[32];
  __shared__ double total;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) total = t;
  }
  __syncthreads();
  const double r = total;
  __syncthreads();
  return r;
}

// dst = Hermitian completion of the lower triangle of src (32 x 32 tiles through shared
// memory so both the direct and the transposed reads are coalesced).
__global__ void herm_from_lower_kernel(const zd* src, int64_t lds, zd* dst, int64_t ldd, int n,
                                       int* status) {
  __shared__ zd tile[TILE][TILE + 1];
  const int bi = blockIdx.x * TILE, bj = blockIdx.y * TILE;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  int bad = 0;
  if (bi >= bj) {  // tile on or below the diagonal: copy (upper part of diagonal tiles below)
    for (int r = ty; r < TILE; r += 8) {
      const int i = bi + tx, j = bj + r;
      if (i < n && j < n) {
        zd v = src[i + (int64_t)j * lds];
        bad |= (i >= j) && !(isfinite(v.x) && isfinite(v.y));
        tile[r][tx] = v;
      }
    }
    __syncthreads();
    for (int r = ty; r < TILE; r += 8) {
      const int i = bi + tx, j = bj + r;
      if (i < n && j < n) {
        zd v;
        if (i > j) v = tile[r][tx];
        else if (i == j) v = zmk(tile[r][tx].x, 0.0);
        else v = zconj(tile[tx][r]);  // (i, j) upper within a diagonal tile: conj(src(j, i))
        dst[i + (int64_t)j * ldd] = v;
      }
    }
  } else {  // strictly upper tile: dst(i, j) = conj(src(j, i)); read the mirrored tile
    for (int r = ty; r < TILE; r += 8) {
      const int i = bj + tx, j = bi + r;  // src rows from column block bj... (j, i) pairs
      if (i < n && j < n) tile[r][tx] = src[i + (int64_t)j * lds];
    }
    __syncthreads();
    for (int r = ty; r < TILE; r += 8) {
      const int i = bi + tx, j = bj + r;
      if (i < n && j < n) dst[i + (int64_t)j * ldd] = zconj(tile[tx][r]);
    }
  }
  if (bad) atomicOr(status, DEV_NAN);
}

// In place: H(i, j) = conj(H(j, i)) for i < j, imaginary part of the diagonal dropped.
__global__ void mirror_lower_kernel(zd* H, int64_t ldh, int n) {
  __shared__ zd tile[TILE][TILE + 1];
  const int bi = blockIdx.x * TILE, bj = blockIdx.y * TILE;
  const int tx = threadIdx.x, ty = threadIdx.y;
  if (bi > bj) return;  // only tiles on or above the diagonal are written
  // read the mirrored (lower) tile: rows bj.., cols bi..
  for (int r = ty; r < TILE; r += 8) {
    const int i = bj + tx, j = bi + r;
    if (i < n && j < n) tile[r][tx] = H[i + (int64_t)j * ldh];
  }
  __syncthreads();
  for (int r = ty; r < TILE; r += 8) {
    const int i = bi + tx, j = bj + r;
    if (i < n && j < n) {
      if (i < j) H[i + (int64_t)j * ldh] = zconj(tile[tx][r]);
      else if (i == j) H[i + (int64_t)j * ldh] = zmk(tile[tx][r].x, 0.0);
    }
  }
}

// H <- H + H^H in place (H full, n x n), exactly Hermitian: the CTA of a tile pair (I, J),
// I >= J, reads both tiles and writes both (a diagonal tile alone), so no entry is read after
// another CTA wrote it.
__global__ void herm_sum_kernel(zd* H, int64_t ldh, int n) {
  __shared__ zd lo[TILE][TILE + 1];  // tile (I, J): rows bi.., cols bj..
  __shared__ zd up[TILE][TILE + 1];  // tile (J, I): rows bj.., cols bi..
  const int bi = blockIdx.x * TILE, bj = blockIdx.y * TILE;
  const int tx = threadIdx.x, ty = threadIdx.y;
  if (bi < bj) return;
  for (int r = ty; r < TILE; r += 8) {
    const int i = bi + tx, j = bj + r;
    if (i < n && j < n) lo[r][tx] = H[i + (int64_t)j * ldh];
    const int i2 = bj + tx, j2 = bi + r;
    if (i2 < n && j2 < n) up[r][tx] = H[i2 + (int64_t)j2 * ldh];
  }
  __syncthreads();
  // S(i, j) = H(i, j) + conj(H(j, i)); lo[r][tx] = H(bi + tx, bj + r), up[tx][r] = H(bj + r, bi + tx)
  for (int r = ty; r < TILE; r += 8) {
    const int i = bi + tx, j = bj + r;
    if (i < n && j < n) {
      zd v = zadd(lo[r][tx], zconj(up[tx][r]));
      if (i == j) v.y = 0.0;
      H[i + (int64_t)j * ldh] = v;
      if (bi != bj) H[j + (int64_t)i * ldh] = zconj(v);
    }
  }
}

__global__ void zero_upper_kernel(zd* L, int64_t ldl, int n) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (i < j) L[i + (int64_t)j * ldl] = zmk(0.0, 0.0);
  }
}

// out[0] = max_i |L_ii|^2, out[1] = min_i |L_ii|^2 (one CTA): a lower bound of cond(L L^H).
__global__ void diag_ratio_kernel(const zd* L, int64_t ldl, int n, double* out) {
  __shared__ double mx[256], mn[256];
  double a = 0.0, b = INFINITY;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double d = zabs2(L[i + (int64_t)i * ldl]);
    a = fmax(a, d);
    b = fmin(b, d);
  }
  mx[threadIdx.x] = a;
  mn[threadIdx.x] = b;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      mx[threadIdx.x] = fmax(mx[threadIdx.x], mx[threadIdx.x + o]);
      mn[threadIdx.x] = fmin(mn[threadIdx.x], mn[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = mx[0];
    out[1] = mn[0];
  }
}

__global__ void copy_cols_kernel(const zd* src, int64_t lds, zd* dst, int64_t ldd, int n, int m,
                                 const int* perm, const int* flag) {
  const int64_t total = (int64_t)n * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (flag && !flag[j]) continue;
    const int sj = perm ? perm[j] : j;
    dst[i + (int64_t)j * ldd] = src[i + (int64_t)sj * lds];
  }
}

__global__ void compare_kernel(const zd* a, int64_t lda, const zd* b, int64_t ldb, int n, int m,
                               int* diff) {
  const int64_t total = (int64_t)n * m;
  int d = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (i < j) continue;  // lower triangle only
    const zd x = a[i + (int64_t)j * lda], y = b[i + (int64_t)j * ldb];
    d |= (__double_as_longlong(x.x) != __double_as_longlong(y.x)) ||
         (__double_as_longlong(x.y) != __double_as_longlong(y.y));
  }
  if (__any_sync(0xffffffffu, d) && (threadIdx.x & 31) == 0) atomicOr(diff, 1);
}

// r_j = ||HY_j - theta_j Y_j|| / ||Y_j||, one CTA per column (fixed reduction order).
__global__ void column_residuals_kernel(const zd* HY, int64_t ldhy, const zd* Y, int64_t ldy,
                                        const double* theta, int n, double* r) {
  const int j = blockIdx.x;
  const double th = theta[j];
  double num = 0.0, den = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const zd y = Y[i + (int64_t)j * ldy];
    const zd h = HY[i + (int64_t)j * ldhy];
    const zd d = zmk(h.x - th * y.x, h.y - th * y.y);
    num += zabs2(d);
    den += zabs2(y);
  }
  num = block_sum(num);
  den = block_sum(den);
  if (threadIdx.x == 0) r[j] = sqrt(num) / sqrt(den);
}

// theta_j = Re(y_j^H (H y_j)) / (y_j^H y_j): the Rayleigh quotient of column j.
__global__ void rayleigh_quotients_kernel(const zd* HY, int64_t ldhy, const zd* Y, int64_t ldy, int n,
                                          double* theta) {
  const int j = blockIdx.x;
  double num = 0.0, den = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const zd y = Y[i + (int64_t)j * ldy];
    const zd h = HY[i + (int64_t)j * ldhy];
    num += y.x * h.x + y.y * h.y;
    den += zabs2(y);
  }
  num = block_sum(num);
  den = block_sum(den);
  if (threadIdx.x == 0) theta[j] = num / den;
}

// ||AX_j - lam_j BX_j|| / (a_norm ||X_j||)
__global__ void gen_residuals_kernel(const zd* AX, int64_t ldax, const zd* BX, int64_t ldbx,
                                     const zd* X, int64_t ldx, const double* lam, int n,
                                     const double* a_norm, double* r) {
  const int j = blockIdx.x;
  const double l = lam[j];
  double num = 0.0, den = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const zd a = AX[i + (int64_t)j * ldax], b = BX[i + (int64_t)j * ldbx];
    const zd x = X[i + (int64_t)j * ldx];
    const zd d = zmk(a.x - l * b.x, a.y - l * b.y);
    num += zabs2(d);
    den += zabs2(x);
  }
  num = block_sum(num);
  den = block_sum(den);
  if (threadIdx.x == 0) r[j] = sqrt(num) / (a_norm[0] * sqrt(den));
}

// ---------------------------------------------------------------- SplitMix64
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed,
                                                         unsigned long long idx) {
  unsigned long long z = seed + (idx + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double u01(unsigned long long seed, unsigned long long idx) {
  return (double)(splitmix64(seed, idx) >> 11) * 0x1.0p-53;
}

__global__ void start_vector_kernel(zd* v, int n, unsigned long long seed) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    v[j] = zmk(u01(seed, 2ull * j) - 0.5, u01(seed, 2ull * j + 1) - 0.5);
}

__global__ void gaussian_block_kernel(zd* Y, int64_t ldy, int n, int m, unsigned long long seed) {
  const int64_t total = (int64_t)n * m;
  const double pi2 = 6.283185307179586476925286766559;
  const double rs2 = 0.70710678118654752440084436210485;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double u1 = u01(seed, 2ull * t), u2 = u01(seed, 2ull * t + 1);
    const double rr = sqrt(-2.0 * log1p(-u1));
    double sn, cs;
    sincos(pi2 * u2, &sn, &cs);
    const int i = (int)(t % n), j = (int)(t / n);
    Y[i + (int64_t)j * ldy] = zmk(rr * cs * rs2, rr * sn * rs2);
  }
}

// ---------------------------------------------------------------- degrees and locking
// Inputs of the learned degree model for active column i (global index g = g0 + i), in the
// order of include/chfsi.h: log10 of the residual over tau now and in the last two loops
// (the current value where a loop is missing), the degrees of the last two loops (0 where
// missing), the Ritz-value position t_i = (theta_i - c)/e, the position t_0 of the smallest
// Ritz value a0 = theta_0, and the bound ratio (a - a0)/(b - a0).  History arrays may be
// null (no history).
__global__ void degree_features_kernel(const double* theta, const double* r, int m, double a, double b,
                                       double tau, int g0, const double* rh1, const double* rh2,
                                       const int* dh1, const int* dh2, float* X) {
  const double e = 0.5 * (b - a), c = 0.5 * (b + a);
  const double a0 = theta[0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const int g = g0 + i;
    const double r0 = r[i];
    double r1 = rh1 ? rh1[g] : 0.0;
    if (!(r1 > 0.0)) r1 = r0;
    double r2 = rh2 ? rh2[g] : 0.0;
    if (!(r2 > 0.0)) r2 = r1;
    float* x = X + (int64_t)i * CHFSI_MLP_IN;
    x[0] = (float)log10(r0 / tau);
    x[1] = (float)log10(r1 / tau);
    x[2] = (float)log10(r2 / tau);
    x[3] = dh1 ? (float)dh1[g] : 0.f;
    x[4] = dh2 ? (float)dh2[g] : 0.f;
    x[5] = (float)((theta[i] - c) / e);
    x[6] = (float)((a0 - c) / e);
    x[7] = (float)((a - a0) / (b - a0));
  }
}

// g(x) of the learned degree model for every column: one warp per column, FP16 weights (the
// order of chfsi_mlp, then mean and scale) converted to FP32 in shared memory and stored
// transposed (input-major) so that the lanes of a warp, which own consecutive units, read
// consecutive words.  FP32 arithmetic.
constexpr int DM_WARPS = 8;
__global__ void __launch_bounds__(32 * DM_WARPS) degree_model_kernel(const __half* W, const float* X, int m,
                                                                    float* gout) {
  constexpr int IN = CHFSI_MLP_IN, HID = CHFSI_MLP_HID;
  extern __shared__ float dm_smem[];
  float* w1t = dm_smem;                 // [IN][HID]
  float* b1 = w1t + IN * HID;
  float* w2t = b1 + HID;                // [HID][HID]
  float* b2 = w2t + HID * HID;
  float* w3t = b2 + HID;
  float* b3 = w3t + HID * HID;
  float* w4 = b3 + HID;
  float* act = w4 + HID + 2 * IN + 1;   // per warp: xh[IN], h[HID], h'[HID]
  const __half *s1 = W, *sb1 = s1 + HID * IN, *s2 = sb1 + HID, *sb2 = s2 + HID * HID, *s3 = sb2 + HID,
               *sb3 = s3 + HID * HID, *s4 = sb3 + HID, *sb4 = s4 + HID, *smean = sb4 + 1, *sscale = smean + IN;
  for (int e = threadIdx.x; e < HID * IN; e += blockDim.x) {
    const int j = e / IN, k = e % IN;
    w1t[k * HID + j] = __half2float(s1[e]);
  }
  for (int e = threadIdx.x; e < HID * HID; e += blockDim.x) {
    const int j = e / HID, k = e % HID;
    w2t[k * HID + j] = __half2float(s2[e]);
    w3t[k * HID + j] = __half2float(s3[e]);
  }
  for (int j = threadIdx.x; j < HID; j += blockDim.x) {
    b1[j] = __half2float(sb1[j]);
    b2[j] = __half2float(sb2[j]);
    b3[j] = __half2float(sb3[j]);
    w4[j] = __half2float(s4[j]);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float* xh = act + wid * (IN + 2 * HID);
  float* h = xh + IN;
  float* h2 = h + HID;
  const float bias4 = __half2float(sb4[0]);
  for (int col = blockIdx.x * DM_WARPS + wid; col < m; col += gridDim.x * DM_WARPS) {
    if (lane < IN)
      xh[lane] = (X[(int64_t)col * IN + lane] - __half2float(smean[lane])) * __half2float(sscale[lane]);
    __syncwarp();
    for (int j = lane; j < HID; j += 32) {
      float a = b1[j];
#pragma unroll
      for (int k = 0; k < IN; ++k) a += w1t[k * HID + j] * xh[k];
      h[j] = tanhf(a);
    }
    __syncwarp();
    for (int j = lane; j < HID; j += 32) {
      float a = b2[j];
      for (int k = 0; k < HID; ++k) a += w2t[k * HID + j] * h[k];
      h2[j] = tanhf(a);
    }
    __syncwarp();
    float y = 0.f;
    for (int j = lane; j < HID; j += 32) {
      float a = b3[j];
      for (int k = 0; k < HID; ++k) a += w3t[k * HID + j] * h2[k];
      y += w4[j] * tanhf(a);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
    if (lane == 0) gout[col] = y + bias4;
    __syncwarp();
  }
}

// Per-column degrees: the closed-form rule, with the learned rate correction g (clamped to
// [-3, 3]) where gcorr is given and the result is finite; columns past the wanted ones take
// the largest wanted degree; then the stable descending order.  With history arrays the
// residual and degree of every column are pushed into them (global index g0 + i).
__global__ void degrees_kernel(const double* theta, const double* r, int m, double a, double b,
                               double tau, int dmin, int dmax, int n_wanted, int* deg, int* perm,
                               int* degs, const float* gcorr, int g0, double* rh1, double* rh2,
                               int* dh1, int* dh2) {
  extern __shared__ int sd[];
  const double e = 0.5 * (b - a), c = 0.5 * (b + a);
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    int d = dmax;
    const double ri = r[i];
    if (ri <= tau) {
      d = dmin;
    } else {
      const double t = fabs((theta[i] - c) / e);
      if (t > 1.0) {
        const double rho = t + sqrt(t * t - 1.0);
        const double lrho = log(rho);
        double need = log(ri / tau) / lrho;
        if (gcorr) {
          const float g = fminf(3.f, fmaxf(-3.f, gcorr[i]));
          const double learned = log(ri / tau) / (lrho * exp((double)g));
          if (isfinite(learned)) need = learned;
        }
        if (isfinite(need) && need < (double)dmax) d = min(dmax, max(dmin, (int)ceil(need)));
      }
    }
    sd[i] = d;
  }
  __syncthreads();
  __shared__ int top;
  if (threadIdx.x == 0) {
    int t = dmin;
    for (int i = 0; i < min(n_wanted, m); ++i) t = max(t, sd[i]);
    top = t;
  }
  __syncthreads();
  for (int i = n_wanted + threadIdx.x; i < m; i += blockDim.x) sd[i] = top;
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const int di = sd[i];
    int rank = 0;
    for (int j = 0; j < m; ++j) rank += (sd[j] > di) || (sd[j] == di && j < i);
    deg[i] = di;
    perm[rank] = i;
    degs[rank] = di;
    if (rh1) {
      const int g = g0 + i;
      rh2[g] = rh1[g];
      dh2[g] = dh1[g];
      rh1[g] = r[i];
      dh1[g] = di;
    }
  }
}

__global__ void lock_scan_kernel(const double* r, int m, double tau, int max_lock, int* nlock) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int c = 0;
    const int lim = min(m, max_lock);
    while (c < lim && r[c] < tau) ++c;
    *nlock = c;
  }
}

__global__ void fill_nan_kernel(double* x, int m) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    x[i] = __longlong_as_double(0x7ff8000000000000ll);
}

// ---------------------------------------------------------------- Lanczos pieces
// w_i = sum_j H(i, j) v_j = sum_j conj(H(j, i)) v_j (H Hermitian): one warp per row reads
// column i contiguously.
__global__ void hemv_rows_kernel(const zd* H, int64_t ldh, const zd* v, zd* w, int n) {
  const int lane = threadIdx.x & 31;
  const int warps = (blockDim.x >> 5) * gridDim.x;
  for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    const zd* col = H + (int64_t)i * ldh;
    double sr = 0.0, si = 0.0;
    for (int j = lane; j < n; j += 32) {
      const zd h = col[j], x = v[j];
      sr += h.x * x.x + h.y * x.y;
      si += h.x * x.y - h.y * x.x;
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    if (lane == 0) w[i] = zmk(sr, si);
  }
}

// FP64 -> FP32 by truncation of the significand, in integer operations (a conversion
// instruction would run at the FP64 pipe's rate, which would bound the whole product):
// magnitudes below 2^-126 become 0, above the FP32 range infinity; relative error < 2^-23.
__device__ __forceinline__ float f32_trunc(double x) {
  const int hi = __double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const int e = ((hi >> 20) & 0x7FF) - 896;  // FP32 biased exponent (1023 - 127)
  unsigned b = (unsigned)hi & 0x80000000u;
  if (e >= 255) b |= 0x7F800000u;
  else if (e > 0) b |= ((unsigned)e << 23) | (((unsigned)hi & 0xFFFFFu) << 3) | (lo >> 29);
  return __uint_as_float(b);
}

// The same product with FP32 multiply-adds on the FP64 data (per-lane FP32 partial sums of
// at most 8 terms, then FP64): relative error ~1e-7, enough for a spectral bound.  The
// operands are narrowed by f32_trunc; v once per CTA into shared memory (vsh, n entries,
// when the launch gives it room) or per use from global memory.
__global__ void hemv_rows_f32_kernel(const zd* H, int64_t ldh, const zd* v, zd* w, int n, int v_in_smem) {
  extern __shared__ float2 vsh[];
  const int lane = threadIdx.x & 31;
  const int warps = (blockDim.x >> 5) * gridDim.x;
  if (v_in_smem) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      const zd x = v[j];
      vsh[j] = make_float2(f32_trunc(x.x), f32_trunc(x.y));
    }
    __syncthreads();
  }
  for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    const zd* col = H + (int64_t)i * ldh;
    double sr = 0.0, si = 0.0;
    for (int j0 = 0; j0 < n; j0 += 256) {
      float fr = 0.f, fi = 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + u * 32 + lane;
        if (j < n) {
          const zd h = col[j];
          float2 x;
          if (v_in_smem) {
            x = vsh[j];
          } else {
            const zd xv = v[j];
            x = make_float2(f32_trunc(xv.x), f32_trunc(xv.y));
          }
          const float hx = f32_trunc(h.x), hy = f32_trunc(h.y);
          fr = fmaf(hx, x.x, fmaf(hy, x.y, fr));
          fi = fmaf(hx, x.y, fmaf(-hy, x.x, fi));
        }
      }
      sr += (double)fr;
      si += (double)fi;
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    if (lane == 0) w[i] = zmk(sr, si);
  }
}

// c_l = V_l^H w for l = 0..j  (one CTA per l)
__global__ void block_dots_kernel(const zd* V, int64_t ldv, const zd* w, int n, zd* c) {
  const int l = blockIdx.x;
  double sr = 0.0, si = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const zd a = V[i + (int64_t)l * ldv], b = w[i];
    sr += a.x * b.x + a.y * b.y;
    si += a.x * b.y - a.y * b.x;
  }
  sr = block_sum(sr);
  si = block_sum(si);
  if (threadIdx.x == 0) c[l] = zmk(sr, si);
}

// w -= V c  (V: n x (j+1))
__global__ void block_update_kernel(const zd* V, int64_t ldv, int jp1, const zd* c, zd* w, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    zd s = w[i];
    for (int l = 0; l < jp1; ++l) {
      const zd a = V[i + (int64_t)l * ldv], cl = c[l];
      s.x -= a.x * cl.x - a.y * cl.y;
      s.y -= a.x * cl.y + a.y * cl.x;
    }
    w[i] = s;
  }
}

__global__ void vec_norm_kernel(const zd* w, int n, double* out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += zabs2(w[i]);
  s = block_sum(s);
  if (threadIdx.x == 0) *out = sqrt(s);
}

__global__ void vec_scale_into_kernel(const zd* w, int n, const double* nrm, zd* dst) {
  const double inv = 1.0 / nrm[0];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    dst[i] = zscale(w[i], inv);
}

__global__ void lanczos_record_kernel(const zd* c, int j, const double* nrm, double* alpha,
                                      double* beta) {
  if (threadIdx.x == 0) {
    alpha[j] = c[j].x;
    beta[j] = nrm[0];
  }
}

// Number of eigenvalues of the symmetric tridiagonal T (alpha, beta) below x (Sturm).
__device__ int sturm_count(const double* al, const double* be, int k, double x) {
  int cnt = 0;
  double q = al[0] - x;
  if (q < 0.0) ++cnt;
  for (int i = 1; i < k; ++i) {
    if (q == 0.0) q = 1e-300;
    q = (al[i] - x) - be[i - 1] * be[i - 1] / q;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// out[0] = min eig(T_k), out[1] = max eig(T_k), out[2] = max eig + |beta_{k-1}|.
__global__ void tridiag_extremes_kernel(const double* al, const double* be, int k, double* out) {
  if (threadIdx.x != 0) return;
  double lo = al[0], hi = al[0];
  for (int i = 0; i < k; ++i) {
    const double rad = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i < k - 1 ? fabs(be[i]) : 0.0);
    lo = fmin(lo, al[i] - rad);
    hi = fmax(hi, al[i] + rad);
  }
  const double pad = 1e-12 * fmax(fabs(lo), fabs(hi)) + 1e-300;
  lo -= pad;
  hi += pad;
  // smallest: largest x with count(x) == 0
  double a = lo, b = hi;
  for (int it = 0; it < 200 && b - a > 0.0; ++it) {
    const double mid = 0.5 * (a + b);
    if (mid <= a || mid >= b) break;
    if (sturm_count(al, be, k, mid) >= 1) b = mid; else a = mid;
  }
  out[0] = 0.5 * (a + b);
  // largest: smallest x with count(x) == k
  a = lo; b = hi;
  for (int it = 0; it < 200 && b - a > 0.0; ++it) {
    const double mid = 0.5 * (a + b);
    if (mid <= a || mid >= b) break;
    if (sturm_count(al, be, k, mid) >= k) b = mid; else a = mid;
  }
  out[1] = 0.5 * (a + b);
  out[2] = out[1] + fabs(be[k - 1]);
}

inline int grid_for(int64_t total, int threads = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(8 * sm_count(), (total + threads - 1) / threads));
}

// ------------------------------------------------------------------ deviation angles
// Deviation angles between eigenvectors of adjacent problems (Section 2.2 and Fig. 1).
// nrm[j] = sqrt(Re(x_j^H w_j)), w_j = B x_j: the B-norm of column j.
__global__ void bnorm_kernel(const zd* X, int64_t ldx, const zd* W, int64_t ldw, int n, double* nrm) {
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const zd x = X[i + (int64_t)j * ldx], w = W[i + (int64_t)j * ldw];
    acc += x.x * w.x + x.y * w.y;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) nrm[j] = sqrt(fmax(acc, 0.0));
}

// One-to-one association from |M| (k x k): k times, the largest |M_ij| over unassigned
// rows and columns (ties: smallest row, then smallest column) is assigned.  One CTA; the
// free flags of rows and columns live in shared memory (2k ints).
__global__ void associate_kernel(const zd* M, int64_t ldm, int k, int* assoc) {
  extern __shared__ int free_rc[];
  int* free_r = free_rc;
  int* free_c = free_rc + k;
  __shared__ double bv[32];
  __shared__ long long bi[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  for (int i = tid; i < k; i += blockDim.x) { free_r[i] = 1; free_c[i] = 1; }
  __syncthreads();
  for (int step = 0; step < k; ++step) {
    double best = -1.0;
    long long idx = 0x7fffffffffffffffLL;
    for (long long e = tid; e < (long long)k * k; e += blockDim.x) {
      const int i = (int)(e / k), j = (int)(e % k);  // e = i k + j: lexicographic (i, j)
      if (!free_r[i] || !free_c[j]) continue;
      const zd v = M[i + (int64_t)j * ldm];
      const double a = sqrt(v.x * v.x + v.y * v.y);
      if (a > best || (a == best && e < idx)) { best = a; idx = e; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const long long oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (ob > best || (ob == best && oi < idx)) { best = ob; idx = oi; }
    }
    if (lane == 0) { bv[w] = best; bi[w] = idx; }
    __syncthreads();
    if (tid == 0) {
      double b = bv[0];
      long long x = bi[0];
      for (int q = 1; q < nw; ++q)
        if (bv[q] > b || (bv[q] == b && bi[q] < x)) { b = bv[q]; x = bi[q]; }
      const int i = (int)(x / k), j = (int)(x % k);
      assoc[i] = j;
      free_r[i] = 0;
      free_c[j] = 0;
    }
    __syncthreads();
  }
}

// R[:, i] = u_c - u_p (u_p^H B u_c) with u_p = x_prev_i / np_i, u_c = x_cur_a / nc_a,
// a = assoc[i], and u_p^H B u_c = M(i, a) / (np_i nc_a).
__global__ void dev_residual_kernel(const zd* Xp, int64_t ldp, const zd* Xc, int64_t ldc, const zd* M,
                                    int64_t ldm, const double* np_, const double* nc_, const int* assoc,
                                    int n, zd* R, int64_t ldr) {
  const int i = blockIdx.x;
  const int a = assoc[i];
  const double ip = 1.0 / np_[i], ic = 1.0 / nc_[a];
  const zd mu = zscale(M[i + (int64_t)a * ldm], ip * ic);
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const zd up = zscale(Xp[r + (int64_t)i * ldp], ip);
    const zd uc = zscale(Xc[r + (int64_t)a * ldc], ic);
    R[r + (int64_t)i * ldr] = zsub(uc, zmul(up, mu));
  }
}

// theta_i = asin(min(1, sqrt(Re(r_i^H (B r_i))))).
__global__ void dev_theta_kernel(const zd* R, int64_t ldr, const zd* BR, int64_t ldbr, int n, double* theta) {
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const zd x = R[r + (int64_t)i * ldr], w = BR[r + (int64_t)i * ldbr];
    acc += x.x * w.x + x.y * w.y;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) theta[i] = asin(fmin(1.0, sqrt(fmax(acc, 0.0))));
}

// Y[:, j] *= d[j] for every column when *flag is set (the column scaling a Cholesky QR
// step of the mixed-precision re-orthonormalisation asks for), nothing otherwise.
__global__ void scale_cols_flag_kernel(zd* Y, int64_t ldy, int n, int m, const double* d, const int* flag) {
  if (!*flag) return;
  const int64_t tot = (int64_t)n * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    Y[i + (int64_t)j * ldy] = zscale(Y[i + (int64_t)j * ldy], d[j]);
  }
}

}  // namespace

cudaError_t herm_from_lower(const zd* src, int64_t lds, zd* dst, int64_t ldd, int n, int* status,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int nb = (n + TILE - 1) / TILE;
  herm_from_lower_kernel<<<dim3(nb, nb), dim3(32, 8), 0, s>>>(src, lds, dst, ldd, n, status);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t mirror_lower(zd* H, int64_t ldh, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int nb = (n + TILE - 1) / TILE;
  mirror_lower_kernel<<<dim3(nb, nb), dim3(32, 8), 0, s>>>(H, ldh, n);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t herm_sum(zd* H, int64_t ldh, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int nb = (n + TILE - 1) / TILE;
  herm_sum_kernel<<<dim3(nb, nb), dim3(32, 8), 0, s>>>(H, ldh, n);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t zero_upper(zd* L, int64_t ldl, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  zero_upper_kernel<<<grid_for((int64_t)n * n), 256, 0, s>>>(L, ldl, n);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t copy_cols(const zd* src, int64_t lds, zd* dst, int64_t ldd, int n, int m, cudaStream_t s) {
  if (n <= 0 || m <= 0) return cudaSuccess;
  copy_cols_kernel<<<grid_for((int64_t)n * m), 256, 0, s>>>(src, lds, dst, ldd, n, m, nullptr, nullptr);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t gather_cols(const zd* src, int64_t lds, zd* dst, int64_t ldd, int n, int m,
                        const int* perm, cudaStream_t s) {
  if (n <= 0 || m <= 0) return cudaSuccess;
  copy_cols_kernel<<<grid_for((int64_t)n * m), 256, 0, s>>>(src, lds, dst, ldd, n, m, perm, nullptr);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t select_cols(const zd* src1, int64_t ld1, zd* dst, int64_t ldd, int n, int m,
                        const int* flag, cudaStream_t s) {
  if (n <= 0 || m <= 0) return cudaSuccess;
  copy_cols_kernel<<<grid_for((int64_t)n * m), 256, 0, s>>>(src1, ld1, dst, ldd, n, m, nullptr, flag);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t compare_equal(const zd* a, int64_t lda, const zd* b, int64_t ldb, int n, int m,
                          int* diff_flag, cudaStream_t s) {
  if (n <= 0 || m <= 0) return cudaSuccess;
  compare_kernel<<<grid_for((int64_t)n * m), 256, 0, s>>>(a, lda, b, ldb, n, m, diff_flag);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t column_residuals(const zd* HY, int64_t ldhy, const zd* Y, int64_t ldy,
                             const double* theta, int n, int m, double* r, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  column_residuals_kernel<<<m, 256, 0, s>>>(HY, ldhy, Y, ldy, theta, n, r);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t generalized_residuals(const zd* AX, int64_t ldax, const zd* BX, int64_t ldbx,
                                  const zd* X, int64_t ldx, const double* lam, int n, int m,
                                  const double* a_norm, double* r, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  gen_residuals_kernel<<<m, 256, 0, s>>>(AX, ldax, BX, ldbx, X, ldx, lam, n, a_norm, r);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t splitmix_start_vector(zd* v, int n, uint64_t seed, cudaStream_t s) {
  start_vector_kernel<<<grid_for(n), 256, 0, s>>>(v, n, (unsigned long long)seed);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t splitmix_gaussian_block(zd* Y, int64_t ldy, int n, int m, uint64_t seed, cudaStream_t s) {
  gaussian_block_kernel<<<grid_for((int64_t)n * m), 256, 0, s>>>(Y, ldy, n, m,
                                                                 (unsigned long long)seed);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t degree_features(const double* theta, const double* r, int m, double a, double b, double tau,
                            int g0, const double* rh1, const double* rh2, const int* dh1, const int* dh2,
                            float* X, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  degree_features_kernel<<<(m + 127) / 128, 128, 0, s>>>(theta, r, m, a, b, tau, g0, rh1, rh2, dh1, dh2, X);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t degree_model_eval(const __half* mlp, const float* X, int m, float* g, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  constexpr int IN = CHFSI_MLP_IN, HID = CHFSI_MLP_HID;
  const size_t smem = sizeof(float) * ((size_t)HID * IN + 2 * (size_t)HID * HID + 4 * HID + 2 * IN + 1 +
                                       (size_t)DM_WARPS * (IN + 2 * HID));
  static const cudaError_t attr =
      cudaFuncSetAttribute(degree_model_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (attr != cudaSuccess) return attr;
  const int blocks = std::min((m + DM_WARPS - 1) / DM_WARPS, 2 * sm_count());
  degree_model_kernel<<<blocks, 32 * DM_WARPS, smem, s>>>(mlp, X, m, g);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t degrees_kernel_run(const double* theta, const double* r, int m, double a, double b,
                               double tau, int dmin, int dmax, int n_wanted, int* deg,
                               int* perm_desc, int* deg_sorted, cudaStream_t s, const float* gcorr,
                               int g0, double* rh1, double* rh2, int* dh1, int* dh2) {
  if (m <= 0) return cudaSuccess;
  degrees_kernel<<<1, 256, m * sizeof(int), s>>>(theta, r, m, a, b, tau, dmin, dmax, n_wanted,
                                                 deg, perm_desc, deg_sorted, gcorr, g0, rh1, rh2, dh1, dh2);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t diag_ratio(const zd* L, int64_t ldl, int n, double* out2, cudaStream_t s) {
  diag_ratio_kernel<<<1, 256, 0, s>>>(L, ldl, n, out2);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t rayleigh_quotients(const zd* HY, int64_t ldhy, const zd* Y, int64_t ldy, int n, int m,
                               double* theta, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  rayleigh_quotients_kernel<<<m, 256, 0, s>>>(HY, ldhy, Y, ldy, n, theta);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t lock_scan(const double* r, int m, double tau, int max_lock, int* nlock, cudaStream_t s) {
  lock_scan_kernel<<<1, 32, 0, s>>>(r, m, tau, max_lock, nlock);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t fill_nan(double* x, int m, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  fill_nan_kernel<<<grid_for(m), 256, 0, s>>>(x, m);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t hemv_rows_prepare(int n, int* per_sm) {
  constexpr size_t kVshMax = 128 * 1024;
  static const cudaError_t attr = cudaFuncSetAttribute(
      hemv_rows_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kVshMax);
  if (attr != cudaSuccess) return attr;
  static thread_local int last_n = -1, last_per_sm = 0;
  const size_t smem = sizeof(float2) * (size_t)n;
  if (n != last_n) {
    int p = 0;
    if (n > 0 && smem <= kVshMax) {
      const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, hemv_rows_f32_kernel, 256, smem);
      if (e != cudaSuccess) return e;
    }
    last_n = n;
    last_per_sm = p;
  }
  if (per_sm) *per_sm = last_per_sm;
  return cudaSuccess;
}
cudaError_t hemv_rows(const zd* H, int64_t ldh, const zd* v, zd* w, int n, cudaStream_t s, bool f32) {
  const int warps_per_block = 8;
  int blocks = std::max(1, std::min((n + warps_per_block - 1) / warps_per_block, 16 * sm_count()));
  if (f32) {
    // v in shared memory up to 128 KB (n <= 16384), with as many CTAs as fit on the SMs
    int per_sm = 0;
    const cudaError_t e = hemv_rows_prepare(n, &per_sm);
    if (e != cudaSuccess) return e;
    const int in_smem = per_sm > 0 ? 1 : 0;
    if (in_smem) blocks = std::max(1, std::min(blocks, per_sm * sm_count()));
    hemv_rows_f32_kernel<<<blocks, 32 * warps_per_block, in_smem ? sizeof(float2) * (size_t)n : 0, s>>>(
        H, ldh, v, w, n, in_smem);
  } else {
    hemv_rows_kernel<<<blocks, 32 * warps_per_block, 0, s>>>(H, ldh, v, w, n);
  }
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t block_dots(const zd* V, int64_t ldv, int j, const zd* w, int n, zd* c, cudaStream_t s) {
  block_dots_kernel<<<j + 1, 256, 0, s>>>(V, ldv, w, n, c);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t block_update(const zd* V, int64_t ldv, int j, const zd* c, zd* w, int n, cudaStream_t s) {
  block_update_kernel<<<grid_for(n), 256, 0, s>>>(V, ldv, j + 1, c, w, n);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t vec_norm(const zd* w, int n, double* out, cudaStream_t s) {
  vec_norm_kernel<<<1, 1024, 0, s>>>(w, n, out);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t vec_scale_into(const zd* w, int n, const double* nrm, zd* dst, cudaStream_t s) {
  vec_scale_into_kernel<<<grid_for(n), 256, 0, s>>>(w, n, nrm, dst);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t lanczos_record(const zd* c, int j, const double* nrm, double* alpha, double* beta,
                           cudaStream_t s) {
  lanczos_record_kernel<<<1, 32, 0, s>>>(c, j, nrm, alpha, beta);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t tridiag_extremes(const double* alpha, const double* beta, int k, double* out3,
                             cudaStream_t s) {
  tridiag_extremes_kernel<<<1, 32, 0, s>>>(alpha, beta, k, out3);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t bnorms(const zd* X, int64_t ldx, const zd* W, int64_t ldw, int n, int k, double* nrm,
                   cudaStream_t s) {
  bnorm_kernel<<<k, 256, 0, s>>>(X, ldx, W, ldw, n, nrm);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t associate(const zd* M, int64_t ldm, int k, int* assoc, cudaStream_t s) {
  const size_t smem = 2 * sizeof(int) * (size_t)k;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(associate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  associate_kernel<<<1, 1024, smem, s>>>(M, ldm, k, assoc);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t deviation_residual(const zd* Xp, int64_t ldp, const zd* Xc, int64_t ldc, const zd* M,
                               int64_t ldm, const double* np_, const double* nc_, const int* assoc,
                               int n, int k, zd* R, int64_t ldr, cudaStream_t s) {
  dev_residual_kernel<<<k, 256, 0, s>>>(Xp, ldp, Xc, ldc, M, ldm, np_, nc_, assoc, n, R, ldr);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t deviation_theta(const zd* R, int64_t ldr, const zd* BR, int64_t ldbr, int n, int k,
                            double* theta, cudaStream_t s) {
  dev_theta_kernel<<<k, 256, 0, s>>>(R, ldr, BR, ldbr, n, theta);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
cudaError_t scale_cols_flag(zd* Y, int64_t ldy, int n, int m, const double* d, const int* flag, cudaStream_t s) {
  const int64_t tot = (int64_t)n * m;
  const int blocks = (int)std::min<int64_t>(4 * sm_count(), (tot + 255) / 256);
  scale_cols_flag_kernel<<<std::max(1, blocks), 256, 0, s>>>(Y, ldy, n, m, d, flag);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
