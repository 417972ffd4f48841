// Small dense kernels on blk x blk (or panel-sized) matrices: Cholesky factorisation with
// optional column scaling and shift (Cholesky QR), triangular inverse, and a cooperative
// multi-CTA cyclic Jacobi eigensolver for the Rayleigh-Ritz matrix.
//
// The FP64 pipe of one SM is slow (two FMAs per clock), so the Jacobi solver spreads each
// round of rotations over m/2 CTAs, one rotation pair per CTA, synchronised by a bounded
// grid barrier (every wait has an iteration limit and reports DEV_TIMEOUT instead of
// hanging).
#include <cmath>

#include "internal.cuh"

namespace {

// ------------------------------------------------------------------ Cholesky (one CTA)
// In place on the lower triangle of G (m x m).  Optional unit-diagonal scaling
// (dscale[i] = 1/sqrt(G_ii)) and a shifted retry (G + s I, s = shift_base * trace) when a
// pivot is not positive.  backup: m x m scratch used for the retry.
__global__ void cholesky_kernel(zd* G, int64_t ldg, int m, int scale, int shift_on_fail,
                                double shift_base, double* dscale, zd* backup, int* status,
                                int* info, int info_base, int* shift_flag) {
  __shared__ int fail;
  __shared__ double pivot;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (scale) {
    for (int i = tid; i < m; i += nt) {
      const double d = G[i + (int64_t)i * ldg].x;
      dscale[i] = (d > 0.0 && isfinite(d)) ? rsqrt(d) : 1.0;
    }
    __syncthreads();
    for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
      const int i = (int)(e % m), j = (int)(e / m);
      if (i >= j) G[i + (int64_t)j * ldg] = zscale(G[i + (int64_t)j * ldg], dscale[i] * dscale[j]);
    }
    __syncthreads();
  } else if (dscale) {
    for (int i = tid; i < m; i += nt) dscale[i] = 1.0;
  }
  if (shift_on_fail) {
    for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
      const int i = (int)(e % m), j = (int)(e / m);
      if (i >= j) backup[i + (int64_t)j * m] = G[i + (int64_t)j * ldg];
    }
  }
  __syncthreads();
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (tid == 0) fail = -1;
    __syncthreads();
    for (int j = 0; j < m; ++j) {
      if (tid == 0) {
        const double d = G[j + (int64_t)j * ldg].x;
        if (!(d > 0.0) || !isfinite(d)) {
          fail = j;
          pivot = 1.0;
        } else {
          pivot = sqrt(d);
        }
        G[j + (int64_t)j * ldg] = zmk(pivot, 0.0);
      }
      __syncthreads();
      if (fail >= 0) break;
      const double inv = 1.0 / pivot;
      for (int i = j + 1 + tid; i < m; i += nt)
        G[i + (int64_t)j * ldg] = zscale(G[i + (int64_t)j * ldg], inv);
      __syncthreads();
      // trailing update of the lower triangle: G(i,k) -= G(i,j) conj(G(k,j)), j < k <= i
      const int r = m - j - 1;
      for (int64_t e = tid; e < (int64_t)r * r; e += nt) {
        const int ii = (int)(e % r), kk = (int)(e / r);
        if (ii < kk) continue;
        const int gi = j + 1 + ii, gk = j + 1 + kk;
        const zd lij = G[gi + (int64_t)j * ldg];
        const zd lkj = G[gk + (int64_t)j * ldg];
        zd v = G[gi + (int64_t)gk * ldg];
        v.x -= lij.x * lkj.x + lij.y * lkj.y;
        v.y -= lij.y * lkj.x - lij.x * lkj.y;
        G[gi + (int64_t)gk * ldg] = v;
      }
      __syncthreads();
    }
    if (fail < 0) break;
    if (!shift_on_fail || attempt == 1) {
      if (tid == 0) {
        atomicOr(status, DEV_NOTPD);
        if (info) atomicMin(info, info_base + fail);
      }
      return;
    }
    // shifted retry: G <- backup + s I with s = shift_base * trace(backup)
    __shared__ double tr;
    if (tid == 0 && shift_flag) *shift_flag = 1;
    if (tid == 0) {
      double t = 0.0;
      for (int i = 0; i < m; ++i) t += backup[i + (int64_t)i * m].x;
      tr = t;
    }
    __syncthreads();
    const double s = shift_base * tr;
    for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
      const int i = (int)(e % m), j = (int)(e / m);
      if (i >= j) {
        zd v = backup[i + (int64_t)j * m];
        if (i == j) v.x += s;
        G[i + (int64_t)j * ldg] = v;
      }
    }
    __syncthreads();
  }
  // zero the strict upper triangle
  for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
    const int i = (int)(e % m), j = (int)(e / m);
    if (i < j) G[i + (int64_t)j * ldg] = zmk(0.0, 0.0);
  }
}

// ------------------------------------------------------------------ triangular inverse
// X = L^{-1} for lower-triangular L (m x m), one warp per column by forward substitution;
// the strict upper triangle of X is zeroed.  X must not alias L.
__global__ void trinv_lower_kernel(const zd* L, int64_t ldl, zd* X, int64_t ldx, int m) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = blockIdx.x * nw + warp; j < m; j += gridDim.x * nw) {
    for (int i = lane; i < j; i += 32) X[i + (int64_t)j * ldx] = zmk(0.0, 0.0);
    for (int i = j; i < m; ++i) {
      // s = sum_{k=j}^{i-1} L(i,k) X(k,j)
      zd s = zmk(0.0, 0.0);
      for (int k = j + lane; k < i; k += 32) s = zfma(L[i + (int64_t)k * ldl], X[k + (int64_t)j * ldx], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
      }
      if (lane == 0) {
        const zd lii = L[i + (int64_t)i * ldl];
        const double den = zabs2(lii);
        const zd inv = zmk(lii.x / den, -lii.y / den);
        const zd rhs = (i == j) ? zmk(1.0, 0.0) : zmk(-s.x, -s.y);
        X[i + (int64_t)j * ldx] = zmul(inv, rhs);
      }
      __syncwarp();
    }
  }
}

// T = D X^H (upper), T(i,j) = d_i conj(X(j,i)) for i <= j, 0 below the diagonal.
__global__ void cholqr_T_kernel(const zd* X, int64_t ldx, int m, const double* dscale, zd* T,
                                int64_t ldt) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    zd v = zmk(0.0, 0.0);
    if (i <= j) {
      v = zconj(X[j + (int64_t)i * ldx]);
      if (dscale) v = zscale(v, dscale[i]);
    }
    T[i + (int64_t)j * ldt] = v;
  }
}

// ------------------------------------------------------------------ mixed-precision Cholesky QR
// One pass of the re-orthonormalisation Y <- Y T used by the mixed-precision path.  G = Y^H Y
// (m x m, lower triangle read) and e = ||G - I||_F decide the pass:
//   e <= 1e-3: first-order Loewdin step T = I - (G - I)/2 in FP64 (full Hermitian T); the
//              new Gram error is about 3/4 e^2, so e <= 1e-8 finishes (flags[0] = 1);
//   e >  1e-3: Cholesky QR step in FP32 on the unit-diagonal scaled Gram,
//              D G D + s I = L L^H (s = 0, then 1e-5, 1e-4, 1e-3 on breakdown), Y <- (Y D) T
//              with T = L^{-H} (upper triangular; flags[3] = 1 asks for the column scaling
//              by D = dscale first, so that the product sees unit columns and O(1) factors),
//              which reduces e to the FP32 level (or, when Y is ill-conditioned, reduces
//              cond(Y) by about sqrt(1/s)).
// Precision of T only affects how far Y T is from orthonormal, never its span: the product
// Y T itself is formed in FP64-level arithmetic and the last step is always an FP64 Loewdin
// step.  flags[1] counts FP32 Cholesky steps, flags[2] records a shifted one.  One CTA of
// QR_THREADS threads; the FP32 factor lives in shared memory (m <= QR_SMEM_MMAX) or in the
// global scratch `gs` (m*m + 32*m float2).
constexpr int QR_THREADS = 1024;
constexpr int QR_SMEM_MMAX = 144;

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void __launch_bounds__(QR_THREADS)
    qr_pass_kernel(const zd* G, int64_t ldg, int m, zd* T, int64_t ldt, double* dscale, float2* gs,
                   int* flags, int* status) {
  extern __shared__ float2 qr_smem[];
  __shared__ double red[QR_THREADS / 32];
  __shared__ double e_all;
  __shared__ int fail;
  __shared__ float piv;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nw = nt >> 5;

  // ---- e = ||G - I||_F from the lower triangle
  double acc = 0.0;
  for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
    const int i = (int)(e % m), j = (int)(e / m);
    if (i < j) continue;
    const zd g = G[i + (int64_t)j * ldg];
    if (i == j) acc += (g.x - 1.0) * (g.x - 1.0) + g.y * g.y;
    else acc += 2.0 * (g.x * g.x + g.y * g.y);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    e_all = sqrt(t);
  }
  __syncthreads();
  const double e_f = e_all;

  if (e_f <= 1e-3) {
    // ---- first-order Loewdin step, FP64
    for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
      const int i = (int)(e % m), j = (int)(e / m);
      zd g = (i >= j) ? G[i + (int64_t)j * ldg] : zconj(G[j + (int64_t)i * ldg]);
      zd t = zmk(-0.5 * g.x, -0.5 * g.y);
      if (i == j) t = zmk(1.0 - 0.5 * (g.x - 1.0), 0.0);
      T[i + (int64_t)j * ldt] = t;
    }
    if (tid == 0) {
      if (e_f <= 1e-8) flags[0] = 1;
      flags[3] = 0;  // T applies to Y as it is
    }
    return;
  }
  if (!(e_f < 1e300)) {  // NaN or Inf in the Gram matrix
    if (tid == 0) {
      atomicOr(status, DEV_NOTPD);
      flags[3] = 0;
    }
    return;
  }

  // ---- FP32 Cholesky QR step
  float2* A = (m <= QR_SMEM_MMAX) ? qr_smem : gs;
  float2* xb = A + (int64_t)m * m;  // per-warp column buffers (32 x m)
  for (int i = tid; i < m; i += nt) {
    const double d = G[i + (int64_t)i * ldg].x;
    dscale[i] = (d > 0.0 && isfinite(d)) ? rsqrt(d) : 1.0;
  }
  if (tid == 0) {
    atomicAdd(flags + 1, 1);
    flags[3] = 1;  // T applies to Y D (columns scaled by dscale first)
  }
  __syncthreads();
  int attempt = 0;
  for (; attempt < 4; ++attempt) {
    for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
      const int i = (int)(e % m), j = (int)(e / m);
      if (i < j) continue;
      const zd g = G[i + (int64_t)j * ldg];
      const double sc = dscale[i] * dscale[j];  // FP64: G may exceed the FP32 range
      float2 v = make_float2((float)(g.x * sc), (float)(g.y * sc));
      const float shift = attempt == 0 ? 0.f : (attempt == 1 ? 1e-5f : (attempt == 2 ? 1e-4f : 1e-3f));
      if (i == j) v = make_float2(v.x + shift, 0.f);
      A[i + (int64_t)j * m] = v;
    }
    if (tid == 0) fail = -1;
    __syncthreads();
    for (int j = 0; j < m; ++j) {
      if (tid == 0) {
        const float d = A[j + (int64_t)j * m].x;
        if (!(d > 0.f) || !isfinite(d)) fail = j;
        else piv = sqrtf(d);
      }
      __syncthreads();
      if (fail >= 0) break;
      const float inv = 1.f / piv;
      for (int i = j + 1 + tid; i < m; i += nt) {
        const float2 v = A[i + (int64_t)j * m];
        A[i + (int64_t)j * m] = make_float2(v.x * inv, v.y * inv);
      }
      if (tid == 0) A[j + (int64_t)j * m] = make_float2(piv, 0.f);
      __syncthreads();
      // trailing update of the lower triangle: A(i,k) -= L(i,j) conj(L(k,j)), j < k <= i
      const int r = m - j - 1;
      for (int e = tid; e < r * r; e += nt) {
        const int ii = e % r, kk = e / r;
        if (ii < kk) continue;
        const int gi = j + 1 + ii, gk = j + 1 + kk;
        const float2 lij = A[gi + (int64_t)j * m], lkj = A[gk + (int64_t)j * m];
        float2 v = A[gi + (int64_t)gk * m];
        v.x -= lij.x * lkj.x + lij.y * lkj.y;
        v.y -= lij.y * lkj.x - lij.x * lkj.y;
        A[gi + (int64_t)gk * m] = v;
      }
      __syncthreads();
    }
    if (fail < 0) break;
  }
  if (attempt == 4) {
    if (tid == 0) {
      atomicOr(status, DEV_NOTPD);
      flags[3] = 0;
    }
    return;
  }
  if (attempt > 0 && tid == 0) flags[2] = 1;

  // ---- X = L^{-1} column by column (one warp per column, forward substitution), and
  // T = D X^H: row j of T holds d_j conj(X(:, j)).
  float2* x = xb + (int64_t)warp * m;
  for (int j = warp; j < m; j += nw) {
    for (int i = j; i < m; ++i) {
      float2 sacc = make_float2(0.f, 0.f);
      for (int k = j + lane; k < i; k += 32) {
        const float2 p = cmulf(A[i + (int64_t)k * m], x[k]);
        sacc.x += p.x;
        sacc.y += p.y;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sacc.x += __shfl_xor_sync(0xffffffffu, sacc.x, o);
        sacc.y += __shfl_xor_sync(0xffffffffu, sacc.y, o);
      }
      if (lane == 0) {
        const float dinv = 1.f / A[i + (int64_t)i * m].x;
        x[i] = (i == j) ? make_float2(dinv, 0.f) : make_float2(-sacc.x * dinv, -sacc.y * dinv);
      }
      __syncwarp();
    }
    for (int i = lane; i < m; i += 32)
      T[j + (int64_t)i * ldt] = (i < j) ? zmk(0.0, 0.0) : zmk((double)x[i].x, -(double)x[i].y);
    __syncwarp();
  }
}

// ------------------------------------------------------------------ Jacobi eigensolver
struct JacParams {
  const zd* G;
  int64_t ldg;
  int m, mp;
  zd* Ga;
  zd* Gb;
  zd* Vw;   // mp x mp, ld mp
  unsigned* bar;
  int* status;
  int max_sweeps;
  long long spin_limit;  // polls of a grid-barrier wait before it gives up
  int pairs_per_cta;     // rotation pairs (and 2x as many rows of V) per CTA
};

constexpr long kBarrierSpinLimit = 8000000;  // polls of an L2 word: a few seconds at most

// Sense-free generation barrier over all CTAs of a cooperative launch.  Returns false (and
// sets DEV_TIMEOUT) if the wait ran past its limit or another CTA already reported it.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* status, long long limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      while (*vgen == gen) {
        if (++it > limit || (*(volatile int*)status & DEV_TIMEOUT)) {
          atomicOr(status, DEV_TIMEOUT);
          ok = 0;
          break;
        }

      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ void pair_of(int round, int slot, int mp, int& p, int& q) {
  const int M1 = mp - 1;
  q = 1 + ((mp - 2 - slot + round) % M1);
  p = (slot == 0) ? 0 : 1 + ((slot - 1 + round) % M1);
}

__device__ __forceinline__ zd ldcg(const zd* p) { return __ldcg(p); }

// 2x2 products with the rotation U = [[c, s], [-s w, c w]], w = e^{-i phi}.
struct Rot { double c, s; zd w; int active; };

constexpr int JAC_THREADS = 256;
constexpr int kJacSmemMax = 224 * 1024;  // dynamic shared memory a Jacobi CTA may use

__device__ __forceinline__ Rot jacobi_rotation(const zd* src, int mp, int p, int q, double thresh) {
  const double a = ldcg(src + p + (int64_t)p * mp).x;
  const double d = ldcg(src + q + (int64_t)q * mp).x;
  const zd b = ldcg(src + p + (int64_t)q * mp);
  const double ab2 = zabs2(b);
  Rot R;
  if (!(ab2 > thresh * thresh)) {
    R.c = 1.0; R.s = 0.0; R.w = zmk(1.0, 0.0); R.active = 0;
  } else {
    // tan of the rotation angle from zeta = (d - a) / (2 |b|), with reciprocal square roots
    // in place of divisions where the formula allows (the FP64 pipe is this part's bottleneck)
    const double inv_ab = rsqrt(ab2);
    const double zeta = 0.5 * (d - a) * inv_ab;
    const double az = fabs(zeta);
    // |zeta| large: 1/(|zeta| + sqrt(1 + zeta^2)) without overflow of zeta^2
    const double t_ = (zeta >= 0.0 ? 1.0 : -1.0) /
                      (az + (az < 1e150 ? sqrt(1.0 + zeta * zeta) : az));
    R.c = rsqrt(1.0 + t_ * t_);
    R.s = t_ * R.c;
    R.w = zmk(b.x * inv_ab, -b.y * inv_ab);  // e^{-i phi}
    R.active = 1;
  }
  return R;
}

// CTA c takes the rotation pairs (slots) c*ppc .. c*ppc + ppc - 1 of every round (ppc =
// P.pairs_per_cta; one pair per CTA while the grid fits, more for large blocks).  Per round
// the CTA computes all rotations of the round; then, one pair at a time, it copies columns p
// and q into shared memory (coalesced; by Hermitian symmetry column j holds the conjugated
// row j), applies U_P^H on the left and the column-pair rotations U_R on the right in place
// there — work item t owns rows p, q and columns r, s of one 2 x 2 block, so no two items
// touch the same entry — and writes the new columns back (coalesced).  The CTA's 2 ppc rows of V
// (rows 2 slot, 2 slot + 1 of its slots) stay in shared memory for the whole run and take
// the right rotations of every pair of the round.
__global__ void __launch_bounds__(JAC_THREADS) jacobi_kernel(const JacParams P) {
  extern __shared__ unsigned char smem_raw[];
  const int mp = P.mp, half = mp / 2, ppc = P.pairs_per_cta;
  Rot* rot = reinterpret_cast<Rot*>(smem_raw);
  zd* vrow = reinterpret_cast<zd*>(smem_raw + sizeof(Rot) * (size_t)half);  // 2 ppc x mp
  zd* col = vrow + (size_t)2 * ppc * mp;                                      // 2 x mp
  __shared__ double red[JAC_THREADS];
  const int tid = threadIdx.x, nt = blockDim.x;
  const unsigned nb = gridDim.x;
  const int cta = blockIdx.x;
  const int slot0 = cta * ppc;
  const int nslot = max(0, min(ppc, half - slot0));  // pairs this CTA owns

  // ---- set-up: rows 2 slot, 2 slot + 1 of Ga (padded copy of G) and of V (identity)
  for (int rr = 0; rr < 2 * nslot; ++rr) {
    const int i = 2 * slot0 + rr;
    for (int j = tid; j < mp; j += nt) {
      zd v = zmk(0.0, 0.0);
      if (i < P.m && j < P.m) v = P.G[i + (int64_t)j * P.ldg];
      if (i == j) v.y = 0.0;
      P.Ga[i + (int64_t)j * mp] = v;
      vrow[rr * mp + j] = zmk(i == j ? 1.0 : 0.0, 0.0);
    }
  }
  // threshold from ||G||_F (computed redundantly by every CTA)
  double acc = 0.0;
  for (int64_t e = tid; e < (int64_t)P.m * P.m; e += nt) {
    const int i = (int)(e % P.m), j = (int)(e / P.m);
    acc += zabs2(P.G[i + (int64_t)j * P.ldg]);
  }
  red[tid] = acc;
  __syncthreads();
  for (int o = nt / 2; o > 0; o >>= 1) {
    if (tid < o) red[tid] += red[tid + o];
    __syncthreads();
  }
  const double thresh = 1e-15 * sqrt(red[0]) + 1e-300;
  __syncthreads();
  if (!grid_barrier(P.bar, nb, P.status, P.spin_limit)) return;

  int parity = 0;
  int sweep = 0;
  for (; sweep < P.max_sweeps; ++sweep) {
    {  // converged when every off-diagonal entry is below the threshold
      const zd* cur = parity ? P.Gb : P.Ga;
      double mx = 0.0;
      for (int64_t e = tid; e < (int64_t)mp * mp; e += nt) {
        const int i = (int)(e % mp), j = (int)(e / mp);
        if (i != j) mx = fmax(mx, zabs2(ldcg(cur + e)));
      }
      red[tid] = mx;
      __syncthreads();
      for (int o = nt / 2; o > 0; o >>= 1) {
        if (tid < o) red[tid] = fmax(red[tid], red[tid + o]);
        __syncthreads();
      }
      const bool done = !(sqrt(red[0]) > thresh);
      __syncthreads();
      if (done) break;
    }
    for (int round = 0; round < mp - 1; ++round) {
      const zd* src = parity ? P.Gb : P.Ga;
      zd* dst = parity ? P.Ga : P.Gb;
      // all rotations of this round (same inputs, same result on every CTA)
      int any = 0;
      for (int t = tid; t < half; t += nt) {
        int a, b;
        pair_of(round, t, mp, a, b);
        rot[t] = jacobi_rotation(src, mp, a, b, thresh);
        any |= rot[t].active;
      }
      // a round whose pairs are all below the threshold leaves the matrix as it is: every CTA
      // reaches the same decision and skips it (no writes, no barrier)
      if (!__syncthreads_or(any)) continue;
      for (int k = 0; k < nslot; ++k) {
        const int slot = slot0 + k;
        int p, q;
        pair_of(round, slot, mp, p, q);
        zd* cp = col;       // column p: cp[j] = conj(G[p, j])
        zd* cq = col + mp;  // column q
        for (int j = tid; j < mp; j += nt) {
          cp[j] = ldcg(src + j + (int64_t)p * mp);
          cq[j] = ldcg(src + j + (int64_t)q * mp);
        }
        __syncthreads();
        const Rot RP = rot[slot];
        const zd wpc = zconj(RP.w);  // e^{+i phi}
        const zd sw = zscale(wpc, RP.s), cw = zscale(wpc, RP.c);
        for (int t = tid; t < half; t += nt) {
          int r, s;
          pair_of(round, t, mp, r, s);
          const zd m00 = zconj(cp[r]), m01 = zconj(cp[s]), m10 = zconj(cq[r]), m11 = zconj(cq[s]);
          const Rot RR = rot[t];
          // left: U_P^H = [[c, -s e^{i phi}], [s, c e^{i phi}]] on rows p, q
          const zd l0p = zsub(zscale(m00, RP.c), zmul(sw, m10));
          const zd l1p = zsub(zscale(m01, RP.c), zmul(sw, m11));
          const zd l0q = zadd(zscale(m00, RP.s), zmul(cw, m10));
          const zd l1q = zadd(zscale(m01, RP.s), zmul(cw, m11));
          // right: U_R = [[c, s], [-s w, c w]] on columns r, s
          const zd rsw = zscale(RR.w, RR.s), rcw = zscale(RR.w, RR.c);
          zd np0 = zsub(zscale(l0p, RR.c), zmul(l1p, rsw));
          zd np1 = zadd(zscale(l0p, RR.s), zmul(l1p, rcw));
          zd nq0 = zsub(zscale(l0q, RR.c), zmul(l1q, rsw));
          zd nq1 = zadd(zscale(l0q, RR.s), zmul(l1q, rcw));
          if (t == slot) {  // diagonal block: exact diagonal result
            np0.y = 0.0;
            nq1.y = 0.0;
            if (RP.active) { np1 = zmk(0.0, 0.0); nq0 = zmk(0.0, 0.0); }
          }
          cp[r] = zconj(np0);
          cp[s] = zconj(np1);
          cq[r] = zconj(nq0);
          cq[s] = zconj(nq1);
        }
        __syncthreads();
        for (int j = tid; j < mp; j += nt) {
          dst[j + (int64_t)p * mp] = cp[j];
          dst[j + (int64_t)q * mp] = cq[j];
        }
        __syncthreads();
      }
      // V rows 2 slot + row (shared memory): V[i, R] <- V[i, R] U_R
      for (int e = tid; e < 2 * nslot * half; e += nt) {
        const int vr = e / half, t = e - vr * half;
        const Rot RR = rot[t];
        if (!RR.active) continue;
        int r, s;
        pair_of(round, t, mp, r, s);
        const zd rsw = zscale(RR.w, RR.s), rcw = zscale(RR.w, RR.c);
        zd* vi = vrow + vr * mp;
        const zd a0 = vi[r], a1 = vi[s];
        vi[r] = zsub(zscale(a0, RR.c), zmul(a1, rsw));
        vi[s] = zadd(zscale(a0, RR.s), zmul(a1, rcw));
      }
      parity ^= 1;
      if (!grid_barrier(P.bar, nb, P.status, P.spin_limit)) return;
    }
  }
  __syncthreads();
  for (int rr = 0; rr < 2 * nslot; ++rr) {
    const int i = 2 * slot0 + rr;
    for (int j = tid; j < mp; j += nt) P.Vw[i + (int64_t)j * mp] = vrow[rr * mp + j];
  }
  if (cta == 0 && tid == 0) {
    if (sweep >= P.max_sweeps) atomicOr(P.status, DEV_NOCONV);
    P.bar[2] = parity;  // where the final matrix lives
  }
}

// Sort eigenvalues ascending and copy the matching eigenvector columns.
__global__ void jacobi_finish_kernel(const zd* Ga, const zd* Gb, const zd* Vw, const unsigned* bar,
                                     int m, int mp, double* w, zd* V, int64_t ldv) {
  extern __shared__ unsigned char smem_raw[];
  double* val = reinterpret_cast<double*>(smem_raw);
  int* rank = reinterpret_cast<int*>(val + m);
  const zd* Gf = bar[2] ? Gb : Ga;
  for (int i = threadIdx.x; i < m; i += blockDim.x) val[i] = Gf[i + (int64_t)i * mp].x;
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    int r = 0;
    const double v = val[i];
    for (int j = 0; j < m; ++j) r += (val[j] < v) || (val[j] == v && j < i);
    rank[i] = r;
    w[r] = v;
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
    const int i = (int)(e % m), c = (int)(e / m);
    V[i + (int64_t)rank[c] * ldv] = Vw[i + (int64_t)c * mp];
  }
}

// ------------------------------------------------------------------ Jacobi in double-float
// The Rayleigh-Ritz eigensolver of the mixed-precision path for wide blocks: the cyclic
// parallel Jacobi of jacobi_kernel with the matrix and the CTA's rows of V held as
// unevaluated sums of two FP32 numbers (hi + lo, |lo| <= ulp(hi) / 2, about 48 significand
// bits) and rotated with FP32 arithmetic (products made exact by fma, sums by two-sum), since
// the FP64 pipe bounds the FP64 solver on wide blocks.  Each rotation is computed in FP64
// from the double-float entries by the CTA that owns its pair and published in global memory
// (two buffers by round parity) behind a grid barrier, so a round costs two barriers.  The
// matrix is scaled by a power of two (exact) so that ||G||_F lies in [1/2, 1), which keeps
// the FP32 convergence test in range.  Convergence: no off-diagonal entry above the
// threshold (tested on the high words, spread over the CTAs), or a sweep without an active
// rotation.
struct RotDF {
  float2 c, s;    // cosine and sine, hi + lo
  float2 wr, wi;  // e^{-i phi}: real and imaginary part, hi + lo
  int active;
  int pad;
};
// bytes of the rotation table at the head of the Jacobi CTA's shared memory (16-aligned)
__host__ __device__ __forceinline__ size_t rotdf_bytes(int half) {
  return (sizeof(RotDF) * (size_t)half + 15) / 16 * 16;
}
__device__ __forceinline__ float4 rot_w(const RotDF& R) { return make_float4(R.wr.x, R.wr.y, R.wi.x, R.wi.y); }

__device__ __forceinline__ float2 df_of(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double dbl_of(float h, float l) { return (double)h + (double)l; }

// s + e: a sum of double-float products, the error terms kept apart until df_norm
struct DfSum {
  float s, e;
};
__device__ __forceinline__ DfSum df_prod(float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);  // the rounding error of ah bh, exactly
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  DfSum r;
  r.s = p;
  r.e = e;
  return r;
}
__device__ __forceinline__ void df_acc(DfSum& a, const DfSum& b) {
  const float s = __fadd_rn(a.s, b.s);  // two-sum: s + err = a.s + b.s exactly
  const float bb = __fsub_rn(s, a.s);
  const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bb)), __fsub_rn(b.s, bb));
  a.s = s;
  a.e = __fadd_rn(__fadd_rn(a.e, b.e), err);
}
__device__ __forceinline__ float2 df_norm(const DfSum& a) {
  const float s = __fadd_rn(a.s, a.e);
  return make_float2(s, __fsub_rn(a.e, __fsub_rn(s, a.s)));
}
__device__ __forceinline__ float4 dfc(float2 re, float2 im) { return make_float4(re.x, re.y, im.x, im.y); }
__device__ __forceinline__ float4 dfc_conj(float4 x) { return make_float4(x.x, x.y, -x.z, -x.w); }
// x w
__device__ __forceinline__ float4 dfc_mul(float4 x, float4 w) {
  DfSum re = df_prod(x.x, x.y, w.x, w.y);
  df_acc(re, df_prod(-x.z, -x.w, w.z, w.w));
  DfSum im = df_prod(x.x, x.y, w.z, w.w);
  df_acc(im, df_prod(x.z, x.w, w.x, w.y));
  return dfc(df_norm(re), df_norm(im));
}
// conj(w) x
__device__ __forceinline__ float4 dfc_mulconj(float4 x, float4 w) {
  DfSum re = df_prod(x.x, x.y, w.x, w.y);
  df_acc(re, df_prod(x.z, x.w, w.z, w.w));
  DfSum im = df_prod(x.z, x.w, w.x, w.y);
  df_acc(im, df_prod(-x.x, -x.y, w.z, w.w));
  return dfc(df_norm(re), df_norm(im));
}
// a x + b y, a and b real
__device__ __forceinline__ float4 dfc_comb(float2 a, float4 x, float2 b, float4 y) {
  DfSum re = df_prod(a.x, a.y, x.x, x.y);
  df_acc(re, df_prod(b.x, b.y, y.x, y.y));
  DfSum im = df_prod(a.x, a.y, x.z, x.w);
  df_acc(im, df_prod(b.x, b.y, y.z, y.w));
  return dfc(df_norm(re), df_norm(im));
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

// 512 threads: the double-float updates are chains of dependent FP32 operations, and one
// CTA per SM (its shared memory) needs 16 warps to keep the FP32 pipes busy.
constexpr int JAC_DF_THREADS = 512;

struct JacDfParams {
  const zd* G;
  int64_t ldg;
  int m, mp;
  float4* Ga;
  float4* Gb;
  zd* Vw;          // output rows of V (mp x mp, ld mp); during the run: rotations, partials
  unsigned* bar;
  int* status;
  int max_sweeps;
  long long spin_limit;
  int pairs_per_cta;
};

__global__ void __launch_bounds__(JAC_DF_THREADS, 1) jacobi_df_kernel(const JacDfParams P) {
  extern __shared__ unsigned char smem_raw[];
  const int mp = P.mp, half = mp / 2, ppc = P.pairs_per_cta;
  RotDF* rot = reinterpret_cast<RotDF*>(smem_raw);
  float4* vrow = reinterpret_cast<float4*>(smem_raw + rotdf_bytes(half));  // 2 ppc x mp
  float4* col = vrow + (size_t)2 * ppc * mp;                                          // 2 x mp
  __shared__ double red[JAC_DF_THREADS];
  __shared__ float redf[JAC_DF_THREADS];
  const int tid = threadIdx.x, nt = blockDim.x;
  const unsigned nb = gridDim.x;
  const int cta = blockIdx.x;
  const int slot0 = cta * ppc;
  const int nslot = max(0, min(ppc, half - slot0));
  // global scratch inside Vw until the end: rotations of the two round parities, partials
  RotDF* rotg = reinterpret_cast<RotDF*>(P.Vw);
  double* part = reinterpret_cast<double*>(rotg + 2 * half);
  float* partf = reinterpret_cast<float*>(part + nb);

  // ---- ||G||_F from per-CTA partial sums (fixed order), the power-of-two scale
  double acc = 0.0;
  for (int64_t e = (int64_t)cta * nt + tid; e < (int64_t)P.m * P.m; e += (int64_t)nb * nt) {
    const int i = (int)(e % P.m), j = (int)(e / P.m);
    acc += zabs2(P.G[i + (int64_t)j * P.ldg]);
  }
  red[tid] = acc;
  __syncthreads();
  for (int o = nt / 2; o > 0; o >>= 1) {
    if (tid < o) red[tid] += red[tid + o];
    __syncthreads();
  }
  if (tid == 0) part[cta] = red[0];
  if (!grid_barrier(P.bar, nb, P.status, P.spin_limit)) return;
  __shared__ double s_norm;
  if (tid == 0) {
    double t = 0.0;
    for (unsigned b = 0; b < nb; ++b) t += __ldcg(part + b);
    s_norm = sqrt(t);
  }
  __syncthreads();
  const double nrm = s_norm;
  const int kexp = nrm > 0.0 ? ilogb(nrm) + 1 : 0;
  const double scale = ldexp(1.0, -kexp);       // ||G scale||_F in [1/2, 1)
  const double thresh = 1e-15 * nrm * scale + 1e-300;
  const float thresh2f = (float)(thresh * thresh);

  // ---- set-up: rows 2 slot, 2 slot + 1 of Ga (scaled, double-float) and of V (identity)
  for (int rr = 0; rr < 2 * nslot; ++rr) {
    const int i = 2 * slot0 + rr;
    for (int j = tid; j < mp; j += nt) {
      zd v = zmk(0.0, 0.0);
      if (i < P.m && j < P.m) v = P.G[i + (int64_t)j * P.ldg];
      if (i == j) v.y = 0.0;
      P.Ga[i + (int64_t)j * mp] = dfc(df_of(v.x * scale), df_of(v.y * scale));
      vrow[rr * mp + j] = make_float4(i == j ? 1.f : 0.f, 0.f, 0.f, 0.f);
    }
  }
  if (!grid_barrier(P.bar, nb, P.status, P.spin_limit)) return;

  int parity = 0, sweep = 0;
  for (; sweep < P.max_sweeps; ++sweep) {
    {  // largest off-diagonal |G_ij|^2 (high words) over all CTAs' shares
      const float4* cur = parity ? P.Gb : P.Ga;
      float mx = 0.f;
      for (int64_t e = (int64_t)cta * nt + tid; e < (int64_t)mp * mp; e += (int64_t)nb * nt) {
        const int i = (int)(e % mp), j = (int)(e / mp);
        if (i != j) {
          const float4 g = __ldcg(cur + e);
          mx = fmaxf(mx, g.x * g.x + g.z * g.z);
        }
      }
      redf[tid] = mx;
      __syncthreads();
      for (int o = nt / 2; o > 0; o >>= 1) {
        if (tid < o) redf[tid] = fmaxf(redf[tid], redf[tid + o]);
        __syncthreads();
      }
      if (tid == 0) partf[cta] = redf[0];
      if (!grid_barrier(P.bar, nb, P.status, P.spin_limit)) return;
      __shared__ int s_done;
      if (tid == 0) {
        float m2 = 0.f;
        for (unsigned b = 0; b < nb; ++b) m2 = fmaxf(m2, __ldcg(partf + b));
        s_done = !(m2 > thresh2f);
      }
      __syncthreads();
      if (s_done) break;
    }
    int sweep_any = 0;
    for (int round = 0; round < mp - 1; ++round) {
      const float4* src = parity ? P.Gb : P.Ga;
      float4* dst = parity ? P.Ga : P.Gb;
      RotDF* rg = rotg + (round & 1) * half;
      // the rotations of this CTA's pairs, in FP64 from the double-float entries
      for (int k = tid; k < nslot; k += nt) {
        const int slot = slot0 + k;
        int a, b;
        pair_of(round, slot, mp, a, b);
        const float4 ga = __ldcg(src + a + (int64_t)a * mp), gd_ = __ldcg(src + b + (int64_t)b * mp);
        const float4 gb = __ldcg(src + a + (int64_t)b * mp);
        const double av = dbl_of(ga.x, ga.y), dv = dbl_of(gd_.x, gd_.y);
        const zd bv = zmk(dbl_of(gb.x, gb.y), dbl_of(gb.z, gb.w));
        const double ab2 = zabs2(bv);
        RotDF R;
        R.pad = 0;
        if (!(ab2 > thresh * thresh)) {
          R.c = make_float2(1.f, 0.f);
          R.s = make_float2(0.f, 0.f);
          R.wr = make_float2(1.f, 0.f);
          R.wi = make_float2(0.f, 0.f);
          R.active = 0;
        } else {
          const double inv_ab = rsqrt(ab2);
          const double zeta = 0.5 * (dv - av) * inv_ab;
          const double az = fabs(zeta);
          const double t_ = (zeta >= 0.0 ? 1.0 : -1.0) / (az + (az < 1e150 ? sqrt(1.0 + zeta * zeta) : az));
          const double c = rsqrt(1.0 + t_ * t_);
          R.c = df_of(c);
          R.s = df_of(t_ * c);
          R.wr = df_of(bv.x * inv_ab);
          R.wi = df_of(-bv.y * inv_ab);
          R.active = 1;
        }
        rg[slot] = R;
      }
      if (!grid_barrier(P.bar, nb, P.status, P.spin_limit)) return;
      int any = 0;
      for (int t = tid; t < half; t += nt) {
        const float2* src2 = reinterpret_cast<const float2*>(rg + t);  // 5 x 8 bytes through L2
        RotDF R;
        R.c = __ldcg(src2);
        R.s = __ldcg(src2 + 1);
        R.wr = __ldcg(src2 + 2);
        R.wi = __ldcg(src2 + 3);
        const float2 ap = __ldcg(src2 + 4);
        R.active = __float_as_int(ap.x);
        R.pad = 0;
        rot[t] = R;
        any |= R.active;
      }
      // every CTA reads the same rotations and reaches the same decision
      if (!__syncthreads_or(any)) continue;
      sweep_any = 1;
      for (int k = 0; k < nslot; ++k) {
        const int slot = slot0 + k;
        int p, q;
        pair_of(round, slot, mp, p, q);
        float4* cp = col;       // column p: cp[j] = conj(G[p, j])
        float4* cq = col + mp;  // column q
        for (int j = tid; j < mp; j += nt) {
          cp[j] = __ldcg(src + j + (int64_t)p * mp);
          cq[j] = __ldcg(src + j + (int64_t)q * mp);
        }
        __syncthreads();
        const RotDF RP = rot[slot];
        for (int t = tid; t < half; t += nt) {
          int r, s;
          pair_of(round, t, mp, r, s);
          float4 l0p = dfc_conj(cp[r]), l1p = dfc_conj(cp[s]), l0q = dfc_conj(cq[r]), l1q = dfc_conj(cq[s]);
          if (RP.active) {
            // left: U_P^H = [[c, -s e^{i phi}], [s, c e^{i phi}]] on rows p, q (e^{i phi} = conj(w))
            const float4 wp = rot_w(RP);
            const float4 v0 = dfc_mulconj(l0q, wp), v1 = dfc_mulconj(l1q, wp);
            const float4 m00 = l0p, m01 = l1p;
            l0p = dfc_comb(RP.c, m00, df_neg(RP.s), v0);
            l1p = dfc_comb(RP.c, m01, df_neg(RP.s), v1);
            l0q = dfc_comb(RP.s, m00, RP.c, v0);
            l1q = dfc_comb(RP.s, m01, RP.c, v1);
          }
          const RotDF RR = rot[t];
          float4 np0 = l0p, np1 = l1p, nq0 = l0q, nq1 = l1q;
          if (RR.active) {
            // right: U_R = [[c, s], [-s w, c w]] on columns r, s
            const float4 wr = rot_w(RR);
            const float4 up = dfc_mul(l1p, wr), uq = dfc_mul(l1q, wr);
            np0 = dfc_comb(RR.c, l0p, df_neg(RR.s), up);
            np1 = dfc_comb(RR.s, l0p, RR.c, up);
            nq0 = dfc_comb(RR.c, l0q, df_neg(RR.s), uq);
            nq1 = dfc_comb(RR.s, l0q, RR.c, uq);
          }
          if (t == slot) {  // diagonal block: exact diagonal result
            np0.z = 0.f; np0.w = 0.f;
            nq1.z = 0.f; nq1.w = 0.f;
            if (RP.active) {
              np1 = make_float4(0.f, 0.f, 0.f, 0.f);
              nq0 = make_float4(0.f, 0.f, 0.f, 0.f);
            }
          }
          cp[r] = dfc_conj(np0);
          cp[s] = dfc_conj(np1);
          cq[r] = dfc_conj(nq0);
          cq[s] = dfc_conj(nq1);
        }
        __syncthreads();
        for (int j = tid; j < mp; j += nt) {
          dst[j + (int64_t)p * mp] = cp[j];
          dst[j + (int64_t)q * mp] = cq[j];
        }
        __syncthreads();
      }
      // V rows 2 slot + row (shared memory): V[i, R] <- V[i, R] U_R
      for (int e = tid; e < 2 * nslot * half; e += nt) {
        const int vr = e / half, t = e - vr * half;
        const RotDF RR = rot[t];
        if (!RR.active) continue;
        int r, s;
        pair_of(round, t, mp, r, s);
        float4* vi = vrow + vr * mp;
        const float4 a0 = vi[r], u = dfc_mul(vi[s], rot_w(RR));
        vi[r] = dfc_comb(RR.c, a0, df_neg(RR.s), u);
        vi[s] = dfc_comb(RR.s, a0, RR.c, u);
      }
      parity ^= 1;
      if (!grid_barrier(P.bar, nb, P.status, P.spin_limit)) return;
    }
    if (!sweep_any) break;
  }
  // every CTA is past its last read of the rotations and partials kept in Vw
  if (!grid_barrier(P.bar, nb, P.status, P.spin_limit)) return;
  const float4* fin = parity ? P.Gb : P.Ga;
  zd* diag_out = reinterpret_cast<zd*>(parity ? P.Ga : P.Gb);  // the buffer no longer read
  const double unscale = ldexp(1.0, kexp);
  for (int rr = 0; rr < 2 * nslot; ++rr) {
    const int i = 2 * slot0 + rr;
    for (int j = tid; j < mp; j += nt) {
      const float4 v = vrow[rr * mp + j];
      P.Vw[i + (int64_t)j * mp] = zmk(dbl_of(v.x, v.y), dbl_of(v.z, v.w));
    }
    if (tid == 0) {
      const float4 g = __ldcg(fin + i + (int64_t)i * mp);
      diag_out[i + (int64_t)i * mp] = zmk(dbl_of(g.x, g.y) * unscale, 0.0);
    }
  }
  if (cta == 0 && tid == 0) {
    if (sweep >= P.max_sweeps) atomicOr(P.status, DEV_NOCONV);
    P.bar[2] = parity ^ 1;  // the finishing kernel reads the diagonal from diag_out
  }
}

// ------------------------------------------------------------------ Cholesky QR pass, many CTAs
// The pass of qr_pass_kernel for blocks wider than one CTA's shared memory, spread over one
// cooperative grid: the Gram error from per-CTA partial sums (added in CTA order, so the
// decision is reproducible); a right-looking blocked FP32 Cholesky factorisation with
// 32-column panels — the diagonal block on CTA 0, the panel's rows below it one warp each
// (forward substitution against the diagonal block), the trailing lower tiles 32 x 32 each
// over all CTAs — retried with the same shifts on a non-positive pivot; and the inverse
// factor one warp per column.  Entries that another CTA wrote during the launch are read
// through L2 (ld.global.cg).  A bounded grid barrier that gives up ends every CTA with
// DEV_TIMEOUT.
constexpr int QRC_THREADS = 256;
constexpr int QRC_WARPS = QRC_THREADS / 32;
constexpr int QRC_NB = 32;

struct QrcParams {
  const zd* G;
  int64_t ldg;
  int m;
  zd* T;
  int64_t ldt;
  double* dscale;
  float2* A;     // m x m FP32 factor (lower triangle), ld m
  double* part;  // one partial Gram-error sum per CTA
  int* fail;     // per attempt: the first non-positive pivot, or -1
  int* flags;
  int* status;
  unsigned* bar;
  long long spin_limit;
};

__device__ __forceinline__ float qrc_shift(int attempt) {
  return attempt == 0 ? 0.f : (attempt == 1 ? 1e-5f : (attempt == 2 ? 1e-4f : 1e-3f));
}

__global__ void __launch_bounds__(QRC_THREADS) qr_pass_coop_kernel(const QrcParams P) {
  extern __shared__ float2 qrc_smem[];
  typedef float2 Tile[QRC_NB + 1];
  Tile* D = reinterpret_cast<Tile*>(qrc_smem);  // D[r][c]: diagonal block
  Tile* Li = D + QRC_NB;                         // rows of tile I, panel columns
  Tile* Lk = Li + QRC_NB;                        // rows of tile K, panel columns
  float2* xbuf = reinterpret_cast<float2*>(Lk + QRC_NB);  // one column of m per warp
  __shared__ double red[QRC_WARPS];
  __shared__ double s_e;
  __shared__ int s_fail;
  __shared__ float s_piv;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = (int)gridDim.x, cta = (int)blockIdx.x, m = P.m;
  const int64_t gtid = (int64_t)cta * QRC_THREADS + tid, gstride = (int64_t)nb * QRC_THREADS;
  const int64_t mm = (int64_t)m * m;
  float2* A = P.A;

  // ---- e = ||G - I||_F from the lower triangle
  if (cta == 0 && tid < 4) P.fail[tid] = -1;
  double acc = 0.0;
  for (int64_t e = gtid; e < mm; e += gstride) {
    const int i = (int)(e % m), j = (int)(e / m);
    if (i < j) continue;
    const zd g = P.G[i + (int64_t)j * P.ldg];
    if (i == j) acc += (g.x - 1.0) * (g.x - 1.0) + g.y * g.y;
    else acc += 2.0 * (g.x * g.x + g.y * g.y);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < QRC_WARPS; ++w) t += red[w];
    P.part[cta] = t;
  }
  if (!grid_barrier(P.bar, nb, P.status, P.spin_limit)) return;
  if (tid == 0) {
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += __ldcg(P.part + b);
    s_e = sqrt(t);
  }
  __syncthreads();
  const double e_f = s_e;  // the same in every CTA: all take the same branch below

  if (e_f <= 1e-3) {
    // ---- first-order Loewdin step, FP64
    for (int64_t e = gtid; e < mm; e += gstride) {
      const int i = (int)(e % m), j = (int)(e / m);
      const zd g = (i >= j) ? P.G[i + (int64_t)j * P.ldg] : zconj(P.G[j + (int64_t)i * P.ldg]);
      zd t = zmk(-0.5 * g.x, -0.5 * g.y);
      if (i == j) t = zmk(1.0 - 0.5 * (g.x - 1.0), 0.0);
      P.T[i + (int64_t)j * P.ldt] = t;
    }
    if (cta == 0 && tid == 0) {
      if (e_f <= 1e-8) P.flags[0] = 1;
      P.flags[3] = 0;
    }
    return;
  }
  if (!(e_f < 1e300)) {
    if (cta == 0 && tid == 0) {
      atomicOr(P.status, DEV_NOTPD);
      P.flags[3] = 0;
    }
    return;
  }

  // ---- FP32 Cholesky QR step: unit-diagonal scaling D, factor of D G D + shift I
  for (int64_t i = gtid; i < m; i += gstride) {
    const double d = P.G[i + (int64_t)i * P.ldg].x;
    P.dscale[i] = (d > 0.0 && isfinite(d)) ? rsqrt(d) : 1.0;
  }
  if (cta == 0 && tid == 0) {
    atomicAdd(P.flags + 1, 1);
    P.flags[3] = 1;
  }
  if (!grid_barrier(P.bar, nb, P.status, P.spin_limit)) return;
  int attempt = 0;
  for (; attempt < 4; ++attempt) {
    const float shift = qrc_shift(attempt);
    for (int64_t e = gtid; e < mm; e += gstride) {
      const int i = (int)(e % m), j = (int)(e / m);
      if (i < j) continue;
      const zd g = P.G[i + (int64_t)j * P.ldg];
      const double sc = __ldcg(P.dscale + i) * __ldcg(P.dscale + j);
      float2 v = make_float2((float)(g.x * sc), (float)(g.y * sc));
      if (i == j) v = make_float2(v.x + shift, 0.f);
      A[i + (int64_t)j * m] = v;
    }
    if (!grid_barrier(P.bar, nb, P.status, P.spin_limit)) return;
    int failed = -1;
    for (int jb = 0; jb < m; jb += QRC_NB) {
      const int w = min(QRC_NB, m - jb);
      if (cta == 0) {
        // diagonal block, unblocked in shared memory
        for (int e = tid; e < QRC_NB * QRC_NB; e += QRC_THREADS) {
          const int r = e % QRC_NB, c = e / QRC_NB;
          if (r < w && c <= r) D[r][c] = __ldcg(A + (jb + r) + (int64_t)(jb + c) * m);
        }
        if (tid == 0) s_fail = -1;
        __syncthreads();
        for (int c = 0; c < w; ++c) {
          if (tid == 0) {
            const float d = D[c][c].x;
            if (!(d > 0.f) || !isfinite(d)) s_fail = jb + c;
            else s_piv = sqrtf(d);
          }
          __syncthreads();
          if (s_fail >= 0) break;
          const float inv = 1.f / s_piv;
          if (tid > c && tid < w) {
            D[tid][c].x *= inv;
            D[tid][c].y *= inv;
          }
          if (tid == 0) D[c][c] = make_float2(s_piv, 0.f);
          __syncthreads();
          const int r = w - c - 1;
          for (int e = tid; e < r * r; e += QRC_THREADS) {
            const int ii = c + 1 + e % r, kk = c + 1 + e / r;
            if (ii < kk) continue;
            const float2 lij = D[ii][c], lkj = D[kk][c];
            D[ii][kk].x -= lij.x * lkj.x + lij.y * lkj.y;
            D[ii][kk].y -= lij.y * lkj.x - lij.x * lkj.y;
          }
          __syncthreads();
        }
        if (s_fail >= 0) {
          if (tid == 0) P.fail[attempt] = s_fail;
        } else {
          for (int e = tid; e < QRC_NB * QRC_NB; e += QRC_THREADS) {
            const int r = e % QRC_NB, c = e / QRC_NB;
            if (r < w && c <= r) A[(jb + r) + (int64_t)(jb + c) * m] = D[r][c];
          }
        }
      }
      if (!grid_barrier(P.bar, nb, P.status, P.spin_limit)) return;
      failed = __ldcg(P.fail + attempt);
      if (failed >= 0) break;
      const int r0 = jb + w;
      if (r0 < m) {
        // panel rows: L(i, panel) L_jj^H = A(i, panel), forward substitution, one warp a row
        // (lane c holds column jb + c)
        for (int e = tid; e < QRC_NB * QRC_NB; e += QRC_THREADS) {
          const int r = e % QRC_NB, c = e / QRC_NB;
          if (r < w && c <= r) D[r][c] = __ldcg(A + (jb + r) + (int64_t)(jb + c) * m);
        }
        __syncthreads();
        for (int i = r0 + cta * QRC_WARPS + warp; i < m; i += nb * QRC_WARPS) {
          float2 a = lane < w ? __ldcg(A + i + (int64_t)(jb + lane) * m) : make_float2(0.f, 0.f);
          for (int c = 0; c < w; ++c) {
            if (lane == c) {
              const float inv = 1.f / D[c][c].x;
              a.x *= inv;
              a.y *= inv;
            }
            const float2 xc = make_float2(__shfl_sync(0xffffffffu, a.x, c), __shfl_sync(0xffffffffu, a.y, c));
            if (lane > c && lane < w) {  // a_lane -= x_c conj(L_jj(lane, c))
              const float2 l = D[lane][c];
              a.x -= xc.x * l.x + xc.y * l.y;
              a.y -= xc.y * l.x - xc.x * l.y;
            }
          }
          if (lane < w) A[i + (int64_t)(jb + lane) * m] = a;
        }
      }
      if (!grid_barrier(P.bar, nb, P.status, P.spin_limit)) return;
      if (r0 < m) {
        // trailing update A(i, k) -= L(i, panel) L(k, panel)^H on the lower 32 x 32 tiles
        // (I, K), I >= K, of rows and columns r0.., tile t = I (I + 1) / 2 + K
        const int nt = (m - r0 + QRC_NB - 1) / QRC_NB;
        const int ntiles = nt * (nt + 1) / 2;
        for (int t = cta; t < ntiles; t += nb) {
          int I = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
          while ((I + 1) * (I + 2) / 2 <= t) ++I;
          while (I * (I + 1) / 2 > t) --I;
          const int K = t - I * (I + 1) / 2;
          const int i0 = r0 + I * QRC_NB, k0 = r0 + K * QRC_NB;
          __syncthreads();  // the previous tile's reads of Li and Lk are done
          for (int e = tid; e < QRC_NB * QRC_NB; e += QRC_THREADS) {
            const int r = e % QRC_NB, l = e / QRC_NB;
            const bool lv = l < w;
            Li[r][l] = (lv && i0 + r < m) ? __ldcg(A + (i0 + r) + (int64_t)(jb + l) * m) : make_float2(0.f, 0.f);
            Lk[r][l] = (lv && k0 + r < m) ? __ldcg(A + (k0 + r) + (int64_t)(jb + l) * m) : make_float2(0.f, 0.f);
          }
          __syncthreads();
          const int r = lane;
#pragma unroll
          for (int q = 0; q < QRC_NB / QRC_WARPS; ++q) {
            const int c = warp + QRC_WARPS * q;
            const int gi = i0 + r, gk = k0 + c;
            if (gi >= m || gk >= m || gi < gk) continue;
            float sx = 0.f, sy = 0.f;
            for (int l = 0; l < w; ++l) {
              const float2 a = Li[r][l], b = Lk[c][l];  // a conj(b)
              sx += a.x * b.x + a.y * b.y;
              sy += a.y * b.x - a.x * b.y;
            }
            float2 v = __ldcg(A + gi + (int64_t)gk * m);
            v.x -= sx;
            v.y -= sy;
            A[gi + (int64_t)gk * m] = v;
          }
        }
      }
      if (!grid_barrier(P.bar, nb, P.status, P.spin_limit)) return;
    }
    if (failed < 0) break;
  }
  if (attempt == 4) {
    if (cta == 0 && tid == 0) {
      atomicOr(P.status, DEV_NOTPD);
      P.flags[3] = 0;
    }
    return;
  }
  if (attempt > 0 && cta == 0 && tid == 0) P.flags[2] = 1;

  // ---- X = L^{-1} one warp per column (forward substitution), T = X^H: row j of T holds
  // conj(X(:, j)) (the scaling by D applies to Y first)
  float2* x = xbuf + (int64_t)warp * m;
  for (int j = cta * QRC_WARPS + warp; j < m; j += nb * QRC_WARPS) {
    for (int i = j; i < m; ++i) {
      float2 sacc = make_float2(0.f, 0.f);
      for (int k = j + lane; k < i; k += 32) {
        const float2 p = cmulf(__ldcg(A + i + (int64_t)k * m), x[k]);
        sacc.x += p.x;
        sacc.y += p.y;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sacc.x += __shfl_xor_sync(0xffffffffu, sacc.x, o);
        sacc.y += __shfl_xor_sync(0xffffffffu, sacc.y, o);
      }
      if (lane == 0) {
        const float dinv = 1.f / __ldcg(A + i + (int64_t)i * m).x;
        x[i] = (i == j) ? make_float2(dinv, 0.f) : make_float2(-sacc.x * dinv, -sacc.y * dinv);
      }
      __syncwarp();
    }
    for (int i = lane; i < m; i += 32)
      P.T[j + (int64_t)i * P.ldt] = (i < j) ? zmk(0.0, 0.0) : zmk((double)x[i].x, -(double)x[i].y);
    __syncwarp();
  }
}

}  // namespace

cudaError_t small_cholesky(zd* G, int64_t ldg, int m, int scale, int shift_on_fail,
                           double shift_base, double* dscale, zd* backup, int* status, int* info,
                           int info_base, cudaStream_t s, int* shift_flag) {
  if (m <= 0) return cudaSuccess;
  cholesky_kernel<<<1, 1024, 0, s>>>(G, ldg, m, scale, shift_on_fail, shift_base, dscale, backup,
                                     status, info, info_base, shift_flag);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t trinv_lower(const zd* L, int64_t ldl, zd* X, int64_t ldx, int m,
                               cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const int warps = 8;
  const int blocks = (m + warps - 1) / warps;
  trinv_lower_kernel<<<blocks, 32 * warps, 0, s>>>(L, ldl, X, ldx, m);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t qr_pass(const zd* G, int64_t ldg, int m, zd* T, int64_t ldt, double* dscale, void* scratch,
                    int* flags, int* status, cudaStream_t s, unsigned* barrier, long long spin_limit) {
  if (m <= 0) return cudaSuccess;
  if (m > QR_SMEM_MMAX && barrier) {
    // one cooperative grid of one CTA per SM; scratch: the FP32 factor, then the per-CTA
    // partial sums and the per-attempt failure words (m m float2 + grid doubles + 4 ints,
    // within the 3 mp^2 complex entries of the Jacobi work area it shares)
    const size_t smem = sizeof(float2) * (3 * QRC_NB * (QRC_NB + 1) + (size_t)QRC_WARPS * m);
    static const cudaError_t coop_attr =
        cudaFuncSetAttribute(qr_pass_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kJacSmemMax);
    if (coop_attr != cudaSuccess) return coop_attr;
    int per_sm = 0;
    cudaError_t e = cudaSuccess;
    if (smem <= (size_t)kJacSmemMax)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qr_pass_coop_kernel, QRC_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (per_sm >= 1) {
      const int grid = sm_count();
      e = cudaMemsetAsync(barrier, 0, 4 * sizeof(unsigned), s);
      if (e != cudaSuccess) return e;
      QrcParams P;
      P.G = G; P.ldg = ldg; P.m = m; P.T = T; P.ldt = ldt; P.dscale = dscale;
      P.A = static_cast<float2*>(scratch);
      P.part = reinterpret_cast<double*>(P.A + (int64_t)m * m);
      P.fail = reinterpret_cast<int*>(P.part + grid);
      P.flags = flags; P.status = status; P.bar = barrier;
      P.spin_limit = spin_limit > 0 ? spin_limit : kBarrierSpinLimit;
      void* args[] = {(void*)&P};
      e = cudaLaunchCooperativeKernel((const void*)qr_pass_coop_kernel, dim3(grid), dim3(QRC_THREADS), args,
                                      smem, s);
      CHFSI_COUNT_LAUNCH();
      return e;
    }
  }
  const size_t smem = (m <= QR_SMEM_MMAX) ? sizeof(float2) * ((size_t)m * m + 32 * (size_t)m) : 0;
  static const cudaError_t attr = cudaFuncSetAttribute(
      qr_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)(sizeof(float2) * ((size_t)QR_SMEM_MMAX * QR_SMEM_MMAX + 32 * (size_t)QR_SMEM_MMAX)));
  if (attr != cudaSuccess) return attr;
  qr_pass_kernel<<<1, QR_THREADS, smem, s>>>(G, ldg, m, T, ldt, dscale, static_cast<float2*>(scratch), flags,
                                             status);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t cholqr_T(const zd* X, int64_t ldx, int m, const double* dscale, zd* T, int64_t ldt,
                     cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  const int64_t tot = (int64_t)m * m;
  cholqr_T_kernel<<<(int)std::min<int64_t>(1024, (tot + 255) / 256), 256, 0, s>>>(X, ldx, m, dscale,
                                                                                   T, ldt);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t jacobi_heev_df(const zd* G, int64_t ldg, int m, double* w, zd* V, int64_t ldv, zd* work,
                           unsigned* barrier, int* status, cudaStream_t s, long long spin_limit) {
  if (m <= 0) return cudaSuccess;
  const int mp = (m + 1) & ~1;
  if (mp < 64) return jacobi_heev(G, ldg, m, w, V, ldv, work, barrier, status, s, spin_limit);
  JacDfParams P;
  P.G = G; P.ldg = ldg; P.m = m; P.mp = mp;
  P.Ga = reinterpret_cast<float4*>(work);
  P.Gb = reinterpret_cast<float4*>(work + (int64_t)mp * mp);
  P.Vw = work + 2 * (int64_t)mp * mp;
  P.bar = barrier;
  P.status = status;
  P.max_sweeps = 40;
  P.spin_limit = spin_limit > 0 ? spin_limit : kBarrierSpinLimit;
  cudaError_t e = cudaMemsetAsync(barrier, 0, 4 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  const int half = mp / 2;
  // dynamic shared memory: the opt-in limit per block less the kernel's static arrays
  // once per process (a static initialised once, also when batch workers call from several
  // host threads): the kernel's attribute and the limit the ppc search uses
  struct DynSmem {
    cudaError_t err;
    int max_bytes;
  };
  static const DynSmem dyn = [] {
    DynSmem d{cudaSuccess, 0};
    cudaFuncAttributes fa;
    int dev = 0, optin = 0;
    d.err = cudaFuncGetAttributes(&fa, jacobi_df_kernel);
    if (d.err == cudaSuccess) d.err = cudaGetDevice(&dev);
    if (d.err == cudaSuccess) d.err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (d.err != cudaSuccess) return d;
    d.max_bytes = std::min(kJacSmemMax, optin - (int)fa.sharedSizeBytes);
    d.err = cudaFuncSetAttribute(jacobi_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, d.max_bytes);
    return d;
  }();
  if (dyn.err != cudaSuccess) return dyn.err;
  const int dyn_max = dyn.max_bytes;
  int ppc = 1;
  size_t smem = 0;
  for (;; ++ppc) {
    smem = rotdf_bytes(half) + 2 * sizeof(float4) * (size_t)(ppc + 1) * mp;
    if (smem > (size_t)dyn_max) return cudaErrorInvalidValue;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_df_kernel, JAC_DF_THREADS, smem);
    if (e != cudaSuccess) return e;
    if ((int64_t)per_sm * sm_count() >= (half + ppc - 1) / ppc) break;
  }
  P.pairs_per_cta = ppc;
  const int grid = (half + ppc - 1) / ppc;
  // the rotation tables of both parities and the partial sums live in Vw during the run
  if (2 * sizeof(RotDF) * (size_t)half + 12 * (size_t)grid > sizeof(zd) * (size_t)mp * mp)
    return cudaErrorInvalidValue;
  void* args[] = {(void*)&P};
  e = cudaLaunchCooperativeKernel((const void*)jacobi_df_kernel, dim3(grid), dim3(JAC_DF_THREADS), args, smem, s);
  CHFSI_COUNT_LAUNCH();
  if (e != cudaSuccess) return e;
  const size_t smem2 = (size_t)m * (sizeof(double) + sizeof(int));
  if (smem2 > 48 * 1024) {
    e = cudaFuncSetAttribute(jacobi_finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    if (e != cudaSuccess) return e;
  }
  jacobi_finish_kernel<<<1, 1024, smem2, s>>>(reinterpret_cast<const zd*>(P.Ga), reinterpret_cast<const zd*>(P.Gb),
                                              P.Vw, barrier, m, mp, w, V, ldv);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t jacobi_heev(const zd* G, int64_t ldg, int m, double* w, zd* V, int64_t ldv, zd* work,
                        unsigned* barrier, int* status, cudaStream_t s, long long spin_limit) {
  if (m <= 0) return cudaSuccess;
  const int mp = (m + 1) & ~1;
  JacParams P;
  P.G = G; P.ldg = ldg; P.m = m; P.mp = mp;
  P.Ga = work;
  P.Gb = work + (int64_t)mp * mp;
  P.Vw = work + 2 * (int64_t)mp * mp;
  P.bar = barrier;
  P.status = status;
  P.max_sweeps = 40;
  P.spin_limit = spin_limit > 0 ? spin_limit : kBarrierSpinLimit;
  cudaError_t e = cudaMemsetAsync(barrier, 0, 4 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  const int half = mp / 2;
  // Pairs per CTA: the fewest for which the whole grid is co-resident (a cooperative launch),
  // each CTA keeping 2 ppc rows of V in shared memory.
  static const cudaError_t attr = cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       kJacSmemMax);
  if (attr != cudaSuccess) return attr;
  int ppc = 1;
  size_t smem = 0;
  for (;; ++ppc) {
    smem = sizeof(Rot) * (size_t)half + 2 * sizeof(zd) * (size_t)(ppc + 1) * mp;
    if (smem > (size_t)kJacSmemMax) return cudaErrorInvalidValue;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel, JAC_THREADS, smem);
    if (e != cudaSuccess) return e;
    if ((int64_t)per_sm * sm_count() >= (half + ppc - 1) / ppc) break;
  }
  P.pairs_per_cta = ppc;
  const int grid = (half + ppc - 1) / ppc;
  void* args[] = {(void*)&P};
  e = cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(grid), dim3(JAC_THREADS), args, smem, s);
  CHFSI_COUNT_LAUNCH();
  if (e != cudaSuccess) return e;
  const size_t smem2 = (size_t)m * (sizeof(double) + sizeof(int));
  if (smem2 > 48 * 1024) {
    e = cudaFuncSetAttribute(jacobi_finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem2);
    if (e != cudaSuccess) return e;
  }
  jacobi_finish_kernel<<<1, 1024, smem2, s>>>(P.Ga, P.Gb, P.Vw, barrier, m, mp, w, V, ldv);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}
