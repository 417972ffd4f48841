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

// ------------------------------------------------------------------ Gram scaling for Cholesky QR
// dscale_i = 1/sqrt(G_ii); G <- D G D on the lower triangle; backup (ld m) <- the scaled lower
// triangle, kept for a shifted retry.  One CTA.
__global__ void gram_scale_kernel(zd* G, int64_t ldg, int m, double* dscale, zd* backup) {
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double d = G[i + (int64_t)i * ldg].x;
    dscale[i] = (d > 0.0 && isfinite(d)) ? rsqrt(d) : 1.0;
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    if (i < j) continue;
    const zd v = zscale(G[i + (int64_t)j * ldg], dscale[i] * dscale[j]);
    G[i + (int64_t)j * ldg] = v;
    backup[i + (int64_t)j * m] = v;
  }
}

// G <- backup + s I (lower), s = shift_base * trace(backup).  One CTA.
__global__ void gram_shift_kernel(const zd* backup, int m, double shift_base, zd* G, int64_t ldg) {
  __shared__ double tr;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < m; ++i) t += backup[i + (int64_t)i * m].x;
    tr = t;
  }
  __syncthreads();
  const double sft = shift_base * tr;
  for (int64_t e = threadIdx.x; e < (int64_t)m * m; e += blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    if (i < j) continue;
    zd v = backup[i + (int64_t)j * m];
    if (i == j) v.x += sft;
    G[i + (int64_t)j * ldg] = v;
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
};

constexpr long kBarrierSpinLimit = 20000000;  // ~1-2 s with the back-off below

// Sense-free generation barrier over all CTAs of a cooperative launch.  Returns false (and
// sets DEV_TIMEOUT) if the wait ran past its limit or another CTA already reported it.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* status) {
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
      long it = 0;
      while (*vgen == gen) {
        if (++it > kBarrierSpinLimit || (*(volatile int*)status & DEV_TIMEOUT)) {
          atomicOr(status, DEV_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
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

__global__ void __launch_bounds__(128) jacobi_kernel(const JacParams P) {
  extern __shared__ unsigned char smem_raw[];
  Rot* rot = reinterpret_cast<Rot*>(smem_raw);
  __shared__ double red[128];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int mp = P.mp, half = mp / 2;
  const unsigned nb = gridDim.x;
  const int cta = blockIdx.x;

  // ---- set-up: rows 2cta, 2cta+1 of Ga (padded copy of G) and of Vw (identity)
  for (int rr = 0; rr < 2; ++rr) {
    const int i = 2 * cta + rr;
    for (int j = tid; j < mp; j += nt) {
      zd v = zmk(0.0, 0.0);
      if (i < P.m && j < P.m) v = P.G[i + (int64_t)j * P.ldg];
      if (i == j) v.y = 0.0;
      P.Ga[i + (int64_t)j * mp] = v;
      P.Vw[i + (int64_t)j * mp] = zmk(i == j ? 1.0 : 0.0, 0.0);
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
  if (!grid_barrier(P.bar, nb, P.status)) return;

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
      for (int t = tid; t < half; t += nt) {
        int p, q;
        pair_of(round, t, mp, p, q);
        const double a = ldcg(src + p + (int64_t)p * mp).x;
        const double d = ldcg(src + q + (int64_t)q * mp).x;
        const zd b = ldcg(src + p + (int64_t)q * mp);
        const double ab = sqrt(zabs2(b));
        Rot R;
        if (!(ab > thresh)) {
          R.c = 1.0; R.s = 0.0; R.w = zmk(1.0, 0.0); R.active = 0;
        } else {
          const double zeta = (d - a) / (2.0 * ab);
          const double t_ = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + hypot(1.0, zeta));
          R.c = 1.0 / sqrt(1.0 + t_ * t_);
          R.s = t_ * R.c;
          R.w = zmk(b.x / ab, -b.y / ab);  // e^{-i phi}
          R.active = 1;
        }
        rot[t] = R;
      }
      __syncthreads();
      // my pair: rows p, q of dst = U_P^H src[P, R] U_R for every pair R
      int p, q;
      pair_of(round, cta, mp, p, q);
      const Rot RP = rot[cta];
      const zd wpc = zconj(RP.w);  // e^{+i phi}
      for (int t = tid; t < half; t += nt) {
        int r, s;
        pair_of(round, t, mp, r, s);
        const Rot RR = rot[t];
        const zd m00 = ldcg(src + p + (int64_t)r * mp), m01 = ldcg(src + p + (int64_t)s * mp);
        const zd m10 = ldcg(src + q + (int64_t)r * mp), m11 = ldcg(src + q + (int64_t)s * mp);
        // left: U_P^H = [[c, -s e^{i phi}], [s, c e^{i phi}]]
        const zd sw = zscale(wpc, RP.s), cw = zscale(wpc, RP.c);
        const zd l00 = zsub(zscale(m00, RP.c), zmul(sw, m10));
        const zd l01 = zsub(zscale(m01, RP.c), zmul(sw, m11));
        const zd l10 = zadd(zscale(m00, RP.s), zmul(cw, m10));
        const zd l11 = zadd(zscale(m01, RP.s), zmul(cw, m11));
        // right: U_R = [[c, s], [-s w, c w]]
        const zd rsw = zscale(RR.w, RR.s), rcw = zscale(RR.w, RR.c);
        zd n00 = zsub(zscale(l00, RR.c), zmul(l01, rsw));
        zd n01 = zadd(zscale(l00, RR.s), zmul(l01, rcw));
        zd n10 = zsub(zscale(l10, RR.c), zmul(l11, rsw));
        zd n11 = zadd(zscale(l10, RR.s), zmul(l11, rcw));
        if (t == cta) {  // diagonal block: exact diagonal result
          n00.y = 0.0; n11.y = 0.0;
          if (RP.active) { n01 = zmk(0.0, 0.0); n10 = zmk(0.0, 0.0); }
        }
        dst[p + (int64_t)r * mp] = n00;
        dst[p + (int64_t)s * mp] = n01;
        dst[q + (int64_t)r * mp] = n10;
        dst[q + (int64_t)s * mp] = n11;
      }
      // V rows 2cta, 2cta+1 (owned for the whole run): V[i, R] <- V[i, R] U_R
      for (int e = tid; e < 2 * half; e += nt) {
        const int i = 2 * cta + (e & 1);
        const int t = e >> 1;
        int r, s;
        pair_of(round, t, mp, r, s);
        const Rot RR = rot[t];
        if (!RR.active) continue;
        zd* vr = P.Vw + i + (int64_t)r * mp;
        zd* vs = P.Vw + i + (int64_t)s * mp;
        const zd a0 = *vr, a1 = *vs;
        const zd rsw = zscale(RR.w, RR.s), rcw = zscale(RR.w, RR.c);
        *vr = zsub(zscale(a0, RR.c), zmul(a1, rsw));
        *vs = zadd(zscale(a0, RR.s), zmul(a1, rcw));
      }
      parity ^= 1;
      if (!grid_barrier(P.bar, nb, P.status)) return;
    }
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

cudaError_t gram_scale(zd* G, int64_t ldg, int m, double* dscale, zd* backup, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  gram_scale_kernel<<<1, 1024, 0, s>>>(G, ldg, m, dscale, backup);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t gram_shift(const zd* backup, int m, double shift_base, zd* G, int64_t ldg, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  gram_shift_kernel<<<1, 1024, 0, s>>>(backup, m, shift_base, G, ldg);
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

cudaError_t jacobi_heev(const zd* G, int64_t ldg, int m, double* w, zd* V, int64_t ldv, zd* work,
                        unsigned* barrier, int* status, cudaStream_t s) {
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
  cudaError_t e = cudaMemsetAsync(barrier, 0, 4 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  const int half = mp / 2;
  const size_t smem = sizeof(Rot) * (size_t)half;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  void* args[] = {(void*)&P};
  e = cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(half), dim3(128), args, smem, s);
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
