// Split-BF16 tensor-core products for the Chebyshev filter (mixed-precision filter).
//
// A complex FP64 product C = Hs Y (Hs n x n Hermitian, Y n x m) is computed as the real
// product C^ = H^ Y^ of the 2n x 2n real embedding H^ (rows and columns interleaved as
// (re, im), so that Y^ and C^ are the complex column-major arrays read as real arrays)
// with the 2n x m real Y^.  Each operand is split into S "digit slices":
//
//     H^(r, k) = 2^{eA(r)} sum_s a_s(r, k) 2^{-7 s},   a_1 in [-128, 128], a_{s>1} in [-64, 64]
//     Y^(k, j) = 2^{eB(j)} sum_t b_t(k, j) 2^{-7 t}
//
// with power-of-two scales per (complex) row of Hs and per column of Y.  Every digit is an
// integer that bf16 holds exactly, every digit product is exact in FP32, and a sum of at
// most 1024 such products stays below 2^24, so each K-chunk of 1024 accumulates EXACTLY in
// the FP32 accumulators of mma.sync.m16n8k16 (bf16 inputs, FP32 accumulation).  Chunks
// are scaled by 2^{-7(s+t)} (exact) and summed in double-float (FP32 pairs), and slice
// pairs with s + t <= S + 1 are kept.  The truncation error of the kept pairs is about
// 2^{-7S} relative to the row and column scales, so S = 7 gives FP64-level products and
// S = 3 about 1e-6, at 6 ... 28 tensor-core GEMMs per product instead of FP64 FMAs (which
// run 570x slower than bf16 mma.sync on this part).
#include <algorithm>
#include <cmath>
#include <cuda_bf16.h>

#include "internal.cuh"

namespace {

constexpr int OZ_BM = 128, OZ_BN = 64, OZ_BK = 64, OZ_THREADS = 256, OZ_STAGES = 3;
constexpr int OZ_BETA = 7;         // bits per digit slice
constexpr int OZ_CHUNK_KB = 16;    // k-blocks of 64 per exact FP32 chunk (1024)
constexpr int OZ_MAX_PAIRS = 64;

struct OzPairs {
  int n;
  unsigned char s[OZ_MAX_PAIRS], t[OZ_MAX_PAIRS];
};

struct OzParams {
  const __nv_bfloat16* A;  // S_A slices, each Mp x Kp row-major
  const __nv_bfloat16* B;  // S_B slices, each Np x Kp (column j of B^ contiguous)
  int64_t sliceA, sliceB;  // elements per slice
  int Kp;                  // padded K (multiple of 64)
  int nkb;                 // k-blocks of 64 per pair
  int tiles_m;
  int splits;
  OzPairs pairs;
  double* part;            // splits x (Np x Mp) partials, column-major (ld Mp)
  int Mp, Np;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                            uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// byte offset of element (row, k) in a [rows][64] bf16 tile with 16-byte chunks XOR-swizzled
__device__ __forceinline__ uint32_t swz(int row, int k) {
  return (uint32_t)(row * 128 + ((((k >> 3) ^ (row & 7))) << 4) + ((k & 7) << 1));
}

// error-free addition of x into the double-float (hi, lo)
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += err;
}

__global__ void __launch_bounds__(OZ_THREADS, 1) oz_gemm_kernel(const OzParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* sA = smem;                                    // stages x 128 x 64 bf16
  unsigned char* sB = smem + OZ_STAGES * OZ_BM * OZ_BK * 2;    // stages x 64 x 64 bf16
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 3, wn = warp >> 2;
  const int tm = blockIdx.x % p.tiles_m, tn = blockIdx.x / p.tiles_m;
  const int m0 = tm * OZ_BM, n0 = tn * OZ_BN;

  const int total = p.pairs.n * p.nkb;
  const int per = (total + p.splits - 1) / p.splits;
  const int q0 = min(total, (int)blockIdx.y * per), q1 = min(total, q0 + per);

  float acc[2][4][4];
  float hi[2][4][4], lo[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = hi[a][b][c] = lo[a][b][c] = 0.f;

  auto load_stage = [&](int q, int stage) {
    const int pr = q / p.nkb, kb = q - pr * p.nkb;
    const __nv_bfloat16* Ag = p.A + (int64_t)p.pairs.s[pr] * p.sliceA + (int64_t)m0 * p.Kp + kb * OZ_BK;
    const __nv_bfloat16* Bg = p.B + (int64_t)p.pairs.t[pr] * p.sliceB + (int64_t)n0 * p.Kp + kb * OZ_BK;
    const uint32_t sa = smem_u32(sA + stage * OZ_BM * OZ_BK * 2);
    const uint32_t sb = smem_u32(sB + stage * OZ_BN * OZ_BK * 2);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int idx = tid + i * OZ_THREADS;  // 0..1023
      const int row = idx >> 3, ch = idx & 7;
      cp_async16(sa + swz(row, ch * 8), Ag + (int64_t)row * p.Kp + ch * 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int idx = tid + i * OZ_THREADS;  // 0..511
      const int row = idx >> 3, ch = idx & 7;
      cp_async16(sb + swz(row, ch * 8), Bg + (int64_t)row * p.Kp + ch * 8);
    }
  };

#pragma unroll
  for (int st = 0; st < OZ_STAGES - 1; ++st) {
    if (q0 + st < q1) load_stage(q0 + st, st);
    cp_async_commit();
  }

  for (int q = q0; q < q1; ++q) {
    const int stage = (q - q0) % OZ_STAGES;
    cp_async_wait<OZ_STAGES - 2>();
    __syncthreads();
    {
      const int qn = q + OZ_STAGES - 1;
      if (qn < q1) load_stage(qn, (qn - q0) % OZ_STAGES);
      cp_async_commit();
    }
    const uint32_t sa = smem_u32(sA + stage * OZ_BM * OZ_BK * 2);
    const uint32_t sb = smem_u32(sB + stage * OZ_BN * OZ_BK * 2);
#pragma unroll
    for (int kk = 0; kk < OZ_BK / 16; ++kk) {
      uint32_t af[2][4], bf[4][2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int row = wm * 32 + mt * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
        const int k = kk * 16 + (lane >> 4) * 8;
        ldmatrix_x4(sa + swz(row, k), af[mt][0], af[mt][1], af[mt][2], af[mt][3]);
      }
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        const int row = wn * 32 + np * 16 + (lane & 7) + (lane >> 4) * 8;
        const int k = kk * 16 + ((lane >> 3) & 1) * 8;
        ldmatrix_x4(sb + swz(row, k), bf[2 * np][0], bf[2 * np][1], bf[2 * np + 1][0],
                    bf[2 * np + 1][1]);
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], af[mt], bf[nt][0], bf[nt][1]);
    }
    // drain the exact FP32 chunk at chunk ends, pair ends and the end of this CTA's range
    const int pr = q / p.nkb, kb = q - pr * p.nkb;
    if (((kb + 1) % OZ_CHUNK_KB) == 0 || kb == p.nkb - 1 || q == q1 - 1) {
      const float sc = ldexpf(1.0f, -OZ_BETA * (p.pairs.s[pr] + p.pairs.t[pr] + 2));
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            two_sum_acc(hi[a][b][c], lo[a][b][c], acc[a][b][c] * sc);
            acc[a][b][c] = 0.f;
          }
    }
  }
  cp_async_wait<0>();

  // partial (unscaled by the row/column exponents) -> p.part[split][col * Mp + row]
  double* P = p.part + (int64_t)blockIdx.y * p.Mp * p.Np;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int r = m0 + wm * 32 + mt * 16 + (lane >> 2);
      const int c = n0 + wn * 32 + nt * 8 + 2 * (lane & 3);
      P[(int64_t)c * p.Mp + r] = (double)hi[mt][nt][0] + (double)lo[mt][nt][0];
      P[(int64_t)(c + 1) * p.Mp + r] = (double)hi[mt][nt][1] + (double)lo[mt][nt][1];
      P[(int64_t)c * p.Mp + r + 8] = (double)hi[mt][nt][2] + (double)lo[mt][nt][2];
      P[(int64_t)(c + 1) * p.Mp + r + 8] = (double)hi[mt][nt][3] + (double)lo[mt][nt][3];
    }
}

// Complex epilogue: C(i, j) = 2^{eA(i)+eB(j)} (sum_s P[s](2i, j), sum_s P[s](2i+1, j)),
// out = alpha C + beta Cin + gamma D (out may alias Cin or D element-wise).
__global__ void oz_epilogue_kernel(const double* part, int splits, int Mp, int Np, const int* eA,
                                   const int* eB, int n, int m, double alpha, double beta,
                                   const zd* Cin, int64_t ldcin, double gamma, const zd* D,
                                   int64_t ldd, zd* out, int64_t ldo) {
  const int64_t total = (int64_t)n * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    double re = 0.0, im = 0.0;
    for (int s = 0; s < splits; ++s) {
      const double2 v = *reinterpret_cast<const double2*>(part + (int64_t)s * Mp * Np +
                                                          (int64_t)j * Mp + 2 * i);
      re += v.x;
      im += v.y;
    }
    // the kernel applied the slice-level scales 2^{-7(s+t)}; the row and column scales remain
    const int ex = eA[i] + eB[j];
    zd o = zmk(alpha * ldexp(re, ex), alpha * ldexp(im, ex));
    if (beta != 0.0) o = zadd(o, zscale(Cin[i + (int64_t)j * ldcin], beta));
    if (gamma != 0.0) o = zadd(o, zscale(D[i + (int64_t)j * ldd], gamma));
    out[i + (int64_t)j * ldo] = o;
  }
}

__device__ __forceinline__ int exponent_bound(double mx) {
  // smallest e with mx < 2^e (0 for mx == 0)
  if (!(mx > 0.0)) return 0;
  int e;
  frexp(mx, &e);
  return e;
}

// Digits of x (|x| < 2^e) for S slices: x 2^{7-e} = d_1 + 2^{-7} d_2 + ...
__device__ __forceinline__ void digits(double x, int e, int S, __nv_bfloat16* out, int64_t stride) {
  double r = ldexp(x, OZ_BETA - e);
  for (int s = 0; s < S; ++s) {
    const double d = rint(r);
    out[s * stride] = __float2bfloat16_rn((float)d);
    r = ldexp(r - d, OZ_BETA);
  }
}

__device__ double block_max(double v) {
  __shared__ double sh[32];
  __shared__ double res;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (lane == 0) res = t;
  }
  __syncthreads();
  const double r = res;
  __syncthreads();
  return r;
}

// A-side slices of the real embedding of Hermitian Hs: one CTA per complex row i.
// Row i of Hs is conj(column i), read contiguously.  Real rows 2i, 2i+1; columns 2k, 2k+1:
//   [ Re h  -Im h ]      h = Hs(i, k) = conj(Hs(k, i))
//   [ Im h   Re h ]
__global__ void oz_slice_hermitian_kernel(const zd* Hs, int64_t ldh, int n, int S,
                                          __nv_bfloat16* A, int64_t sliceA, int Kp, int* eA) {
  const int i = blockIdx.x;
  const zd* col = Hs + (int64_t)i * ldh;
  double mx = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const zd h = col[k];
    mx = fmax(mx, fmax(fabs(h.x), fabs(h.y)));
  }
  mx = block_max(mx);
  const int e = exponent_bound(mx);
  if (threadIdx.x == 0) eA[i] = e;
  __nv_bfloat16* r0 = A + (int64_t)(2 * i) * Kp;
  __nv_bfloat16* r1 = r0 + Kp;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const zd hc = col[k];
    const double re = hc.x, im = -hc.y;  // H(i,k) = conj(Hs(k,i))
    digits(re, e, S, r0 + 2 * k, sliceA);
    digits(-im, e, S, r0 + 2 * k + 1, sliceA);
    digits(im, e, S, r1 + 2 * k, sliceA);
    digits(re, e, S, r1 + 2 * k + 1, sliceA);
  }
}

// B-side slices of Y^ (the n x m complex block read as a 2n x m real array): one CTA per
// column j; columns j >= m of the padded block are zero.
__global__ void oz_slice_cols_kernel(const zd* Y, int64_t ldy, int n, int m, int S,
                                     __nv_bfloat16* B, int64_t sliceB, int Kp, int* eB) {
  const int j = blockIdx.x;
  __nv_bfloat16* col = B + (int64_t)j * Kp;
  if (j >= m) {
    for (int k = threadIdx.x; k < Kp; k += blockDim.x)
      for (int s = 0; s < S; ++s) col[s * sliceB + k] = __float2bfloat16_rn(0.f);
    if (threadIdx.x == 0) eB[j] = 0;
    return;
  }
  const zd* y = Y + (int64_t)j * ldy;
  double mx = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) mx = fmax(mx, fmax(fabs(y[k].x), fabs(y[k].y)));
  mx = block_max(mx);
  const int e = exponent_bound(mx);
  if (threadIdx.x == 0) eB[j] = e;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const zd v = y[k];
    digits(v.x, e, S, col + 2 * k, sliceB);
    digits(v.y, e, S, col + 2 * k + 1, sliceB);
  }
}

int choose_oz_splits(int tiles, int total_kb, size_t cap_elems, int64_t tile_elems) {
  const int sms = sm_count();
  int best = 1;
  double best_cost = (double)((tiles + sms - 1) / sms);
  for (int S = 2; S <= 32; ++S) {
    if (total_kb / S < 4) break;
    if ((size_t)S * (size_t)tile_elems > cap_elems) break;
    const int64_t units = (int64_t)tiles * S;
    const double cost = (double)((units + sms - 1) / sms) / S + 0.004 * S;
    if (cost < best_cost * 0.97) { best_cost = cost; best = S; }
  }
  return best;
}

}  // namespace

// ---------------------------------------------------------------------------- host side
int oz_padded_k(int n) { return ((2 * n + OZ_BK - 1) / OZ_BK) * OZ_BK; }
int oz_padded_m(int n) { return ((2 * n + OZ_BM - 1) / OZ_BM) * OZ_BM; }
int oz_padded_n(int m) { return ((m + OZ_BN - 1) / OZ_BN) * OZ_BN; }

cudaError_t oz_slice_hermitian(const zd* Hs, int64_t ldh, int n, int S, OzWorkspace& oz,
                               cudaStream_t s) {
  const int Kp = oz_padded_k(n), Mp = oz_padded_m(n);
  if (S > oz.S_max || Kp > oz.Kp_max || Mp > oz.Mp_max) return cudaErrorInvalidValue;
  oz.Kp = Kp;
  oz.Mp = Mp;
  oz.S_A = S;
  oz.sliceA = (int64_t)Mp * Kp;
  // zero the padding (rows >= 2n and columns >= 2n) once per slicing
  cudaError_t e = cudaMemsetAsync(oz.A, 0, sizeof(__nv_bfloat16) * (size_t)S * oz.sliceA, s);
  if (e != cudaSuccess) return e;
  oz_slice_hermitian_kernel<<<n, 256, 0, s>>>(Hs, ldh, n, S, oz.A, oz.sliceA, Kp, oz.eA);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}

// out(n x m) = alpha Hs Y + beta Cin + gamma D with Hs given by its slices in oz (S_A of
// them) and Y sliced here into S slices; pairs (s, t) with s + t <= S + 1.
cudaError_t oz_filter_product(const zd* Y, int64_t ldy, int n, int m, int S, double alpha,
                              double beta, const zd* Cin, int64_t ldcin, double gamma, const zd* D,
                              int64_t ldd, zd* out, int64_t ldo, OzWorkspace& oz, cudaStream_t s,
                              cudaEvent_t ev_gemm_begin, cudaEvent_t ev_gemm_end) {
  if (m <= 0) return cudaSuccess;
  if (S > oz.S_A || S < 1) return cudaErrorInvalidValue;
  const int Np = oz_padded_n(m);
  if (Np > oz.Np_max) return cudaErrorInvalidValue;
  const int Kp = oz.Kp, Mp = oz.Mp;
  const int64_t sliceB = (int64_t)Np * Kp;
  // B-side slices (padding rows k >= 2n of each column are zeroed by the memset)
  cudaError_t e = cudaMemsetAsync(oz.B, 0, sizeof(__nv_bfloat16) * (size_t)S * sliceB, s);
  if (e != cudaSuccess) return e;
  oz_slice_cols_kernel<<<Np, 256, 0, s>>>(Y, ldy, n, m, S, oz.B, sliceB, Kp, oz.eB);
  CHFSI_COUNT_LAUNCH();
  OzParams p;
  p.A = oz.A;
  p.B = oz.B;
  p.sliceA = oz.sliceA;
  p.sliceB = sliceB;
  p.Kp = Kp;
  p.nkb = Kp / OZ_BK;
  p.tiles_m = Mp / OZ_BM;
  p.Mp = Mp;
  p.Np = Np;
  p.pairs.n = 0;
  for (int lvl = 2; lvl <= S + 1; ++lvl)
    for (int si = 1; si <= S; ++si) {
      const int ti = lvl - si;
      if (ti < 1 || ti > S) continue;
      p.pairs.s[p.pairs.n] = (unsigned char)(si - 1);
      p.pairs.t[p.pairs.n] = (unsigned char)(ti - 1);
      ++p.pairs.n;
    }
  const int tiles = p.tiles_m * (Np / OZ_BN);
  p.splits = choose_oz_splits(tiles, p.pairs.n * p.nkb, oz.part_elems, (int64_t)Mp * Np);
  p.part = oz.part;
  const size_t smem = (size_t)OZ_STAGES * (OZ_BM + OZ_BN) * OZ_BK * 2;
  static bool attr_set = false;
  if (!attr_set) {
    e = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  if (ev_gemm_begin) cudaEventRecord(ev_gemm_begin, s);
  oz_gemm_kernel<<<dim3(tiles, p.splits), OZ_THREADS, smem, s>>>(p);
  CHFSI_COUNT_LAUNCH();
  if (ev_gemm_end) cudaEventRecord(ev_gemm_end, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t tot = (int64_t)n * m;
  const int blocks = (int)std::min<int64_t>(4 * sm_count(), (tot + 255) / 256);
  oz_epilogue_kernel<<<blocks, 256, 0, s>>>(oz.part, p.splits, Mp, Np, oz.eA, oz.eB, n, m, alpha,
                                            beta, Cin, ldcin, gamma, D, ldd, out, ldo);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}

int64_t oz_pair_count(int S) { return (int64_t)S * (S + 1) / 2; }

cudaError_t oz_alloc(OzWorkspace& oz, int n_max, int blk_max, int S_max) {
  oz.S_max = S_max;
  oz.Kp_max = oz_padded_k(n_max);
  oz.Mp_max = oz_padded_m(n_max);
  oz.Np_max = oz_padded_n(blk_max);
  cudaError_t e;
  e = cudaMalloc((void**)&oz.A, sizeof(__nv_bfloat16) * (size_t)S_max * oz.Mp_max * oz.Kp_max);
  if (e != cudaSuccess) return e;
  e = cudaMalloc((void**)&oz.B, sizeof(__nv_bfloat16) * (size_t)S_max * oz.Np_max * oz.Kp_max);
  if (e != cudaSuccess) return e;
  e = cudaMalloc((void**)&oz.eA, sizeof(int) * (size_t)oz.Mp_max);
  if (e != cudaSuccess) return e;
  e = cudaMalloc((void**)&oz.eB, sizeof(int) * (size_t)oz.Np_max);
  if (e != cudaSuccess) return e;
  oz.part_elems = (size_t)16 * oz.Mp_max * oz.Np_max;
  e = cudaMalloc((void**)&oz.part, sizeof(double) * oz.part_elems);
  return e;
}

void oz_free(OzWorkspace& oz) {
  if (oz.A) cudaFree(oz.A);
  if (oz.B) cudaFree(oz.B);
  if (oz.eA) cudaFree(oz.eA);
  if (oz.eB) cudaFree(oz.eB);
  if (oz.part) cudaFree(oz.part);
  oz = OzWorkspace{};
}
