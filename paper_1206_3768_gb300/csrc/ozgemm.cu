// Split-BF16 tensor-core products for the Chebyshev filter (mixed-precision filter).
//
// A complex FP64 product C = Hs Y (Hs n x n Hermitian, Y n x m) is computed as the real
// product C^ = H^ Y^ of the 2n x 2n real embedding H^ (rows and columns interleaved as
// (re, im), so that Y^ and C^ are the complex column-major arrays read as real arrays)
// with the 2n x m real Y^.  Each operand is split into S "digit slices":
//
//     H^(r, k) = 2^{eA(r)} sum_s a_s(r, k) 2^{-7 s},   |a_1| <= 129, |a_{s>1}| <= 64
//     Y^(k, j) = 2^{eB(j)} sum_t b_t(k, j) 2^{-7 t}
//
// with power-of-two scales per (complex) row of Hs and per column of Y.  Every digit is an
// integer that bf16 holds exactly, every digit product is exact in FP32, and a sum of at
// most 960 such products stays below 2^24, so each K-chunk of 960 accumulates EXACTLY in
// the FP32 accumulators of mma.sync.m16n8k16 (bf16 inputs, FP32 accumulation).  Chunks
// are scaled by 2^{-7(s+t)} (exact) and summed in double-float (FP32 pairs), and slice
// pairs with s + t <= S + 1 are kept.  The truncation error of the kept pairs is about
// 2^{-7S} relative to the row and column scales, so S = 7 gives FP64-level products and
// S = 3 about 1e-6, at 6 ... 28 tensor-core GEMMs per product instead of FP64 FMAs (which
// run 570x slower than bf16 mma.sync on this part).
#include <algorithm>
#include <cmath>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "internal.cuh"

namespace {

constexpr int OZ_BM = 128, OZ_BN = 64, OZ_BK = 64, OZ_THREADS = 256, OZ_STAGES = 3;
constexpr int OZ_BETA = 7;         // bits per digit slice
constexpr int OZ_CHUNK_KB = 15;    // k-blocks of 64 per exact FP32 chunk (960 terms: 960 * 129^2 < 2^24)
constexpr int OZ_MAX_PAIRS = 64;

struct OzPairs {
  int n;
  unsigned char s[OZ_MAX_PAIRS], t[OZ_MAX_PAIRS];
};

struct OzParams {
  int a_lower;             // A^ is the embedding of a lower-triangular matrix: skip zero k-blocks
  int c_lower;             // only the lower triangle of the complex result is needed
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
  if (p.c_lower && n0 > (m0 + OZ_BM - 1) / 2) return;
  const int nkb = p.a_lower ? min(p.nkb, m0 / OZ_BK + OZ_BM / OZ_BK) : p.nkb;

  const int total = p.pairs.n * nkb;
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
    const int pr = q / nkb, kb = q - pr * nkb;
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
    const int pr = q / nkb, kb = q - pr * nkb;
    if (((kb + 1) % OZ_CHUNK_KB) == 0 || kb == nkb - 1 || q == q1 - 1) {
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
// out = alpha C + beta Cin + gamma D (out may alias Cin or D element-wise).  The partial
// sums are FP64 (pairs == 0) or double-float (hi, lo) pairs of FP32 (pairs != 0), which are
// summed over the splits in double-float arithmetic and converted to FP64 once.
__global__ void oz_epilogue_kernel(const double* part, int splits, int Mp, int Np, const int* eA,
                                   const int* eB, int n, int m, double alpha, double beta,
                                   const zd* Cin, int64_t ldcin, double gamma, const zd* D,
                                   int64_t ldd, zd* out, int64_t ldo, int lower, int pairs) {
  const int64_t total = (int64_t)n * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (lower && j > i) continue;
    double re = 0.0, im = 0.0;
    if (pairs) {
      float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
      for (int s = 0; s < splits; ++s) {
        const float4 v = *reinterpret_cast<const float4*>(part + (int64_t)s * Mp * Np +
                                                          (int64_t)j * Mp + 2 * i);
        two_sum_acc(rh, rl, v.x);
        rl += v.y;
        two_sum_acc(ih, il, v.z);
        il += v.w;
      }
      re = (double)rh + (double)rl;
      im = (double)ih + (double)il;
    } else {
      for (int s = 0; s < splits; ++s) {
        const double2 v = *reinterpret_cast<const double2*>(part + (int64_t)s * Mp * Np +
                                                            (int64_t)j * Mp + 2 * i);
        re += v.x;
        im += v.y;
      }
    }
    // the kernel applied the slice-level scales 2^{-7(s+t)}; the row and column scales remain
    const int ex = eA[i] + eB[j];
    zd o = zmk(alpha * ldexp(re, ex), alpha * ldexp(im, ex));
    if (beta != 0.0) o = zadd(o, zscale(Cin[i + (int64_t)j * ldcin], beta));
    if (gamma != 0.0) o = zadd(o, zscale(D[i + (int64_t)j * ldd], gamma));
    out[i + (int64_t)j * ldo] = o;
  }
}


// ============================================================================ tcgen05 path
// The same digit products on the 5th-generation tensor cores: TMA (128-byte swizzle) stages
// a 128 x 64 bf16 tile of A and an (up to) 160 x 64 tile of B in shared memory, one elected
// thread issues tcgen05.mma (kind::f16, bf16 inputs, FP32 accumulator in tensor memory, N up
// to 160 so that a 130-column block is one tile and a 320-column block two), and sixteen
// drain warps fold each exact 960-term chunk into double-float sums.  Tensor memory (512
// columns): two sets of accumulators used alternately (one fills while the other drains) and
// the high words of the sums after them; the low words live in the drain threads' registers.
// Slice groups: the pairs are issued in groups (s, t0 .. t0 + g - 1) that share the A slice
// s.  One stage holds one A tile and the B tiles of the whole group (consecutive slices of B
// are consecutive rows of its buffer, so one TMA box of g x Np rows), and the MMA thread
// issues the group's products into g accumulators.  The A stream then carries one tile per
// group instead of one per pair.  g = 1 for blocks wider than 96 columns (two 160-column
// accumulators at columns 0 and 160, high words at 320); narrower blocks take g up to 7 as
// tensor memory allows: 2 g accumulators of the block's width (rounded up to 32 columns)
// plus the high words.
// Clusters: the CTAs of consecutive row tiles (2 or 4) form a cluster and share every B
// tile: each CTA loads its share of the B box and multicasts it to the cluster, and the MMAs
// of every CTA release a stage to all of them (the empty barriers count one arrival per
// CTA), which divides the B stream from L2 by the cluster size.
// Warp 0 issues TMA loads, warp 1 issues MMAs, warps 2..17 drain: four warps per group of 32
// tensor-memory lanes; warp h of a lane group owns the 8-column blocks h, h + 4, ... of the
// tile, so that narrow blocks still spread over all four.  18 warps allow 112 registers per
// thread.  Every wait on an mbarrier is bounded; a wait that runs out sets DEV_TIMEOUT and the
// CTA unwinds (waiting, again bounded, for its own copies and MMAs) before freeing tensor
// memory.
constexpr int TC_BM = 128, TC_BN = 160, TC_BK = 64;
constexpr int TC_DWQ = 3;                                  // drain warps per 32-lane quarter
constexpr int TC_THREADS = 64 + 32 * 4 * TC_DWQ;           // producer, MMA issuer, drain warps
// The ring holds as many stages as fit: 6 for a 144-row B box, up to TC_MAX_STAGES for narrow
// blocks, whose smaller B boxes leave room for more of the (dominant) A stream in flight.
constexpr int TC_MAX_STAGES = 12;
constexpr int TC_SMEM_BUDGET = 227 * 1024 - 1024 - 512;  // dynamic shared memory for the ring
constexpr int TC_DRAIN_THREADS = TC_THREADS - 64;
constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;       // 16 KB per stage
constexpr int TC_ACC1 = 160, TC_HI = 320;           // tensor-memory columns for groups of one
constexpr int TC_LO = 480;                         // low words of tile columns 128..159
constexpr int TC_GROUP_MAX_N = 96;                  // widest block issued in groups of g > 1
constexpr int TC_GROUP_MAX = 7;
static_assert((16 * TC_BK * 2) % 1024 == 0, "B stages (16-row multiples) stay 1024-byte aligned");
static_assert(TC_HI + TC_BN <= TC_LO && TC_LO + (TC_BN - 128) <= 512 && TC_ACC1 + TC_BN <= TC_HI,
              "tensor-memory layout");
constexpr long kMbarSpinLimit = 1L << 26;

struct TcParams {
  int a_lower, c_lower;                      // as in OzParams
  int b_tri;                                 // op(B) (complex) zero for k > j (1) or k < j (2)
  int nkb, tiles_m, splits, Mp, Np, n_real;  // n_real: columns of B^ that hold data
  int b_box_rows;                            // rows of the B box (<= TC_BN, multiple of 16)
  int stages;                                // TMA ring depth (<= TC_MAX_STAGES)
  int pair_split;                            // splits partition the slice groups (else k-blocks)
  int group;                                 // g: largest group (B box = g x Np rows when g > 1)
  int acc_stride;                            // tensor-memory columns between accumulators
  int ngroups;
  unsigned char gs[OZ_MAX_PAIRS], gt[OZ_MAX_PAIRS], gc[OZ_MAX_PAIRS];  // group: s, first t, size
  double* part;
  int* status;
  long long spin_limit;                      // polls before a first-level wait gives up
  int cl;                                    // CTAs per cluster along M sharing the B tiles (1, 2, 4)
  int tiles_m_pad;                           // tiles_m rounded up to a multiple of cl
  int col_major_order;                       // 1: blockIdx.x runs over column tiles first (cl == 1)
  // Gauss form (nz = 3): blockIdx.z picks one of three real products whose operands follow
  // each other in the slice buffers (a_zrows rows of A, b_zrows rows of B apart) and whose
  // split partials follow each other in part (splits x Mp x Np entries apart)
  int nz;
  int a_zrows, b_zrows;
  int kfac;  // real k (and rows of A) per complex index: 2 in the embedding, 1 in the Gauss form
};

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar));
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity));
  return ok != 0;
}
// Bounded wait: false (with DEV_TIMEOUT set and the CTA's abort flag raised) if it ran out
// or another role of this CTA already gave up.
// The single-thread producer and MMA roles spin without back-off (their waits sit on the
// critical path); the drain warps back off after a while.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          int* status, long long limit, bool backoff = false) {
  long long it = 0;
  while (!mbar_try(bar, parity)) {
    if (++it > limit) {
      *abort_flag = 1;
      atomicOr(status, DEV_TIMEOUT);
      return false;
    }
    if ((it & 255) == 0 && *abort_flag) return false;
    if (backoff && it > 1024) __nanosleep(64);
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
// The same copy delivered to every CTA of the cluster in `mask`, at the same shared-memory
// offsets (destination and mbarrier) as this CTA's.
__device__ __forceinline__ void tma_load_2d_mc(uint32_t dst, const CUtensorMap* map, int x, int y,
                                               uint32_t bar, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1, {%2, %3}], [%4], %5;\n"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "h"(mask)
      : "memory");
}
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                     // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                     // descriptor version
  d |= (uint64_t)2 << 61;                     // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, bf16 A and B, both K-major.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
               ::"r"(bar) : "memory");
}
// Arrive (once the issued MMAs complete) on the mbarrier at this offset in every CTA of mask.
__device__ __forceinline__ void tc_commit_mc(uint32_t bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;\n"
      ::"r"(bar), "h"(mask) : "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n"
               ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]));
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};\n"
               ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

__global__ void __launch_bounds__(TC_THREADS, 1)
    oz_gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const TcParams p) {
  extern __shared__ unsigned char tc_smem_raw[];
  const uintptr_t base = (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023;
  unsigned char* sA = reinterpret_cast<unsigned char*>(base);
  const int NS = p.stages, b_stage = p.b_box_rows * TC_BK * 2;  // B stage bytes: a multiple of 2048
  unsigned char* sB = sA + NS * TC_A_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + NS * b_stage);
  // bars: full[STAGES], empty[STAGES], accf[2], acce[2], done[1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NS + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // tile order: row tiles fastest, or (col_major_order) the column tiles of one row tile next
  // to each other, so that they stream the same A panels at about the same time
  const int tiles_n = (int)(gridDim.x / (unsigned)p.tiles_m_pad);
  const int tm = p.col_major_order ? (int)blockIdx.x / tiles_n : (int)blockIdx.x % p.tiles_m_pad;
  const int tn = p.col_major_order ? (int)blockIdx.x % tiles_n : (int)blockIdx.x / p.tiles_m_pad;
  const int m0 = tm * TC_BM, n0 = tn * TC_BN;
  // Clusters of p.cl CTAs on consecutive row tiles share every B tile: each CTA loads 1/cl of
  // the B box and multicasts it to the whole cluster, so all CTAs of a cluster must walk the
  // same stages.  Their work is therefore decided by the cluster's last row tile (the widest
  // k-range of a lower-triangular A, the last tile to reach the diagonal); the extra work is
  // exact (zero blocks of A) or unused (tiles above the diagonal, rows past Mp).
  const int crank = p.cl > 1 ? (int)cluster_ctarank() : 0;
  const int m0_last = (tm - crank + p.cl - 1) * TC_BM;
  const uint16_t cmask = (uint16_t)((1u << p.cl) - 1u);
  if (p.c_lower && n0 > (m0_last + TC_BM - 1) / p.kfac) return;  // above the diagonal: not needed
  // k-blocks of this CTA: split y takes [y per, (y + 1) per) of the tile's nonzero k-blocks.
  // The work is ordered panel-major: for each panel of at most OZ_CHUNK_KB k-blocks, every
  // slice pair in turn (one exact chunk each), so consecutive chunks reuse the same panel of
  // an A slice from L2 while it is hot.
  const int ncols = min(TC_BN, ((p.n_real - n0 + 15) / 16) * 16);  // MMA N for this tile
  // nonzero k-blocks of the tile (k in real units, kfac per complex index): below
  // (m0 + 128) / 64 for a lower-triangular A (rows are in the same units); from kfac n0 / 64
  // for a lower-triangular B (zero for k < j); below kfac (n0 + ncols) / 64 for an
  // upper-triangular B (zero for k > j)
  int kb_first = 0, nkb = p.a_lower ? min(p.nkb, m0_last / TC_BK + TC_BM / TC_BK) : p.nkb;
  if (p.b_tri == 2) kb_first = min(nkb, (p.kfac * n0) / TC_BK);
  if (p.b_tri == 1) nkb = min(nkb, (p.kfac * (n0 + ncols) + TC_BK - 1) / TC_BK);
  // split y takes either a range of k-blocks (all groups) or, for short K (one panel), a
  // range of slice groups (all k-blocks)
  int kb_lo = kb_first, kb_hi = nkb, pr_lo = 0, pr_hi = p.ngroups;
  if (p.pair_split) {
    const int pp = (p.ngroups + p.splits - 1) / p.splits;
    pr_lo = min(p.ngroups, (int)blockIdx.y * pp);
    pr_hi = min(p.ngroups, pr_lo + pp);
  } else {
    const int per = (nkb - kb_first + p.splits - 1) / p.splits;
    kb_lo = min(nkb, kb_first + (int)blockIdx.y * per);
    kb_hi = min(nkb, kb_lo + per);
  }
  const int npr = pr_hi - pr_lo;
  // tensor-memory columns: accumulator j of buffer b at (b g + j) acc_stride, high words after
  const int G = p.group;
  const uint32_t acc_stride = (uint32_t)p.acc_stride, hi_col = 2u * (uint32_t)G * acc_stride;
  const uint32_t b_pair_bytes = (uint32_t)p.Np * TC_BK * 2;  // B tile of one slice in a group box
  const int b_share = p.b_box_rows / p.cl;                   // B rows each CTA of a cluster loads

  const uint32_t sA_u = smem_u32(sA), sB_u = smem_u32(sB);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * NS;
  const uint32_t accf0 = empty0 + 8 * NS, acce0 = accf0 + 16, done_bar = acce0 + 16;

  if (tid == 0) {
    for (int i = 0; i < NS; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(empty0 + 8 * i, p.cl);  // released by the MMAs of every CTA of the cluster
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, TC_DRAIN_THREADS);
    }
    mbar_init(done_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(
        smem_u32(tmem_slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  __syncthreads();
  // every CTA of the cluster has initialised its barriers before any copy or commit reaches them
  if (p.cl > 1) cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      // ring position kept incrementally (no division on this single-thread issue path)
      int i = 0, stage = 0;
      uint32_t phase = 0;
      bool stop = false;
      for (int k0 = kb_lo; k0 < kb_hi && !stop; k0 += OZ_CHUNK_KB) {
        const int k1 = min(kb_hi, k0 + OZ_CHUNK_KB);
        for (int pr = pr_lo; pr < pr_hi && !stop; ++pr) {
          const int arow = (int)blockIdx.z * p.a_zrows + p.gs[pr] * p.Mp + m0;
          const int brow = (int)blockIdx.z * p.b_zrows + p.gt[pr] * p.Np + n0;
          for (int kb = k0; kb < k1; ++kb, ++i) {
            const uint32_t fb = full0 + 8 * stage;
            if (i >= NS && !mbar_wait(empty0 + 8 * stage, phase ^ 1, abort_flag, p.status, p.spin_limit)) {
              stop = true;
              break;
            }
            mbar_expect_tx(fb, TC_A_BYTES + b_stage);
            tma_load_2d(sA_u + stage * TC_A_BYTES, &tmA, kb * TC_BK, arow, fb);
            if (p.cl > 1)  // this CTA's share of the B box, to every CTA of the cluster
              tma_load_2d_mc(sB_u + stage * b_stage + (uint32_t)(crank * b_share) * (TC_BK * 2), &tmB,
                             kb * TC_BK, brow + crank * b_share, fb, cmask);
            else
              tma_load_2d(sB_u + stage * b_stage, &tmB, kb * TC_BK, brow, fb);
            if (++stage == NS) {
              stage = 0;
              phase ^= 1;
            }
          }
        }
      }
      // on abort: let the copies already issued (stages i - STAGES .. i - 1) land before the
      // CTA can exit
      if (*abort_flag) {
        for (int j = max(0, i - NS); j < i; ++j) {
          long it = 0;
          while (!mbar_try(full0 + 8 * (j % NS), (j / NS) & 1) && ++it < kMbarSpinLimit) {}
        }
      } else if (p.cl > 1) {
        // the B shares this CTA sent to the cluster: every CTA has consumed them (so they have
        // landed) before this CTA may exit
        for (int j = max(0, i - NS); j < i; ++j) {
          long it = 0;
          while (!mbar_try(empty0 + 8 * (j % NS), (j / NS) & 1) && ++it < kMbarSpinLimit) {}
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(TC_BM, ncols);
      int chunk = 0, stage = 0;
      uint32_t phase = 0;
      bool stop = false;
      for (int k0 = kb_lo; k0 < kb_hi && !stop; k0 += OZ_CHUNK_KB) {
        const int k1 = min(kb_hi, k0 + OZ_CHUNK_KB);
        for (int pr = pr_lo; pr < pr_hi && !stop; ++pr, ++chunk) {
          // accumulator chunk & 1 is free once the drain has finished chunk - 2
          if (chunk >= 2 && !mbar_wait(acce0 + 8 * (chunk & 1), ((chunk >> 1) - 1) & 1, abort_flag, p.status,
                                     p.spin_limit)) {
            stop = true;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(chunk & 1) * (uint32_t)G * acc_stride;
          const int gc = p.gc[pr];
          for (int kb = k0; kb < k1; ++kb) {
            if (!mbar_wait(full0 + 8 * stage, phase, abort_flag, p.status, p.spin_limit)) {
              stop = true;
              break;
            }
            tc_fence_after();
            const uint32_t a_s = sA_u + stage * TC_A_BYTES, b_s = sB_u + stage * b_stage;
            // pair j of the group: B tile j of the box into accumulator j
            for (int j = 0; j < gc; ++j) {
#pragma unroll
              for (int kk = 0; kk < TC_BK / 16; ++kk)
                tc_mma(d + (uint32_t)j * acc_stride, sw128_desc(a_s + kk * 32),
                       sw128_desc(b_s + (uint32_t)j * b_pair_bytes + kk * 32), idesc,
                       (kb == k0 && kk == 0) ? 0u : 1u);
            }
            if (p.cl > 1) tc_commit_mc(empty0 + 8 * stage, cmask);
            else tc_commit(empty0 + 8 * stage);
            if (kb == k1 - 1) tc_commit(accf0 + 8 * (chunk & 1));
            if (++stage == NS) {
              stage = 0;
              phase ^= 1;
            }
          }
        }
      }
      // all MMAs issued by this thread are complete once done_bar fires
      tc_commit(done_bar);
      long it = 0;
      while (!mbar_try(done_bar, 0) && ++it < kMbarSpinLimit) {}
    }
  } else {
    // ------------------------------------------------------------ drain warps (2..13)
    // Thread (quarter, lane) of warp h (0..2 within its lane group) owns row 32 * quarter +
    // lane of the tile and the 8-column blocks h + 3 i: the high words of its sums sit in
    // tensor memory, the low words of columns 0..127 in lo[] (registers; the block loops below
    // are unrolled so that every index into lo[] is a constant) and those of columns 128..159
    // in the last 32 tensor-memory columns (blocks 16..19 are only used with groups of one,
    // whose high words end at column 480).  Tensor memory is moved in blocks of 8 columns to
    // keep the live registers within the 128 that 14 warps allow.
    const int quarter = warp & 3;  // tensor-memory lanes 32*quarter .. +31
    constexpr int kRegCols = 128;                                       // columns with lo[] in registers
    constexpr int kBlocks = (kRegCols / 8 + TC_DWQ - 1) / TC_DWQ;       // register blocks per warp
    constexpr int kTmBlocks = ((TC_BN - kRegCols) / 8 + TC_DWQ - 1) / TC_DWQ;  // tensor-memory blocks
    const int h = (warp - 2) >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const int reg_cols = min(ncols, kRegCols);
    float lo[kBlocks * 8];
    {
      uint32_t zero[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) zero[j] = 0u;
#pragma unroll
      for (int c = 0; c < kBlocks; ++c) {
        // only the tile's columns: with groups the high words end at the last allocated column
        const int col = 8 * (TC_DWQ * c + h);
        if (col < reg_cols) tmem_st8(lane_base + hi_col + col, zero);
#pragma unroll
        for (int j = 0; j < 8; ++j) lo[c * 8 + j] = 0.f;
      }
#pragma unroll
      for (int t = 0; t < kTmBlocks; ++t) {
        const int col = kRegCols + 8 * (TC_DWQ * t + h);
        if (col < ncols) {
          tmem_st8(lane_base + hi_col + col, zero);
          tmem_st8(lane_base + TC_LO + (col - kRegCols), zero);
        }
      }
      tmem_wait_st();
    }
    int chunk = 0;
    bool ok = true;
    const int nchunks = (kb_hi > kb_lo && npr > 0) ? ((kb_hi - kb_lo + OZ_CHUNK_KB - 1) / OZ_CHUNK_KB) * npr : 0;
    for (; chunk < nchunks && ok; ++chunk) {
      const int b = chunk & 1;
      if (!mbar_wait(accf0 + 8 * b, (chunk >> 1) & 1, abort_flag, p.status, p.spin_limit, true)) { ok = false; break; }
      tc_fence_after();
      const int pr = pr_lo + chunk % npr;
      const int gc = p.gc[pr];
      const float sc0 = ldexpf(1.0f, -OZ_BETA * (p.gs[pr] + p.gt[pr] + 2));
      const uint32_t acc_base = lane_base + (uint32_t)b * (uint32_t)G * acc_stride;
#pragma unroll
      for (int c = 0; c < kBlocks; ++c) {
        const int col = 8 * (TC_DWQ * c + h);
        if (col < reg_cols) {
          uint32_t acc[8], hi[8];
          tmem_ld8(lane_base + hi_col + col, hi);
          float sc = sc0;
          for (int j = 0; j < gc; ++j) {  // pair (s, t0 + j), scale 2^{-7 (s + t0 + j + 2)}
            tmem_ld8(acc_base + (uint32_t)j * acc_stride + col, acc);
            tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              float hq = __uint_as_float(hi[q]);
              two_sum_acc(hq, lo[c * 8 + q], __uint_as_float(acc[q]) * sc);
              hi[q] = __float_as_uint(hq);
            }
            sc *= 0.0078125f;  // 2^-7
          }
          tmem_st8(lane_base + hi_col + col, hi);
        }
      }
#pragma unroll
      for (int t = 0; t < kTmBlocks; ++t) {  // groups of one: a single pair per chunk
        const int col = kRegCols + 8 * (TC_DWQ * t + h);
        if (col < ncols) {
#pragma unroll
          for (int half = 0; half < 8; half += 4) {  // four columns at a time (registers)
            uint32_t acc[4], hi[4], lw[4];
            tmem_ld4(lane_base + hi_col + col + half, hi);
            tmem_ld4(lane_base + TC_LO + (col - kRegCols) + half, lw);
            tmem_ld4(acc_base + col + half, acc);
            tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              float hq = __uint_as_float(hi[q]), lq = __uint_as_float(lw[q]);
              two_sum_acc(hq, lq, __uint_as_float(acc[q]) * sc0);
              hi[q] = __float_as_uint(hq);
              lw[q] = __float_as_uint(lq);
            }
            tmem_st4(lane_base + hi_col + col + half, hi);
            tmem_st4(lane_base + TC_LO + (col - kRegCols) + half, lw);
          }
        }
      }
      tmem_wait_st();
      tc_fence_before();
      mbar_arrive(acce0 + 8 * b);
    }
    if (ok && !*abort_flag && m0 < p.Mp) {
      // partial sums of this split as (hi, lo) pairs: P[split][col * Mp + row]
      float2* P = reinterpret_cast<float2*>(p.part) +
                  ((int64_t)blockIdx.z * p.splits + blockIdx.y) * p.Mp * p.Np;
      const int row = m0 + quarter * 32 + lane;
#pragma unroll
      for (int c = 0; c < kBlocks; ++c) {
        const int col0 = 8 * (TC_DWQ * c + h);
        if (col0 < reg_cols) {
          uint32_t hi[8];
          tmem_ld8(lane_base + hi_col + col0, hi);
          tmem_wait_ld();
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int col = n0 + col0 + q;
            if (col < p.Np)
              P[(int64_t)col * p.Mp + row] = make_float2(__uint_as_float(hi[q]), lo[c * 8 + q]);
          }
        }
      }
#pragma unroll
      for (int t = 0; t < kTmBlocks; ++t) {
        const int col0 = kRegCols + 8 * (TC_DWQ * t + h);
        if (col0 < ncols) {
          uint32_t hi[8], lw[8];
          tmem_ld8(lane_base + hi_col + col0, hi);
          tmem_ld8(lane_base + TC_LO + (col0 - kRegCols), lw);
          tmem_wait_ld();
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int col = n0 + col0 + q;
            if (col < p.Np)
              P[(int64_t)col * p.Mp + row] = make_float2(__uint_as_float(hi[q]), __uint_as_float(lw[q]));
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem));
  // no CTA leaves while a CTA of its cluster may still address its shared memory
  if (p.cl > 1) cluster_sync_all();
}

// Digit extraction with integer operations only (the FP64 pipe of this part is 1/64 of the
// FP32 rate, so shifting the 53-bit significand is much cheaper than FP64 arithmetic).
// |x| is a non-negative double: its bit pattern orders like its value.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}
// smallest e with max < 2^e, from the bit pattern of max (0 for max == 0)
__device__ __forceinline__ int exponent_from_bits(unsigned long long mb) {
  if (mb == 0) return 0;
  const int E = (int)(mb >> 52);
  return (E ? E : 1) - 1022;
}
// Balanced digits of x (|x| < 2^e), computed with integer operations: y = |x| 2^{-e} is
// rounded to 7S fractional bits, split into base-128 digits, and re-centred from the least
// significant end (a digit >= 64 becomes digit - 128 with a carry into the next one), so
// that digits 2..S lie in [-64, 63] and digit 1 in [0, 129]; the sign of x is applied to all.
// Then |x - 2^e sum_k d_k 2^{-7k}| <= 2^{e-7S-1}, and the dropped slice pairs of a product
// carry digits of both signs (they largely cancel).  Every digit is exact in bf16.
__device__ __forceinline__ void digits(double x, int e, int S, __nv_bfloat16* out, int64_t stride) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7FF);
  const bool neg = (bits >> 63) != 0;
  unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (E ? (1ull << 52) : 0ull);
  const int Eu = (E ? E : 1) - 1075;  // x = mant * 2^Eu
  const int sh_last = e - Eu - OZ_BETA * S;
  if (sh_last >= 1 && sh_last <= 63) mant += 1ull << (sh_last - 1);  // round half up (magnitude)
  int d[8];
#pragma unroll
  for (int k = 1; k <= 8; ++k) {
    if (k > S) break;
    const int sh = e - Eu - OZ_BETA * k;  // right shift that leaves digit k in the low bits
    unsigned long long w;
    if (sh >= 64) w = 0ull;
    else if (sh >= 0) w = mant >> sh;
    else w = mant << (-sh);
    d[k - 1] = (k == 1) ? (int)w : (int)(w & 127ull);
  }
#pragma unroll
  for (int k = 8; k >= 2; --k) {
    if (k > S) continue;
    if (d[k - 1] >= 64) {
      d[k - 1] -= 128;
      d[k - 2] += 1;
    }
  }
#pragma unroll
  for (int k = 1; k <= 8; ++k) {
    if (k > S) break;
    const float v = (float)(neg ? -d[k - 1] : d[k - 1]);
    out[(int64_t)(k - 1) * stride] = __float2bfloat16_rn(v);
  }
}

__device__ unsigned long long block_max_bits(unsigned long long v) {
  __shared__ unsigned long long sh[32];
  __shared__ unsigned long long res;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, v, o);
    v = t > v ? t : v;
  }
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    unsigned long long t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long u = __shfl_xor_sync(0xffffffffu, t, o);
      t = u > t ? u : t;
    }
    if (lane == 0) res = t;
  }
  __syncthreads();
  const unsigned long long r = res;
  __syncthreads();
  return r;
}

// A-side slices of the real embedding of Hermitian Hs: one CTA per complex row i.
// Row i of Hs is conj(column i), read contiguously.  Real rows 2i, 2i+1; columns 2k, 2k+1:
//   [ Re h  -Im h ]      h = Hs(i, k) = conj(Hs(k, i))
//   [ Im h   Re h ]
__global__ void oz_slice_hermitian_kernel(const zd* Hs, int64_t ldh, int n, int S,
                                          __nv_bfloat16* A, int64_t sliceA, int Kp, int* eA) {
  // (n = K: the length of column i of X, i.e. of row i of op(A) = X^H)
  const int i = blockIdx.x;
  const zd* col = Hs + (int64_t)i * ldh;
  unsigned long long mx = 0ull;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const zd h = col[k];
    const unsigned long long a = abs_bits(h.x), b = abs_bits(h.y);
    mx = a > mx ? a : mx;
    mx = b > mx ? b : mx;
  }
  mx = block_max_bits(mx);
  const int e = exponent_from_bits(mx);
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


// Slices from the ROWS of a general complex matrix X (rows x cols, column-major), in two
// kernels: the row scales need a full pass over each row, and a row is strided in memory,
// so 32-row groups are read column by column (coalesced) to find the row exponents; the
// digits are then written by CTAs that each take one 32-row group and one range of columns
// (transposed through shared memory), so that thin matrices still spread over the GPU.
//   mode 0 (A operand, real embedding): rows 2r, 2r+1 of A^ = [Re x, -Im x], [Im x, Re x]
//   mode 1 (B operand of X^H): column r of B^ = conj(row r of X) = [Re x, -Im x]
__global__ void oz_row_exponents_kernel(const zd* X, int64_t ldx, int rows, int cols, int* e_out) {
  __shared__ unsigned long long red[8][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int r = blockIdx.x * 32 + tx;
  unsigned long long mx = 0ull;
  if (r < rows)
    for (int k = ty; k < cols; k += 8) {
      const zd v = X[r + (int64_t)k * ldx];
      const unsigned long long a = abs_bits(v.x), b = abs_bits(v.y);
      mx = a > mx ? a : mx;
      mx = b > mx ? b : mx;
    }
  red[ty][tx] = mx;
  __syncthreads();
  if (ty == 0 && r < rows) {
    unsigned long long m2 = red[0][tx];
    for (int j = 1; j < 8; ++j) m2 = red[j][tx] > m2 ? red[j][tx] : m2;
    e_out[r] = exponent_from_bits(m2);
  }
}

__global__ void oz_slice_rows_kernel(const zd* X, int64_t ldx, int rows, int cols, int S, int mode,
                                     __nv_bfloat16* out, int64_t slice_stride, int Kp, const int* e_row,
                                     int chunk) {
  __shared__ int ex[32];
  __shared__ zd tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int r0 = blockIdx.x * 32;
  if (ty == 0) ex[tx] = (r0 + tx < rows) ? e_row[r0 + tx] : 0;
  __syncthreads();
  const int k_end = min(cols, (int)(blockIdx.y + 1) * chunk);
  for (int k0 = blockIdx.y * chunk; k0 < k_end; k0 += 32) {
    for (int rr = ty; rr < 32; rr += 8) {
      const int gr = r0 + tx, gk = k0 + rr;  // read column gk, rows r0..r0+31 (coalesced)
      tile[rr][tx] = (gr < rows && gk < k_end) ? X[gr + (int64_t)gk * ldx] : zmk(0.0, 0.0);
    }
    __syncthreads();
    for (int rr = ty; rr < 32; rr += 8) {  // write row r0 + rr, columns k0 + tx (coalesced)
      const int gr = r0 + rr, gk = k0 + tx;
      if (gr < rows && gk < k_end) {
        const zd v = tile[tx][rr];
        const int e = ex[rr];
        if (mode == 0) {
          __nv_bfloat16* o0 = out + (int64_t)(2 * gr) * Kp + 2 * gk;
          __nv_bfloat16* o1 = o0 + Kp;
          digits(v.x, e, S, o0, slice_stride);
          digits(-v.y, e, S, o0 + 1, slice_stride);
          digits(v.y, e, S, o1, slice_stride);
          digits(v.x, e, S, o1 + 1, slice_stride);
        } else {
          __nv_bfloat16* o0 = out + (int64_t)gr * Kp + 2 * gk;
          digits(v.x, e, S, o0, slice_stride);
          digits(-v.y, e, S, o0 + 1, slice_stride);
        }
      }
    }
    __syncthreads();
  }
}

// B-side slices of Y^ (the n x m complex block read as a 2n x m real array): one CTA per
// column j; columns j >= m of the padded block are zero.
// lower_half: column j of the operand is column j of Y below the diagonal, half of Y(j, j)
// on it and zero above (the lower part L_h of a Hermitian Y = L_h + L_h^H).
__global__ void oz_slice_cols_kernel(const zd* Y, int64_t ldy, int n, int m, int S,
                                     __nv_bfloat16* B, int64_t sliceB, int Kp, int* eB, int lower_half) {
  const int j = blockIdx.x;
  __nv_bfloat16* col = B + (int64_t)j * Kp;
  if (j >= m) {
    for (int k = threadIdx.x; k < Kp; k += blockDim.x)
      for (int s = 0; s < S; ++s) col[s * sliceB + k] = __float2bfloat16_rn(0.f);
    if (threadIdx.x == 0) eB[j] = 0;
    return;
  }
  const zd* y = Y + (int64_t)j * ldy;
  auto entry = [&](int k) -> zd {
    zd v = y[k];
    if (lower_half) {
      if (k < j) v = zmk(0.0, 0.0);
      else if (k == j) v = zmk(0.5 * v.x, 0.5 * v.y);
    }
    return v;
  };
  unsigned long long mx = 0ull;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const zd v = entry(k);
    const unsigned long long a = abs_bits(v.x), b = abs_bits(v.y);
    mx = a > mx ? a : mx;
    mx = b > mx ? b : mx;
  }
  mx = block_max_bits(mx);
  const int e = exponent_from_bits(mx);
  if (threadIdx.x == 0) eB[j] = e;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const zd v = entry(k);
    digits(v.x, e, S, col + 2 * k, sliceB);
    digits(v.y, e, S, col + 2 * k + 1, sliceB);
  }
}

// Gauss form of the complex product (three real products instead of the 2n x 2n real
// embedding): Hs Y = (Hr Yr - Hi Yi) + i ((Hr + Hi)(Yr + Yi) - Hr Yr - Hi Yi).  Operand z of
// A is Hr, Hi, Hr + Hi (z = 0, 1, 2) with its own power-of-two scale per row, operand z of B
// is Yr, Yi, Yr + Yi with its own scale per column; slices [z][s][row][k], scales [z][row].
// The sums Hr + Hi and Yr + Yi are formed in FP64 (one rounding) before the digits are taken.
// Rows of A: row i of H = conj(column i of Hs) (Hs Hermitian), read contiguously.
__global__ void oz_slice_hermitian3_kernel(const zd* Hs, int64_t ldh, int n, int S, __nv_bfloat16* A,
                                           int64_t sliceA, int64_t zstride, int Kp, int Mp, int* eA) {
  const int i = blockIdx.x;
  const zd* col = Hs + (int64_t)i * ldh;
  unsigned long long m0 = 0ull, m1 = 0ull, m2 = 0ull;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const zd h = col[k];
    const double hr = h.x, hi = -h.y, hs = hr + hi;
    const unsigned long long a = abs_bits(hr), b = abs_bits(hi), c = abs_bits(hs);
    m0 = a > m0 ? a : m0;
    m1 = b > m1 ? b : m1;
    m2 = c > m2 ? c : m2;
  }
  const int e0 = exponent_from_bits(block_max_bits(m0));
  const int e1 = exponent_from_bits(block_max_bits(m1));
  const int e2 = exponent_from_bits(block_max_bits(m2));
  if (threadIdx.x == 0) {
    eA[i] = e0;
    eA[Mp + i] = e1;
    eA[2 * Mp + i] = e2;
  }
  __nv_bfloat16* r0 = A + (int64_t)i * Kp;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const zd h = col[k];
    const double hr = h.x, hi = -h.y;
    digits(hr, e0, S, r0 + k, sliceA);
    digits(hi, e1, S, r0 + zstride + k, sliceA);
    digits(hr + hi, e2, S, r0 + 2 * zstride + k, sliceA);
  }
}

// Columns of B in the Gauss form: column j of Y gives rows j of Yr, Yi, Yr + Yi; columns
// j >= m of the padded block are zero (the buffer is cleared first).
__global__ void oz_slice_cols3_kernel(const zd* Y, int64_t ldy, int n, int m, int S, __nv_bfloat16* B,
                                      int64_t sliceB, int64_t zstride, int Kp, int Np, int* eB,
                                      int lower_half) {
  const int j = blockIdx.x;
  if (j >= m) {
    if (threadIdx.x == 0) eB[j] = eB[Np + j] = eB[2 * Np + j] = 0;
    return;
  }
  const zd* y = Y + (int64_t)j * ldy;
  // lower_half: as oz_slice_cols_kernel (zero above the diagonal, half of the diagonal entry)
  auto entry = [&](int k) -> zd {
    zd v = y[k];
    if (lower_half) {
      if (k < j) v = zmk(0.0, 0.0);
      else if (k == j) v = zmk(0.5 * v.x, 0.5 * v.y);
    }
    return v;
  };
  unsigned long long m0 = 0ull, m1 = 0ull, m2 = 0ull;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const zd v = entry(k);
    const unsigned long long a = abs_bits(v.x), b = abs_bits(v.y), c = abs_bits(v.x + v.y);
    m0 = a > m0 ? a : m0;
    m1 = b > m1 ? b : m1;
    m2 = c > m2 ? c : m2;
  }
  const int e0 = exponent_from_bits(block_max_bits(m0));
  const int e1 = exponent_from_bits(block_max_bits(m1));
  const int e2 = exponent_from_bits(block_max_bits(m2));
  if (threadIdx.x == 0) {
    eB[j] = e0;
    eB[Np + j] = e1;
    eB[2 * Np + j] = e2;
  }
  __nv_bfloat16* c0 = B + (int64_t)j * Kp;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const zd v = entry(k);
    digits(v.x, e0, S, c0 + k, sliceB);
    digits(v.y, e1, S, c0 + zstride + k, sliceB);
    digits(v.x + v.y, e2, S, c0 + 2 * zstride + k, sliceB);
  }
}

// Gauss-form slices from the ROWS of X (rows x cols, column-major): row r of the operand is
// row r of X (conj = 0: an A operand) or its conjugate (conj = 1: column r of a B operand
// op(B) = X^H); the three parts re, im, re + im get a scale per row each (e[z * e_stride + r])
// and their digits go to out + z * zstride + r * Kp + k.  Same two-kernel scheme as the
// embedding's row slices.
__global__ void oz_row_exponents3_kernel(const zd* X, int64_t ldx, int rows, int cols, int conj, int* e_out,
                                         int e_stride) {
  __shared__ unsigned long long red[3][8][32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int r = blockIdx.x * 32 + tx;
  unsigned long long m0 = 0ull, m1 = 0ull, m2 = 0ull;
  if (r < rows)
    for (int k = ty; k < cols; k += 8) {
      const zd v = X[r + (int64_t)k * ldx];
      const double re = v.x, im = conj ? -v.y : v.y;
      const unsigned long long a = abs_bits(re), b = abs_bits(im), c = abs_bits(re + im);
      m0 = a > m0 ? a : m0;
      m1 = b > m1 ? b : m1;
      m2 = c > m2 ? c : m2;
    }
  red[0][ty][tx] = m0;
  red[1][ty][tx] = m1;
  red[2][ty][tx] = m2;
  __syncthreads();
  if (ty < 3 && r < rows) {
    unsigned long long mz = red[ty][0][tx];
    for (int j = 1; j < 8; ++j) mz = red[ty][j][tx] > mz ? red[ty][j][tx] : mz;
    e_out[ty * e_stride + r] = exponent_from_bits(mz);
  }
}

__global__ void oz_slice_rows3_kernel(const zd* X, int64_t ldx, int rows, int cols, int S, int conj,
                                      __nv_bfloat16* out, int64_t slice_stride, int64_t zstride, int Kp,
                                      const int* e_row, int e_stride, int chunk) {
  __shared__ int ex[3][32];
  __shared__ zd tile[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const int r0 = blockIdx.x * 32;
  if (ty < 3) ex[ty][tx] = (r0 + tx < rows) ? e_row[ty * e_stride + r0 + tx] : 0;
  __syncthreads();
  const int k_end = min(cols, (int)(blockIdx.y + 1) * chunk);
  for (int k0 = blockIdx.y * chunk; k0 < k_end; k0 += 32) {
    for (int rr = ty; rr < 32; rr += 8) {
      const int gr = r0 + tx, gk = k0 + rr;  // read column gk, rows r0..r0+31 (coalesced)
      tile[rr][tx] = (gr < rows && gk < k_end) ? X[gr + (int64_t)gk * ldx] : zmk(0.0, 0.0);
    }
    __syncthreads();
    for (int rr = ty; rr < 32; rr += 8) {  // write row r0 + rr, columns k0 + tx (coalesced)
      const int gr = r0 + rr, gk = k0 + tx;
      if (gr < rows && gk < k_end) {
        const zd v = tile[tx][rr];
        const double re = v.x, im = conj ? -v.y : v.y;
        __nv_bfloat16* o = out + (int64_t)gr * Kp + gk;
        digits(re, ex[0][rr], S, o, slice_stride);
        digits(im, ex[1][rr], S, o + zstride, slice_stride);
        digits(re + im, ex[2][rr], S, o + 2 * zstride, slice_stride);
      }
    }
    __syncthreads();
  }
}

// out = alpha (P0 - P1 + i (P2 - P0 - P1)) + beta Cin + gamma D from the split partials of
// the three real products (double-float pairs, slice scales applied), each scaled by its row
// and column exponents.
__global__ void oz_epilogue3_kernel(const float2* part, int splits, int Mp, int Np, const int* eA,
                                    const int* eB, int n, int m, double alpha, double beta,
                                    const zd* Cin, int64_t ldcin, double gamma, const zd* D,
                                    int64_t ldd, zd* out, int64_t ldo, int lower) {
  const int64_t total = (int64_t)n * m;
  const int64_t zst = (int64_t)splits * Mp * Np;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (lower && j > i) continue;
    double v[3];
#pragma unroll
    for (int z = 0; z < 3; ++z) {
      float h = 0.f, l = 0.f;
      for (int sp = 0; sp < splits; ++sp) {
        const float2 q = part[z * zst + (int64_t)sp * Mp * Np + (int64_t)j * Mp + i];
        two_sum_acc(h, l, q.x);
        l += q.y;
      }
      v[z] = ldexp((double)h + (double)l, eA[z * Mp + i] + eB[z * Np + j]);
    }
    zd o = zmk(alpha * (v[0] - v[1]), alpha * (v[2] - v[0] - v[1]));
    if (beta != 0.0) o = zadd(o, zscale(Cin[i + (int64_t)j * ldcin], beta));
    if (gamma != 0.0) o = zadd(o, zscale(D[i + (int64_t)j * ldd], gamma));
    out[i + (int64_t)j * ldo] = o;
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

// Split count for the tcgen05 kernel: split y takes k-blocks [y per, (y + 1) per) of every
// tile, or (short K) a range of slice pairs.  Modelled CTA time in k-block units: every
// (panel, pair) chunk costs at least the drain of one accumulator (about 3 k-blocks of
// streaming time), plus a pipeline fill; the launch time is that times the number of waves
// of one CTA per SM.
int choose_tc_splits(int tiles, int nkb, int npairs, size_t cap_elems, int64_t tile_elems, int* pair_split) {
  const int sms = sm_count();
  int best = 1;
  double best_cost = 1e300;
  *pair_split = 0;
  for (int S = 1; S <= std::min(nkb, 64); ++S) {
    if ((size_t)S * (size_t)tile_elems > cap_elems) break;
    const int per = (nkb + S - 1) / S;
    double cta = 6.0;
    for (int k0 = 0; k0 < per; k0 += OZ_CHUNK_KB)
      cta += (double)npairs * std::max(3, std::min(OZ_CHUNK_KB, per - k0));
    const int64_t units = (int64_t)tiles * S;
    const double cost = (double)((units + sms - 1) / sms) * cta;
    if (cost < best_cost * 0.999) { best_cost = cost; best = S; }
  }
  // short K (a single panel): splitting the slice pairs gives more CTAs than splitting K
  if (nkb <= OZ_CHUNK_KB) {
    for (int S = 2; S <= npairs; ++S) {
      if ((size_t)S * (size_t)tile_elems > cap_elems) break;
      const int pp = (npairs + S - 1) / S;
      const double cta = 6.0 + (double)pp * std::max(3, nkb);
      const int64_t units = (int64_t)tiles * ((npairs + pp - 1) / pp);
      const double cost = (double)((units + sms - 1) / sms) * cta;
      if (cost < best_cost * 0.999) { best_cost = cost; best = (npairs + pp - 1) / pp; *pair_split = 1; }
    }
  }
  return best;
}

}  // namespace

// ---------------------------------------------------------------------------- host side
// Autotuner of the tcgen05 kernel's split count: the best configuration measured for each
// product shape, shared by all contexts of the process (batch workers tune from several host
// threads).  Environment variable CHFSI_OZ_AUTOTUNE=0 keeps the wave model's choice.
struct TuneKey {
  int Mp, Np, Kp, S, a_lower, c_lower, group, b_box_rows, cl, ngroups, b_tri, nz;
  bool operator<(const TuneKey& o) const {
    const int a[12] = {Mp, Np, Kp, S, a_lower, c_lower, group, b_box_rows, cl, ngroups, b_tri, nz};
    const int b[12] = {o.Mp, o.Np, o.Kp, o.S, o.a_lower, o.c_lower, o.group, o.b_box_rows, o.cl, o.ngroups,
                       o.b_tri, o.nz};
    return std::lexicographical_compare(a, a + 12, b, b + 12);
  }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, std::pair<int, int>> g_tune;
static bool tune_lookup(const TuneKey& k, int* splits, int* pair_split) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(k);
  if (it == g_tune.end()) return false;
  *splits = it->second.first;
  *pair_split = it->second.second;
  return true;
}
static void tune_store(const TuneKey& k, int splits, int pair_split) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[k] = {splits, pair_split};
}
static bool oz_autotune() {
  static const bool v = [] {
    const char* e = std::getenv("CHFSI_OZ_AUTOTUNE");
    return !(e && std::strcmp(e, "0") == 0);
  }();
  return v;
}
int oz_tuned_shapes() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return (int)g_tune.size();
}
// Product kernel: tcgen05 (default) or the mma.sync kernel, chosen once per process by the
// environment variable CHFSI_OZ_KERNEL ("tc" or "mma").
// The choices below are read once (thread-safe static initialisation: batch workers call
// the product from several host threads).
bool oz_use_tcgen05() {
  static const bool tc = [] {
    const char* v = std::getenv("CHFSI_OZ_KERNEL");
    return !(v && std::strcmp(v, "mma") == 0);
  }();
  return tc;
}
// Slice groups sharing one A tile per stage (tcgen05 kernel, blocks up to 96 columns wide);
// CHFSI_OZ_GROUPS=0 issues one pair per stage instead.
static bool oz_grouped_pairs() {
  static const bool grouped = [] {
    const char* v = std::getenv("CHFSI_OZ_GROUPS");
    return !(v && std::strcmp(v, "0") == 0);
  }();
  return grouped;
}
// Largest cluster of CTAs sharing the B tiles of the tcgen05 kernel by multicast: environment
// variable CHFSI_OZ_CLUSTER (1, 2 or 4; default 1: measured slower on the n = 9300 workload,
// whose launches are bound by the bytes in flight per SM rather than by the L2 stream).
static int oz_cluster_max() {
  static const int v = [] {
    const char* e = std::getenv("CHFSI_OZ_CLUSTER");
    const int c = e ? std::atoi(e) : 1;
    return c >= 4 ? 4 : (c >= 2 ? 2 : 1);
  }();
  return v;
}
// Order of the tiles over blockIdx.x: environment variable CHFSI_OZ_ORDER ("col": the column
// tiles of a row tile next to each other; default "row").
static bool oz_col_major_order() {
  static const bool v = [] {
    const char* e = std::getenv("CHFSI_OZ_ORDER");
    return e && std::strcmp(e, "col") == 0;
  }();
  return v;
}
// Smallest TMA ring a slice group may leave (its B box grows with the group): environment
// variable CHFSI_OZ_GROUP_MIN_STAGES, default 4, clamped to [2, TC_MAX_STAGES].
static int oz_group_min_stages() {
  static const int v = [] {
    const char* e = std::getenv("CHFSI_OZ_GROUP_MIN_STAGES");
    return e ? std::max(2, std::min(TC_MAX_STAGES, std::atoi(e))) : 4;
  }();
  return v;
}

// 2-D bf16 tensor map over `rows` rows of `inner` elements (row pitch inner * 2 bytes),
// boxes of 64 elements x box_rows rows, 128-byte swizzle (the layout the tcgen05
// descriptors expect).
static bool encode_bf16_map(CUtensorMap* map, const void* ptr, int inner, uint64_t rows, int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!encode) return false;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)inner * 2};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides,
                            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}
int oz_padded_k(int n) { return ((2 * n + OZ_BK - 1) / OZ_BK) * OZ_BK; }
int oz_padded_m(int n) { return ((2 * n + OZ_BM - 1) / OZ_BM) * OZ_BM; }
int oz_padded_n(int m) {
  // tcgen05: multiples of 32 columns, so that a B box splits into four 8-row-aligned shares
  return oz_use_tcgen05() ? ((m + 31) / 32) * 32 : ((m + OZ_BN - 1) / OZ_BN) * OZ_BN;
}

// ---- operands
// Row exponents, then digits by (32-row group, column range) CTAs: about four CTAs per SM.
static cudaError_t slice_rows(const zd* X, int64_t ldx, int rows, int cols, int S, int mode, __nv_bfloat16* out,
                              int64_t slice_stride, int Kp, int* e_out, cudaStream_t s) {
  const int groups = (rows + 31) / 32, kchunks = (cols + 31) / 32;
  oz_row_exponents_kernel<<<groups, 256, 0, s>>>(X, ldx, rows, cols, e_out);
  CHFSI_COUNT_LAUNCH();
  const int gy = std::max(1, std::min(kchunks, (4 * sm_count() + groups - 1) / groups));
  const int chunk = 32 * ((kchunks + gy - 1) / gy);
  oz_slice_rows_kernel<<<dim3(groups, (cols + chunk - 1) / chunk), 256, 0, s>>>(X, ldx, rows, cols, S, mode, out,
                                                                                slice_stride, Kp, e_out, chunk);
  return cudaGetLastError();
}
#define CK_OZ(expr)                 \
  do {                              \
    cudaError_t e_ = (expr);        \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

cudaError_t oz_slice_a(OzA& a, int op, const zd* X, int64_t ldx, int M, int K, int S, cudaStream_t s) {
  const int Kp = oz_padded_k(K), Mp = oz_padded_m(M);
  if (S > a.S_max || S < 1 || Kp > a.Kp_max || Mp > a.Mp_max || M <= 0 || K <= 0)
    return cudaErrorInvalidValue;
  a.S = S; a.M = M; a.K = K; a.Mp = Mp; a.Kp = Kp; a.nz = 1;
  a.slice = (int64_t)Mp * Kp;
  // zero the padding (rows >= 2M, columns >= 2K)
  cudaError_t e = cudaMemsetAsync(a.ptr, 0, sizeof(__nv_bfloat16) * (size_t)S * a.slice, s);
  if (e != cudaSuccess) return e;
  if (op == OPC) {
    // op(A) = X^H: row i of op(A) is conj(column i of X), contiguous (X is K x M)
    oz_slice_hermitian_kernel<<<M, 256, 0, s>>>(X, ldx, K, S, a.ptr, a.slice, Kp, a.e);
  } else {
    CK_OZ(slice_rows(X, ldx, M, K, S, 0, a.ptr, a.slice, Kp, a.e, s));
  }
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}

cudaError_t oz_slice_b(OzB& b, int op, const zd* X, int64_t ldx, int K, int N, int S, int Kp,
                       cudaStream_t s, int lower_half) {
  const int Np = oz_padded_n(N);
  if (Np > b.Np_max || Kp > b.Kp_max || S > b.S_max || S < 1 || N <= 0) return cudaErrorInvalidValue;
  b.S = S; b.N = N; b.Np = Np; b.Kp = Kp; b.nz = 1;
  b.slice = (int64_t)Np * Kp;
  cudaError_t e = cudaMemsetAsync(b.ptr, 0, sizeof(__nv_bfloat16) * (size_t)S * b.slice, s);
  if (e != cudaSuccess) return e;
  if (op == OPC) {
    // op(B) = X^H (X is N x K): column j = conj(row j of X)
    CK_OZ(slice_rows(X, ldx, N, K, S, 1, b.ptr, b.slice, Kp, b.e, s));
  } else {
    oz_slice_cols_kernel<<<Np, 256, 0, s>>>(X, ldx, K, N, S, b.ptr, b.slice, Kp, b.e, lower_half);
  }
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}

// out (M x N complex, M = a.M, N = b.N) = alpha op(A) op(B) + beta Cin + gamma D from the
// operands' slices, with the slice pairs (s, t), s + t <= S + 1.  a_lower: op(A) is lower
// triangular (zero k-blocks skipped); c_lower: only the lower triangle of out is written.
cudaError_t oz_product(const OzA& a, const OzB& b, int S, double alpha, double beta, const zd* Cin,
                       int64_t ldcin, double gamma, const zd* D, int64_t ldd, zd* out, int64_t ldo,
                       int a_lower, int c_lower, OzWorkspace& oz, cudaStream_t s,
                       cudaEvent_t ev_gemm_begin, cudaEvent_t ev_gemm_end, int b_tri) {
  const int n = a.M, m = b.N, Kp = a.Kp, Mp = a.Mp, Np = b.Np;
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (S > b.S || S > a.S || S < 1 || a.Kp != b.Kp || a.nz != b.nz) return cudaErrorInvalidValue;
  const int nz = a.nz;  // 3: Gauss form (tcgen05 path only)
  if (nz != 1 && (nz != 3 || !oz_use_tcgen05())) return cudaErrorInvalidValue;
  cudaError_t e;
  // Pairs (s, t) with s + t <= S + 1, grouped by the A slice s so that consecutive pairs
  // stream the same slice of the large operand (it stays in L2 between them).
  OzPairs pairs;
  pairs.n = 0;
  for (int si = 1; si <= S; ++si)
    for (int ti = 1; si + ti <= S + 1; ++ti) {
      pairs.s[pairs.n] = (unsigned char)(si - 1);
      pairs.t[pairs.n] = (unsigned char)(ti - 1);
      ++pairs.n;
    }
  int splits = 1;
  if (oz_use_tcgen05()) {
    TcParams tp;
    tp.a_lower = a_lower;
    tp.b_tri = b_tri;
    tp.c_lower = c_lower;
    tp.nkb = Kp / OZ_BK;
    tp.tiles_m = Mp / TC_BM;
    tp.Mp = Mp;
    tp.Np = Np;
    tp.n_real = m;
    tp.part = oz.part;
    tp.status = oz.status;
    tp.nz = nz;
    tp.kfac = nz > 1 ? 1 : 2;
    tp.a_zrows = nz > 1 ? a.S * Mp : 0;
    tp.b_zrows = nz > 1 ? b.S * Np : 0;
    // first-level waits: the context's bound (a test hook) or the default; the waits that
    // let issued copies and MMAs finish after an abort always use the default
    tp.spin_limit = oz.wait_limit > 0 ? oz.wait_limit : kMbarSpinLimit;
    // group size (see the kernel's header): tensor memory holds 2 g accumulators of the
    // block's width rounded up to 32 columns plus the high words, the B box is at most 256
    // rows, and the ring keeps at least oz_group_min_stages() stages
    int G = 1;
    tp.acc_stride = TC_ACC1;
    if (Np <= TC_GROUP_MAX_N && oz_grouped_pairs()) {
      const int w = ((Np + 31) / 32) * 32;
      G = std::min({S, TC_GROUP_MAX, (512 / w - 1) / 2, 256 / Np});
      while (G > 1 && TC_SMEM_BUDGET / (TC_A_BYTES + G * Np * TC_BK * 2) < oz_group_min_stages()) --G;
      if (G > 1) tp.acc_stride = w;
    }
    tp.group = G;
    tp.ngroups = 0;
    for (int si = 1; si <= S; ++si)
      for (int t0 = 1; si + t0 <= S + 1; t0 += G) {
        tp.gs[tp.ngroups] = (unsigned char)(si - 1);
        tp.gt[tp.ngroups] = (unsigned char)(t0 - 1);
        tp.gc[tp.ngroups] = (unsigned char)std::min(G, S + 2 - si - t0);
        ++tp.ngroups;
      }
    CUtensorMap mapA, mapB;
    // The B box is min(Np, TC_BN) rows high (g Np for groups of g); a last tile or group
    // narrower than that reads rows past its slices (the next slice, the buffer's spare rows:
    // the allocation holds at least TC_BN rows, or the fill past the map's last row) that
    // the MMAs never use, since their N covers only the tile's own columns.
    tp.b_box_rows = G > 1 ? G * Np : std::min(Np, TC_BN);
    // Cluster of cl CTAs on consecutive row tiles sharing each B box (each loads b_box_rows /
    // cl rows, a multiple of 8 so that every share starts on a 1024-byte swizzle atom); the
    // single-CTA launch when the context shortens its waits (the timeout test exercises that
    // launch's unwinding) or the grid has too few row tiles.
    tp.cl = 1;
    if (oz.wait_limit == 0 && oz_cluster_max() > 1)
      for (int c = oz_cluster_max(); c >= 2; c /= 2)
        if (tp.tiles_m >= 2 * c && tp.b_box_rows % (8 * c) == 0) {
          tp.cl = c;
          break;
        }
    tp.tiles_m_pad = ((tp.tiles_m + tp.cl - 1) / tp.cl) * tp.cl;
    tp.col_major_order = (tp.cl == 1 && oz_col_major_order()) ? 1 : 0;
    const int tiles = tp.tiles_m_pad * ((Np + TC_BN - 1) / TC_BN);
    int model_pair_split = 0;
    const size_t part_cap = oz.part_elems / (size_t)nz;  // partials of each of the nz products
    const int model_splits =
        choose_tc_splits(tiles, tp.nkb, tp.ngroups, part_cap, (int64_t)Mp * Np, &model_pair_split);
    const uint64_t b_rows = std::max<uint64_t>((uint64_t)nz * b.S * Np, (uint64_t)TC_BN);
    if ((int64_t)b_rows * Kp > b.elems) return cudaErrorInvalidValue;
    if (!encode_bf16_map(&mapA, a.ptr, Kp, (uint64_t)nz * a.S * Mp, TC_BM) ||
        !encode_bf16_map(&mapB, b.ptr, Kp, b_rows, tp.b_box_rows / tp.cl))
      return cudaErrorInvalidValue;
    const int b_stage = tp.b_box_rows * TC_BK * 2;
    tp.stages = std::min(TC_MAX_STAGES, TC_SMEM_BUDGET / (TC_A_BYTES + b_stage));
    const size_t smem = 1024 + (size_t)tp.stages * (TC_A_BYTES + b_stage) + 256;
    // once per process (the library drives one device per process)
    static const cudaError_t tc_attr = cudaFuncSetAttribute(
        oz_gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 1024 + TC_SMEM_BUDGET + 256);
    if (tc_attr != cudaSuccess) return tc_attr;
    auto launch = [&](int sp, int ps) -> cudaError_t {
      tp.splits = sp;
      tp.pair_split = ps;
      if (tp.cl > 1) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(tiles, sp, nz);
        cfg.blockDim = dim3(TC_THREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = tp.cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t le = cudaLaunchKernelEx(&cfg, oz_gemm_tc_kernel, mapA, mapB, tp);
        if (le != cudaSuccess) return le;
      } else {
        oz_gemm_tc_kernel<<<dim3(tiles, sp, nz), TC_THREADS, smem, s>>>(mapA, mapB, tp);
      }
      CHFSI_COUNT_LAUNCH();
      return cudaGetLastError();
    };
    // split count: the wave model's choice, or the fastest of a few candidates around it,
    // measured on the first product of each shape and kept for the process (autotuner)
    int best_splits = model_splits, best_ps = model_pair_split;
    const TuneKey key{Mp, Np, Kp, S, a_lower, c_lower, tp.group, tp.b_box_rows, tp.cl, tp.ngroups, b_tri, nz};
    if (oz_autotune() && !tune_lookup(key, &best_splits, &best_ps)) {
      cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(s, &cap) == cudaSuccess && cap == cudaStreamCaptureStatusNone) {
        std::vector<std::pair<int, int>> cand;
        const int limit_k = model_pair_split ? tp.ngroups : std::min(tp.nkb, 64);
        for (int num : {2, 3, 4, 6, 8}) {  // model x {1/2, 3/4, 1, 3/2, 2}
          const int sp = std::max(1, std::min(limit_k, (model_splits * num + 2) / 4));
          if ((size_t)sp * (size_t)((int64_t)Mp * Np) > part_cap) continue;
          if (model_pair_split) {
            const int pp = (tp.ngroups + sp - 1) / sp;   // groups per split: the grid uses ceil
            const int eff = (tp.ngroups + pp - 1) / pp;
            if (std::find(cand.begin(), cand.end(), std::make_pair(eff, 1)) == cand.end()) cand.push_back({eff, 1});
          } else if (std::find(cand.begin(), cand.end(), std::make_pair(sp, 0)) == cand.end()) {
            cand.push_back({sp, 0});
          }
        }
        cudaEvent_t t0, t1;
        if (cudaEventCreate(&t0) != cudaSuccess || cudaEventCreate(&t1) != cudaSuccess) return cudaGetLastError();
        float best_ms = 1e30f;
        for (const auto& c : cand) {
          cudaEventRecord(t0, s);
          e = launch(c.first, c.second);
          if (e != cudaSuccess) break;
          cudaEventRecord(t1, s);
          e = cudaEventSynchronize(t1);
          if (e != cudaSuccess) break;
          float ms = 0.f;
          cudaEventElapsedTime(&ms, t0, t1);
          if (ms < best_ms) { best_ms = ms; best_splits = c.first; best_ps = c.second; }
        }
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        if (e != cudaSuccess) return e;
        tune_store(key, best_splits, best_ps);
      }
    }
    splits = best_splits;
    if ((size_t)splits * (size_t)nz * (size_t)Mp * (size_t)Np > oz.part_elems) return cudaErrorInvalidValue;
    if (ev_gemm_begin) cudaEventRecord(ev_gemm_begin, s);
    e = launch(best_splits, best_ps);
    if (ev_gemm_end) cudaEventRecord(ev_gemm_end, s);
    if (e != cudaSuccess) return e;
  } else {
    OzParams p;
    p.a_lower = a_lower;
    p.c_lower = c_lower;
    p.A = a.ptr;
    p.B = b.ptr;
    p.sliceA = a.slice;
    p.sliceB = b.slice;
    p.Kp = Kp;
    p.nkb = Kp / OZ_BK;
    p.tiles_m = Mp / OZ_BM;
    p.Mp = Mp;
    p.Np = Np;
    p.pairs = pairs;
    const int tiles = p.tiles_m * (Np / OZ_BN);
    p.splits = splits = choose_oz_splits(tiles, p.pairs.n * p.nkb, oz.part_elems, (int64_t)Mp * Np);
    p.part = oz.part;
    const size_t smem = (size_t)OZ_STAGES * (OZ_BM + OZ_BN) * OZ_BK * 2;
    static const cudaError_t mma_attr =
        cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (mma_attr != cudaSuccess) return mma_attr;
    if (ev_gemm_begin) cudaEventRecord(ev_gemm_begin, s);
    oz_gemm_kernel<<<dim3(tiles, p.splits), OZ_THREADS, smem, s>>>(p);
    CHFSI_COUNT_LAUNCH();
    if (ev_gemm_end) cudaEventRecord(ev_gemm_end, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int64_t tot = (int64_t)n * m;
  const int blocks = (int)std::min<int64_t>(4 * sm_count(), (tot + 255) / 256);
  if (nz == 3)
    oz_epilogue3_kernel<<<blocks, 256, 0, s>>>(reinterpret_cast<const float2*>(oz.part), splits, Mp, Np, a.e,
                                               b.e, n, m, alpha, beta, Cin, ldcin, gamma, D, ldd, out, ldo,
                                               c_lower);
  else
    oz_epilogue_kernel<<<blocks, 256, 0, s>>>(oz.part, splits, Mp, Np, a.e, b.e, n, m, alpha, beta, Cin,
                                              ldcin, gamma, D, ldd, out, ldo, c_lower,
                                              oz_use_tcgen05() ? 1 : 0);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}

// Gauss form of the complex products (three real products, see the slicing kernels above):
// with the tcgen05 kernel, when the workspace allows it (the solver allows it for a
// well-conditioned B), unless environment variable CHFSI_OZ_GAUSS=0 keeps the embedding.
static bool oz_gauss(const OzWorkspace& oz) {
  static const bool v = [] {
    const char* e = std::getenv("CHFSI_OZ_GAUSS");
    return !(e && std::atoi(e) == 0);
  }();
  return v && oz.gauss && oz_use_tcgen05();
}

// op(A) (M x K) as the Gauss-form A operand: slices of its real part, imaginary part and
// their sum, a scale per row of each.  op = OPC: row i is the conjugated column i of X (K x M,
// contiguous); op = OPN: row i of X (M x K, strided; row slices as the embedding's).
static cudaError_t oz_slice_a3(OzA& a, int op, const zd* X, int64_t ldx, int M, int K, int S, cudaStream_t s) {
  const int Mp = ((M + TC_BM - 1) / TC_BM) * TC_BM, Kp = ((K + OZ_BK - 1) / OZ_BK) * OZ_BK;
  if (S > a.S_max || S < 1 || M <= 0 || K <= 0 || Mp > a.Mp_max ||
      (int64_t)3 * S * Mp * Kp > (int64_t)a.S_max * a.Mp_max * a.Kp_max)
    return cudaErrorInvalidValue;
  a.S = S; a.M = M; a.K = K; a.Mp = Mp; a.Kp = Kp; a.nz = 3;
  a.slice = (int64_t)Mp * Kp;
  const int64_t zstride = (int64_t)S * a.slice;
  cudaError_t e = cudaMemsetAsync(a.ptr, 0, sizeof(__nv_bfloat16) * (size_t)3 * zstride, s);
  if (e != cudaSuccess) return e;
  if (op == OPC) {
    oz_slice_hermitian3_kernel<<<M, 256, 0, s>>>(X, ldx, K, S, a.ptr, a.slice, zstride, Kp, Mp, a.e);
    CHFSI_COUNT_LAUNCH();
    return cudaGetLastError();
  }
  const int groups = (M + 31) / 32, kchunks = (K + 31) / 32;
  oz_row_exponents3_kernel<<<groups, 256, 0, s>>>(X, ldx, M, K, 0, a.e, Mp);
  CHFSI_COUNT_LAUNCH();
  const int gy = std::max(1, std::min(kchunks, (4 * sm_count() + groups - 1) / groups));
  const int chunk = 32 * ((kchunks + gy - 1) / gy);
  oz_slice_rows3_kernel<<<dim3(groups, (K + chunk - 1) / chunk), 256, 0, s>>>(
      X, ldx, M, K, S, 0, a.ptr, a.slice, zstride, Kp, a.e, Mp, chunk);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}

// op(B) (K x N) as the Gauss-form B operand, K-padding as the A operand's: op = OPN: column j
// of X (optionally its lower half, as oz_slice_cols_kernel); op = OPC: the conjugated row j of
// X (N x K).
static cudaError_t oz_slice_b3(OzB& b, int op, const zd* X, int64_t ldx, int K, int N, int S, int Kp,
                               cudaStream_t s, int lower_half) {
  const int Np = oz_padded_n(N);
  if (S > b.S_max || S < 1 || N <= 0 || K <= 0 || Np > b.Np_max ||
      (int64_t)3 * S * std::max(Np, TC_BN) * Kp > b.elems)
    return cudaErrorInvalidValue;
  b.S = S; b.N = N; b.Np = Np; b.Kp = Kp; b.nz = 3;
  b.slice = (int64_t)Np * Kp;
  const int64_t zstride = (int64_t)S * b.slice;
  cudaError_t e = cudaMemsetAsync(b.ptr, 0, sizeof(__nv_bfloat16) * (size_t)3 * zstride, s);
  if (e != cudaSuccess) return e;
  if (op == OPC) {
    const int groups = (N + 31) / 32, kchunks = (K + 31) / 32;
    oz_row_exponents3_kernel<<<groups, 256, 0, s>>>(X, ldx, N, K, 1, b.e, Np);
    CHFSI_COUNT_LAUNCH();
    const int gy = std::max(1, std::min(kchunks, (4 * sm_count() + groups - 1) / groups));
    const int chunk = 32 * ((kchunks + gy - 1) / gy);
    oz_slice_rows3_kernel<<<dim3(groups, (K + chunk - 1) / chunk), 256, 0, s>>>(
        X, ldx, N, K, S, 1, b.ptr, b.slice, zstride, Kp, b.e, Np, chunk);
    CHFSI_COUNT_LAUNCH();
    // exponents of the padded columns j >= N
    if (Np > N) {
      e = cudaMemsetAsync(b.e + N, 0, sizeof(int) * (size_t)(Np - N), s);
      if (e == cudaSuccess) e = cudaMemsetAsync(b.e + Np + N, 0, sizeof(int) * (size_t)(Np - N), s);
      if (e == cudaSuccess) e = cudaMemsetAsync(b.e + 2 * Np + N, 0, sizeof(int) * (size_t)(Np - N), s);
      if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
  }
  oz_slice_cols3_kernel<<<Np, 256, 0, s>>>(X, ldx, K, N, S, b.ptr, b.slice, zstride, Kp, Np, b.e, lower_half);
  CHFSI_COUNT_LAUNCH();
  return cudaGetLastError();
}

// ---- the Hermitian matrix of the filter (its slices stay in oz.H for the whole problem)
cudaError_t oz_slice_hermitian(const zd* Hs, int64_t ldh, int n, int S, OzWorkspace& oz,
                               cudaStream_t s) {
  if (oz_gauss(oz)) return oz_slice_a3(oz.H, OPC, Hs, ldh, n, n, S, s);
  return oz_slice_a(oz.H, OPC, Hs, ldh, n, n, S, s);
}

// out(n x m) = alpha Hs Y + beta Cin + gamma D with Hs given by its slices in oz.H and Y
// sliced here into S slices.
cudaError_t oz_filter_product(const zd* Y, int64_t ldy, int n, int m, int S, double alpha,
                              double beta, const zd* Cin, int64_t ldcin, double gamma, const zd* D,
                              int64_t ldd, zd* out, int64_t ldo, OzWorkspace& oz, cudaStream_t s,
                              cudaEvent_t ev_gemm_begin, cudaEvent_t ev_gemm_end) {
  if (m <= 0) return cudaSuccess;
  if (S > oz.H.S || S < 1 || oz.H.M != n) return cudaErrorInvalidValue;
  cudaError_t e = oz.H.nz == 3 ? oz_slice_b3(oz.B, OPN, Y, ldy, n, m, S, oz.H.Kp, s, 0)
                               : oz_slice_b(oz.B, OPN, Y, ldy, n, m, S, oz.H.Kp, s);
  if (e != cudaSuccess) return e;
  return oz_product(oz.H, oz.B, S, alpha, beta, Cin, ldcin, gamma, D, ldd, out, ldo, 0, 0, oz, s,
                    ev_gemm_begin, ev_gemm_end);
}

// General product with split operands: C = alpha op(A) op(B) + beta Cin + gamma D,
// op(A) M x K, op(B) K x N.  Uses the scratch operand buffers (not oz.H).
cudaError_t oz_gemm(int opA, const zd* A, int64_t lda, int opB, const zd* B, int64_t ldb, int M, int N,
                    int K, int S, double alpha, double beta, const zd* Cin, int64_t ldcin, double gamma,
                    const zd* D, int64_t ldd, zd* C, int64_t ldc, int a_lower, int c_lower,
                    OzWorkspace& oz, cudaStream_t s, int b_tri, int b_lower_half) {
  const bool g3 = oz_gauss(oz);
  cudaError_t e = g3 ? oz_slice_a3(oz.X, opA, A, lda, M, K, S, s) : oz_slice_a(oz.X, opA, A, lda, M, K, S, s);
  if (e != cudaSuccess) return e;
  e = g3 ? oz_slice_b3(oz.B, opB, B, ldb, K, N, S, oz.X.Kp, s, b_lower_half)
         : oz_slice_b(oz.B, opB, B, ldb, K, N, S, oz.X.Kp, s, b_lower_half);
  if (e != cudaSuccess) return e;
  return oz_product(oz.X, oz.B, S, alpha, beta, Cin, ldcin, gamma, D, ldd, C, ldc, a_lower, c_lower, oz,
                    s, nullptr, nullptr, b_tri);
}

int64_t oz_pair_count(int S) { return (int64_t)S * (S + 1) / 2; }

static cudaError_t alloc_a(OzA& a, int n_max, int S_max) {
  a.S_max = S_max;
  a.Kp_max = oz_padded_k(n_max);
  a.Mp_max = oz_padded_m(n_max);
  cudaError_t e = cudaMalloc((void**)&a.ptr, sizeof(__nv_bfloat16) * (size_t)S_max * a.Mp_max * a.Kp_max);
  if (e != cudaSuccess) return e;
  return cudaMalloc((void**)&a.e, sizeof(int) * (size_t)3 * a.Mp_max);  // 3 scale sets (Gauss form)
}

cudaError_t oz_alloc(OzWorkspace& oz, int n_max, int blk_max, int S_max) {
  cudaError_t e = alloc_a(oz.H, n_max, S_max);
  if (e != cudaSuccess) return e;
  e = alloc_a(oz.X, n_max, S_max);
  if (e != cudaSuccess) return e;
  // B operands: blocks of up to blk_max columns, and n_max columns for the reduction
  const int cols = std::max(n_max, blk_max);
  oz.B.S_max = S_max;
  oz.B.Kp_max = oz_padded_k(n_max);
  // covers both kernels' paddings and at least one full B box of the tcgen05 kernel
  oz.B.Np_max = ((std::max(cols, TC_BN) + OZ_BN - 1) / OZ_BN) * OZ_BN;
  // the Gauss form holds three K x N parts (K padded to 64 complex entries) per slice, the
  // embedding one 2K-row part
  const int64_t kp1 = ((n_max + OZ_BK - 1) / OZ_BK) * OZ_BK;
  oz.B.elems = std::max<int64_t>((int64_t)S_max * oz.B.Np_max * oz.B.Kp_max,
                                 (int64_t)3 * S_max * std::max(oz.B.Np_max, TC_BN) * kp1);
  e = cudaMalloc((void**)&oz.B.ptr, sizeof(__nv_bfloat16) * (size_t)oz.B.elems);
  if (e != cudaSuccess) return e;
  e = cudaMalloc((void**)&oz.B.e, sizeof(int) * (size_t)3 * oz.B.Np_max);
  if (e != cudaSuccess) return e;
  const int np_blk = ((blk_max + OZ_BN - 1) / OZ_BN) * OZ_BN;
  const size_t mp = (size_t)oz_padded_m(n_max);
  const size_t mp1 = (size_t)((n_max + TC_BM - 1) / TC_BM) * TC_BM;  // rows of a Gauss-form product
  // split partials: 32 splits of a block product, one split of an n x n product (three of
  // them in the Gauss form)
  oz.part_elems = std::max({(size_t)32 * mp * np_blk, mp * oz.B.Np_max, (size_t)3 * mp1 * oz.B.Np_max});
  return cudaMalloc((void**)&oz.part, sizeof(double) * oz.part_elems);
}

void oz_free(OzWorkspace& oz) {
  void* ptrs[] = {oz.H.ptr, oz.H.e, oz.X.ptr, oz.X.e, oz.B.ptr, oz.B.e, oz.part};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  oz = OzWorkspace{};
}
