// Complex FP64 GEMM for every dense product of the solver (filter steps, reduction to
// standard form, Gram matrices, basis rotations).
//
// On sm_103a the FP64 pipe issues two fused multiply-adds per clock per SM (about
// 1 TFLOP/s for the chip), so a complex GEMM is bound by FP64 issue, not by memory:
// a 64 x 32 complex tile reads 1.5 KB per k-step and issues 6144 FMAs.  The kernel
// therefore spends its effort on (1) fewer FMAs per complex product -- the 3M form
//   Re = Ar Br - Ai Bi,  Im = (Ar + Ai)(Br + Bi) - Ar Br - Ai Bi
// with the operand sums formed once per shared-memory tile, i.e. 3 real FMAs per
// complex multiply-add instead of 4 -- and (2) load balance over the 152 SMs: the K
// dimension is split so that every SM gets the same number of equal work units, and
// triangular operands skip the k-tiles that are known to be zero.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace {

constexpr int BM = 64, BN = 32, BK = 16, NT = 128;

struct Params {
  GemmDesc g;
  int splits;
  int tiles_m;
  zd* part;  // splits x (M x N) partial sums, ld = M; nullptr when splits == 1
};

__device__ __forceinline__ void tile_k_range(const GemmDesc& g, int i0, int j0, int& klo,
                                             int& khi) {
  klo = 0;
  khi = g.K;
  if (g.triA == 1) khi = min(khi, i0 + BM);
  if (g.triA == 2) klo = max(klo, i0);
  if (g.triB == 1) khi = min(khi, j0 + BN);
  if (g.triB == 2) klo = max(klo, j0);
  klo = (klo / BK) * BK;
}

template <int OPA, int OPB>
__global__ void __launch_bounds__(NT) zgemm3m_kernel(const Params p) {
  __shared__ double As[3][BK][BM];
  __shared__ double Bs[3][BK][BN];
  const GemmDesc& g = p.g;
  const int tid = threadIdx.x;
  const int tm = blockIdx.x % p.tiles_m, tn = blockIdx.x / p.tiles_m;
  const int i0 = tm * BM, j0 = tn * BN;
  if (g.lowerC && j0 > i0 + BM - 1) return;

  int klo, khi;
  tile_k_range(g, i0, j0, klo, khi);
  const int nkt = khi > klo ? (khi - klo + BK - 1) / BK : 0;
  const int per = (nkt + p.splits - 1) / p.splits;
  const int kt0 = min(nkt, blockIdx.y * per), kt1 = min(nkt, kt0 + per);

  const int tx = tid & 15, ty = tid >> 4;  // rows tx + 16 r, cols ty + 8 c
  double t1[4][4], t2[4][4], t3[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) t1[r][c] = t2[r][c] = t3[r][c] = 0.0;

  for (int kt = kt0; kt < kt1; ++kt) {
    const int k0 = klo + kt * BK;
    // ---- A tile: op(A)(i0+i, k0+k), i < BM, k < BK
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      int i, k;
      if (OPA == OPN) { i = tid & 63; k = (tid >> 6) + 2 * s; }
      else            { k = tid & 15; i = (tid >> 4) + 8 * s; }
      const int gi = i0 + i, gk = k0 + k;
      zd v = zmk(0.0, 0.0);
      if (gi < g.M && gk < g.K) {
        if (OPA == OPN) v = g.A[gi + (int64_t)gk * g.lda];
        else { v = g.A[gk + (int64_t)gi * g.lda]; v.y = -v.y; }
      }
      As[0][k][i] = v.x;
      As[1][k][i] = v.y;
      As[2][k][i] = v.x + v.y;
    }
    // ---- B tile: op(B)(k0+k, j0+j), k < BK, j < BN
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      int k, j;
      if (OPB == OPN) { k = tid & 15; j = (tid >> 4) + 8 * s; }
      else            { j = tid & 31; k = (tid >> 5) + 4 * s; }
      const int gj = j0 + j, gk = k0 + k;
      zd v = zmk(0.0, 0.0);
      if (gj < g.N && gk < g.K) {
        if (OPB == OPN) v = g.B[gk + (int64_t)gj * g.ldb];
        else { v = g.B[gj + (int64_t)gk * g.ldb]; v.y = -v.y; }
      }
      Bs[0][k][j] = v.x;
      Bs[1][k][j] = v.y;
      Bs[2][k][j] = v.x + v.y;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      double br[4], bi[4], bs[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        br[c] = Bs[0][kk][ty + 8 * c];
        bi[c] = Bs[1][kk][ty + 8 * c];
        bs[c] = Bs[2][kk][ty + 8 * c];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const double ar = As[0][kk][tx + 16 * r];
        const double ai = As[1][kk][tx + 16 * r];
        const double as = As[2][kk][tx + 16 * r];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          t1[r][c] = fma(ar, br[c], t1[r][c]);
          t2[r][c] = fma(ai, bi[c], t2[r][c]);
          t3[r][c] = fma(as, bs[c], t3[r][c]);
        }
      }
    }
    __syncthreads();
  }

  // ---- epilogue
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int gi = i0 + tx + 16 * r;
    if (gi >= g.M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gj = j0 + ty + 8 * c;
      if (gj >= g.N) continue;
      const zd acc = zmk(t1[r][c] - t2[r][c], t3[r][c] - t1[r][c] - t2[r][c]);
      if (p.splits > 1) {
        p.part[(int64_t)blockIdx.y * g.M * g.N + gi + (int64_t)gj * g.M] = acc;
        continue;
      }
      if (g.lowerC && gi < gj) continue;
      zd out = zscale(acc, g.alpha);
      if (g.beta != 0.0) out = zadd(out, zscale(g.Cin[gi + (int64_t)gj * g.ldcin], g.beta));
      if (g.gamma != 0.0) out = zadd(out, zscale(g.D[gi + (int64_t)gj * g.ldd], g.gamma));
      g.C[gi + (int64_t)gj * g.ldc] = out;
    }
  }
}

// Sum the split-K partials in split order (deterministic) and apply the epilogue.
__global__ void zgemm_splitk_epilogue(const Params p) {
  const GemmDesc& g = p.g;
  const int64_t total = (int64_t)g.M * g.N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int gi = (int)(e % g.M), gj = (int)(e / g.M);
    if (g.lowerC && gi < gj) continue;
    zd acc = zmk(0.0, 0.0);
    for (int s = 0; s < p.splits; ++s) acc = zadd(acc, p.part[(int64_t)s * total + e]);
    zd out = zscale(acc, g.alpha);
    if (g.beta != 0.0) out = zadd(out, zscale(g.Cin[gi + (int64_t)gj * g.ldcin], g.beta));
    if (g.gamma != 0.0) out = zadd(out, zscale(g.D[gi + (int64_t)gj * g.ldd], g.gamma));
    g.C[gi + (int64_t)gj * g.ldc] = out;
  }
}

// Scale-only path for K == 0 (alpha * 0 + beta Cin + gamma D).
__global__ void zgemm_k0(const GemmDesc g) {
  const int64_t total = (int64_t)g.M * g.N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int gi = (int)(e % g.M), gj = (int)(e / g.M);
    if (g.lowerC && gi < gj) continue;
    zd out = zmk(0.0, 0.0);
    if (g.beta != 0.0) out = zadd(out, zscale(g.Cin[gi + (int64_t)gj * g.ldcin], g.beta));
    if (g.gamma != 0.0) out = zadd(out, zscale(g.D[gi + (int64_t)gj * g.ldd], g.gamma));
    g.C[gi + (int64_t)gj * g.ldc] = out;
  }
}

}  // namespace

int sm_count() {
  static const int cached = [] {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }();
  return cached;
}

// Number of K splits: minimise the per-SM work ceil(units / SMs) / S, units = tiles * S,
// keeping at least two k-tiles per split and the partials within the workspace.
static int choose_splits(int tiles, int nkt, int64_t MN, size_t cap) {
  const int sms = sm_count();
  int best = 1;
  double best_cost = (double)((tiles + sms - 1) / sms);
  for (int S = 2; S <= 48; ++S) {
    if (nkt / S < 2) break;
    if ((size_t)S * (size_t)MN > cap) break;
    const int64_t units = (int64_t)tiles * S;
    const double cost = (double)((units + sms - 1) / sms) / S + 0.002 * S;
    if (cost < best_cost * 0.97) { best_cost = cost; best = S; }
  }
  return best;
}

cudaError_t zgemm_run(const GemmDesc& g, Workspace& ws, cudaStream_t stream) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  if (g.K <= 0) {
    zgemm_k0<<<std::min<int64_t>(1024, ((int64_t)g.M * g.N + 255) / 256), 256, 0, stream>>>(g);
    CHFSI_COUNT_LAUNCH();
    return cudaGetLastError();
  }
  Params p;
  p.g = g;
  p.tiles_m = (g.M + BM - 1) / BM;
  const int tiles_n = (g.N + BN - 1) / BN;
  int tiles = p.tiles_m * tiles_n;
  int active = tiles;
  if (g.lowerC) {
    active = 0;
    for (int tn = 0; tn < tiles_n; ++tn) {
      const int j0 = tn * BN;
      const int first_tm = j0 / BM;  // tiles with i0 + BM - 1 >= j0
      active += std::max(0, p.tiles_m - first_tm);
    }
  }
  // typical k-tiles per tile (triangular operands halve it on average)
  int nkt = (g.K + BK - 1) / BK;
  if (g.triA || g.triB) nkt = std::max(1, nkt / 2);
  p.splits = choose_splits(active, nkt, (int64_t)g.M * g.N, ws.splitk_elems);
  p.part = p.splits > 1 ? ws.splitk : nullptr;
  dim3 grid(tiles, p.splits);
  if (g.opA == OPN && g.opB == OPN) zgemm3m_kernel<OPN, OPN><<<grid, NT, 0, stream>>>(p);
  else if (g.opA == OPN && g.opB == OPC) zgemm3m_kernel<OPN, OPC><<<grid, NT, 0, stream>>>(p);
  else if (g.opA == OPC && g.opB == OPN) zgemm3m_kernel<OPC, OPN><<<grid, NT, 0, stream>>>(p);
  else zgemm3m_kernel<OPC, OPC><<<grid, NT, 0, stream>>>(p);
  CHFSI_COUNT_LAUNCH();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (p.splits > 1) {
    const int64_t total = (int64_t)g.M * g.N;
    const int blocks = (int)std::min<int64_t>(4 * sm_count(), (total + 255) / 256);
    zgemm_splitk_epilogue<<<blocks, 256, 0, stream>>>(p);
    CHFSI_COUNT_LAUNCH();
    e = cudaGetLastError();
  }
  return e;
}
