// Learned per-vector filter degree (an addition to the paper: the adaptive degree of its
// Section 3.1 trade-off between block size and degree, learned from the solver's own logs).
//
// The closed-form rule assumes that a degree-d filter reduces the residual of Ritz vector i
// by rho_i^d, rho_i = exp(acosh|t_i|).  The model predicts a correction g(x) to that rate,
// rate_i = ln(rho_i) * exp(g(x_i)), from eight features of the vector and the loop: its log
// residual over the last three loops, the degrees of the last two, its Ritz-value position
// relative to the filter interval and the filter bounds (the list is in include/chfsi.h),
// with an 8 -> 64 -> 64 -> 64 -> 1 perceptron (tanh hidden units, linear output).  The
// degree is then clamp(ceil(ln(r_i / tau) / rate_i), deg_min, deg_max), the closed form
// wherever that is not finite; an untrained model (zero output layer, g = 0) gives the
// closed form exactly.
//
// Training fits g to the logged per-degree reduction rates with Adam on mean squared error;
// one CTA runs an epoch (minibatches in sub-chunks of 64 samples, every gradient entry owned
// by one thread and accumulated in shared memory, so the sums over samples have a fixed
// order).  The solver evaluates the model with FP16 weights, one warp per vector.
#include <cuda_fp16.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace {

constexpr int IN = CHFSI_MLP_IN, HID = CHFSI_MLP_HID;
constexpr int NPARAM = HID * IN + HID + 2 * (HID * HID + HID) + HID + 1;
static_assert(NPARAM == CHFSI_MLP_NPARAM, "parameter count of the C interface");
constexpr int CHUNK = 64;           // samples per sub-chunk
constexpr int MLP_THREADS = 512;

// Flattened parameter offsets (the order of the chfsi_mlp struct).
constexpr int OW1 = 0, OB1 = OW1 + HID * IN, OW2 = OB1 + HID, OB2 = OW2 + HID * HID,
              OW3 = OB2 + HID, OB3 = OW3 + HID * HID, OW4 = OB3 + HID, OB4 = OW4 + HID;
static_assert(OB4 + 1 == NPARAM, "parameter layout");

// Activations are stored [unit][sample] with rows padded to CHUNK + 1 words, so that both
// access patterns (lanes along samples in the forward pass, lanes along units in the weight
// gradients) hit distinct shared-memory banks.  The gradient accumulates in shared memory
// (G), each entry owned by one thread, so no per-thread arrays are needed.
constexpr int LDC = CHUNK + 1;
struct MlpShared {
  float W[NPARAM];
  float G[NPARAM];
  float xh[IN][LDC];
  float h1[HID][LDC];
  float h2[HID][LDC];
  float h3[HID][LDC];   // activations of layer 3, then dL/d(pre-activation) of layers 3 and 1
  float d[HID][LDC];    // dL/d(pre-activation) of layer 2
  float dy[CHUNK];
};

// One hidden layer: out[j][b] = tanh(b_j + sum_k W[j][k] in[k][b]) for the chunk.
template <int NIN>
__device__ void dense_tanh(const float* W, const float* bias, const float (*in)[LDC], float (*out)[LDC]) {
  for (int e = threadIdx.x; e < HID * CHUNK; e += blockDim.x) {
    const int j = e / CHUNK, b = e % CHUNK;
    float a = bias[j];
#pragma unroll 8
    for (int k = 0; k < NIN; ++k) a += W[j * NIN + k] * in[k][b];
    out[j][b] = tanhf(a);
  }
  __syncthreads();
}

// Forward of `cnt` samples (indices idx[0..cnt)) into s.h1 .. s.h3 and y.
__device__ void mlp_forward_chunk(MlpShared& s, const float* X, const int* idx, int cnt,
                                  const float* mean, const float* scale, float* y) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < IN * CHUNK; e += nt) {
    const int f = e / CHUNK, b = e % CHUNK;
    s.xh[f][b] = (b < cnt) ? (X[(int64_t)idx[b] * IN + f] - mean[f]) * scale[f] : 0.f;
  }
  __syncthreads();
  dense_tanh<IN>(s.W + OW1, s.W + OB1, s.xh, s.h1);
  dense_tanh<HID>(s.W + OW2, s.W + OB2, s.h1, s.h2);
  dense_tanh<HID>(s.W + OW3, s.W + OB3, s.h2, s.h3);
  for (int b = tid; b < CHUNK; b += nt) {
    float a = s.W[OB4];
    for (int k = 0; k < HID; ++k) a += s.W[OW4 + k] * s.h3[k][b];
    y[b] = a;
  }
  __syncthreads();
}

// G[W] += delta in^T and G[bias] += sum_b delta for a layer with NIN inputs.
template <int NIN>
__device__ void layer_grad(float* G, int ow, int ob, const float (*delta)[LDC], const float (*in)[LDC]) {
  for (int e = threadIdx.x; e < HID * NIN + HID; e += blockDim.x) {
    float a = 0.f;
    if (e < HID * NIN) {
      const int j = e / NIN, k = e % NIN;
      for (int b = 0; b < CHUNK; ++b) a += delta[j][b] * in[k][b];
      G[ow + e] += a;
    } else {
      const int j = e - HID * NIN;
      for (int b = 0; b < CHUNK; ++b) a += delta[j][b];
      G[ob + j] += a;
    }
  }
}

// out[k][b] = (sum_j W[j][k] delta[j][b]) (1 - act[k][b]^2): back through a HID x HID layer
// and the tanh of the layer below it.  out may not alias delta.
__device__ void back_delta(const float* W, const float (*delta)[LDC], const float (*act)[LDC],
                           float (*out)[LDC]) {
  for (int e = threadIdx.x; e < HID * CHUNK; e += blockDim.x) {
    const int k = e / CHUNK, b = e % CHUNK;
    float a = 0.f;
    for (int j = 0; j < HID; ++j) a += W[j * HID + k] * delta[j][b];
    const float h = act[k][b];
    out[k][b] = a * (1.f - h * h);
  }
}

// Backward of one sub-chunk: s.dy holds dL/dy per sample (0 beyond the chunk's samples);
// adds the chunk's gradient into s.G.
__device__ void mlp_backward_chunk(MlpShared& s) {
  const int tid = threadIdx.x, nt = blockDim.x;
  // output layer
  for (int e = tid; e < HID + 1; e += nt) {
    float a = 0.f;
    if (e < HID)
      for (int b = 0; b < CHUNK; ++b) a += s.dy[b] * s.h3[e][b];
    else
      for (int b = 0; b < CHUNK; ++b) a += s.dy[b];
    s.G[OW4 + e] += a;   // OB4 == OW4 + HID
  }
  __syncthreads();
  // h3 <- delta3 = dy w4 (1 - h3^2)
  for (int e = tid; e < HID * CHUNK; e += nt) {
    const int j = e / CHUNK, b = e % CHUNK;
    const float h = s.h3[j][b];
    s.h3[j][b] = s.dy[b] * s.W[OW4 + j] * (1.f - h * h);
  }
  __syncthreads();
  // layer 3 parameters from (delta3, h2); d <- delta2 = (W3^T delta3)(1 - h2^2)
  layer_grad<HID>(s.G, OW3, OB3, s.h3, s.h2);
  back_delta(s.W + OW3, s.h3, s.h2, s.d);
  __syncthreads();
  // layer 2 parameters from (delta2, h1); h3 <- delta1 = (W2^T delta2)(1 - h1^2)
  layer_grad<HID>(s.G, OW2, OB2, s.d, s.h1);
  back_delta(s.W + OW2, s.d, s.h1, s.h3);
  __syncthreads();
  // layer 1 parameters from (delta1, xh)
  layer_grad<IN>(s.G, OW1, OB1, s.h3, s.xh);
  __syncthreads();
}

// One epoch of Adam over minibatches of `batch` samples (order idx), in place on params,
// with moments m1, m2 and the step counter *step (device).  One CTA.  With grad != nullptr
// the gradient of the last minibatch is also written there (batch = n and lr = 0 give the
// gradient of L = 1/(2n) sum (y - z)^2 over all samples, parameters unchanged).
__global__ void __launch_bounds__(MLP_THREADS) mlp_epoch_kernel(float* params, float* m1, float* m2, int* step,
                                                                const float* X, const float* z, const int* idx,
                                                                int n, int batch, float lr, const float* mean,
                                                                const float* scale, float* loss, float* grad) {
  extern __shared__ unsigned char mlp_smem[];
  MlpShared& s = *reinterpret_cast<MlpShared*>(mlp_smem);
  __shared__ float yv[CHUNK];
  __shared__ float lsum;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < NPARAM; e += nt) s.W[e] = params[e];
  if (tid == 0) lsum = 0.f;
  __syncthreads();
  int t = *step;
  for (int b0 = 0; b0 < n; b0 += batch) {
    const int bn = min(batch, n - b0);
    for (int e = tid; e < NPARAM; e += nt) s.G[e] = 0.f;
    __syncthreads();
    for (int c0 = 0; c0 < bn; c0 += CHUNK) {
      const int cnt = min(CHUNK, bn - c0);
      mlp_forward_chunk(s, X, idx + b0 + c0, cnt, mean, scale, yv);
      if (tid == 0) {
        float l = 0.f;
        for (int b = 0; b < cnt; ++b) {
          const float d = yv[b] - z[idx[b0 + c0 + b]];
          l += d * d;
        }
        lsum += l;
      }
      for (int b = tid; b < CHUNK; b += nt)
        s.dy[b] = (b < cnt) ? (yv[b] - z[idx[b0 + c0 + b]]) / (float)bn : 0.f;
      __syncthreads();
      mlp_backward_chunk(s);
    }
    if (grad && b0 + batch >= n)
      for (int e = tid; e < NPARAM; e += nt) grad[e] = s.G[e];
    // Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the entries this thread owns
    ++t;
    const float c1 = 1.f - powf(0.9f, (float)t), c2 = 1.f - powf(0.999f, (float)t);
    for (int e = tid; e < NPARAM; e += nt) {
      const float g = s.G[e];
      const float gm = 0.9f * m1[e] + 0.1f * g;
      const float gv = 0.999f * m2[e] + 0.001f * g * g;
      m1[e] = gm;
      m2[e] = gv;
      s.W[e] -= lr * (gm / c1) / (sqrtf(gv / c2) + 1e-8f);
    }
    __syncthreads();
  }
  for (int e = tid; e < NPARAM; e += nt) params[e] = s.W[e];
  if (tid == 0) {
    *step = t;
    *loss = 0.5f * lsum / (float)n;
  }
}

__global__ void __launch_bounds__(MLP_THREADS) mlp_forward_kernel(const float* params, const float* X, const int* idx, int n,
                                   const float* mean, const float* scale, float* y) {
  extern __shared__ unsigned char mlp_smem[];
  MlpShared& s = *reinterpret_cast<MlpShared*>(mlp_smem);
  __shared__ float yv[CHUNK];
  for (int e = threadIdx.x; e < NPARAM; e += blockDim.x) s.W[e] = params[e];
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += CHUNK) {
    const int cnt = min(CHUNK, n - c0);
    mlp_forward_chunk(s, X, idx + c0, cnt, mean, scale, yv);
    for (int b = threadIdx.x; b < cnt; b += blockDim.x) y[c0 + b] = yv[b];
    __syncthreads();
  }
}

// SplitMix64 (Steele, Lea & Flood 2014) for the weight initialisation.
uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
  cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes); }
};

}  // namespace

// --------------------------------------------------------------------------- host side
int mlp_param_count() { return NPARAM; }
size_t mlp_smem_bytes() { return sizeof(MlpShared); }

cudaError_t mlp_to_half(const chfsi_mlp* m, __half* dst_dev, cudaStream_t s) {
  std::vector<__half> h(NPARAM + 2 * IN);
  const float* p = reinterpret_cast<const float*>(m);
  for (int e = 0; e < NPARAM; ++e) h[e] = __float2half(p[e]);
  for (int f = 0; f < IN; ++f) {
    h[NPARAM + f] = __float2half(m->mean[f]);
    h[NPARAM + IN + f] = __float2half(m->scale[f]);
  }
  cudaError_t e = cudaMemcpyAsync(dst_dev, h.data(), sizeof(__half) * h.size(), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

static_assert(sizeof(chfsi_mlp) == sizeof(float) * (NPARAM + 2 * IN), "chfsi_mlp layout");

extern "C" {

void chfsi_mlp_init(chfsi_mlp* m, uint64_t seed) {
  if (!m) return;
  std::memset(m, 0, sizeof(*m));
  uint64_t st = seed;
  auto unif = [&]() { return (double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0); };
  const float a1 = std::sqrt(6.0f / (IN + HID)), a2 = std::sqrt(6.0f / (HID + HID));
  for (int e = 0; e < HID * IN; ++e) m->w1[e] = (float)((2.0 * unif() - 1.0) * a1);
  for (int e = 0; e < HID * HID; ++e) m->w2[e] = (float)((2.0 * unif() - 1.0) * a2);
  for (int e = 0; e < HID * HID; ++e) m->w3[e] = (float)((2.0 * unif() - 1.0) * a2);
  // zero output layer: the untrained model predicts no correction (the closed form)
  for (int f = 0; f < IN; ++f) m->scale[f] = 1.0f;
}

}  // extern "C"

// Runs `epochs` epochs of Adam on (X, z); per-feature mean/scale are set from X first.
cudaError_t mlp_train(chfsi_mlp* m, const float* X, const float* z, int64_t n, int epochs, int batch,
                      float lr, uint64_t seed, float* loss_out, cudaStream_t s) {
  if (n <= 0 || epochs < 0 || batch < 1) return cudaErrorInvalidValue;
  for (int f = 0; f < IN; ++f) {
    double mu = 0.0, v = 0.0;
    for (int64_t i = 0; i < n; ++i) mu += X[i * IN + f];
    mu /= (double)n;
    for (int64_t i = 0; i < n; ++i) v += (X[i * IN + f] - mu) * (X[i * IN + f] - mu);
    const double sd = std::sqrt(v / (double)n);
    m->mean[f] = (float)mu;
    m->scale[f] = (float)(sd > 1e-12 ? 1.0 / sd : 1.0);
  }
  DevBuf dP, dM1, dM2, dStep, dX, dZ, dIdx, dNorm, dLoss;
  cudaError_t e;
  if ((e = dP.alloc(sizeof(float) * NPARAM)) || (e = dM1.alloc(sizeof(float) * NPARAM)) ||
      (e = dM2.alloc(sizeof(float) * NPARAM)) || (e = dStep.alloc(sizeof(int))) ||
      (e = dX.alloc(sizeof(float) * n * IN)) || (e = dZ.alloc(sizeof(float) * n)) ||
      (e = dIdx.alloc(sizeof(int) * n)) || (e = dNorm.alloc(sizeof(float) * 2 * IN)) ||
      (e = dLoss.alloc(sizeof(float))))
    return e;
  float* P = (float*)dP.p;
  float* norm = (float*)dNorm.p;
  if ((e = cudaMemcpyAsync(P, m, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemsetAsync(dM1.p, 0, sizeof(float) * NPARAM, s)) ||
      (e = cudaMemsetAsync(dM2.p, 0, sizeof(float) * NPARAM, s)) ||
      (e = cudaMemsetAsync(dStep.p, 0, sizeof(int), s)) ||
      (e = cudaMemcpyAsync(dX.p, X, sizeof(float) * n * IN, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(dZ.p, z, sizeof(float) * n, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(norm, m->mean, sizeof(float) * IN, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(norm + IN, m->scale, sizeof(float) * IN, cudaMemcpyHostToDevice, s)))
    return e;
  const size_t smem = sizeof(MlpShared);
  if ((e = cudaFuncSetAttribute(mlp_epoch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
    return e;
  std::vector<int> idx(n);
  uint64_t st = seed;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int64_t i = 0; i < n; ++i) idx[i] = (int)i;
    for (int64_t i = n - 1; i > 0; --i) std::swap(idx[i], idx[splitmix(st) % (uint64_t)(i + 1)]);
    if ((e = cudaMemcpyAsync(dIdx.p, idx.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s))) return e;
    mlp_epoch_kernel<<<1, MLP_THREADS, smem, s>>>(P, (float*)dM1.p, (float*)dM2.p, (int*)dStep.p,
                                                  (const float*)dX.p, (const float*)dZ.p, (const int*)dIdx.p,
                                                  (int)n, batch, lr, norm, norm + IN, (float*)dLoss.p, nullptr);
    CHFSI_COUNT_LAUNCH();
    if ((e = cudaGetLastError())) return e;
    // the index buffer is rewritten next epoch: wait for this epoch's kernel first
    if ((e = cudaStreamSynchronize(s))) return e;
  }
  if ((e = cudaMemcpyAsync(m, P, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, s))) return e;
  float l = NAN;
  if (epochs > 0 && (e = cudaMemcpyAsync(&l, dLoss.p, sizeof(float), cudaMemcpyDeviceToHost, s))) return e;
  if ((e = cudaStreamSynchronize(s))) return e;
  if (loss_out) *loss_out = l;
  return cudaSuccess;
}

// One epoch of Adam in a caller-given sample order with caller-given moments (host in, host
// out), for the parity test of the optimiser against the CPU oracle: params, m1, m2 (NPARAM
// each) and *step are updated in place; the model's mean/scale are used as they are.
cudaError_t mlp_adam_epoch(chfsi_mlp* m, float* m1, float* m2, int* step, const float* X, const float* z,
                           const int* order, int64_t n, int batch, float lr, float* loss_out, cudaStream_t s) {
  if (n <= 0 || batch < 1) return cudaErrorInvalidValue;
  DevBuf dP, dM1, dM2, dStep, dX, dZ, dIdx, dNorm, dLoss;
  cudaError_t e;
  if ((e = dP.alloc(sizeof(float) * NPARAM)) || (e = dM1.alloc(sizeof(float) * NPARAM)) ||
      (e = dM2.alloc(sizeof(float) * NPARAM)) || (e = dStep.alloc(sizeof(int))) ||
      (e = dX.alloc(sizeof(float) * n * IN)) || (e = dZ.alloc(sizeof(float) * n)) ||
      (e = dIdx.alloc(sizeof(int) * n)) || (e = dNorm.alloc(sizeof(float) * 2 * IN)) ||
      (e = dLoss.alloc(sizeof(float))))
    return e;
  float* norm = (float*)dNorm.p;
  if ((e = cudaMemcpyAsync(dP.p, m, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(dM1.p, m1, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(dM2.p, m2, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(dStep.p, step, sizeof(int), cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(dX.p, X, sizeof(float) * n * IN, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(dZ.p, z, sizeof(float) * n, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(dIdx.p, order, sizeof(int) * n, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(norm, m->mean, sizeof(float) * IN, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(norm + IN, m->scale, sizeof(float) * IN, cudaMemcpyHostToDevice, s)))
    return e;
  const size_t smem = sizeof(MlpShared);
  if ((e = cudaFuncSetAttribute(mlp_epoch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
    return e;
  mlp_epoch_kernel<<<1, MLP_THREADS, smem, s>>>((float*)dP.p, (float*)dM1.p, (float*)dM2.p, (int*)dStep.p,
                                                (const float*)dX.p, (const float*)dZ.p, (const int*)dIdx.p,
                                                (int)n, batch, lr, norm, norm + IN, (float*)dLoss.p, nullptr);
  CHFSI_COUNT_LAUNCH();
  if ((e = cudaGetLastError())) return e;
  if ((e = cudaMemcpyAsync(m, dP.p, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(m1, dM1.p, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(m2, dM2.p, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(step, dStep.p, sizeof(int), cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(loss_out, dLoss.p, sizeof(float), cudaMemcpyDeviceToHost, s)))
    return e;
  return cudaStreamSynchronize(s);
}

// Gradient of the mean squared error over all n samples (host in, host out), and the loss:
// one epoch with a single minibatch of all samples and a zero step.
cudaError_t mlp_gradient(const chfsi_mlp* m, const float* X, const float* z, int64_t n, float* grad,
                         float* loss_out, cudaStream_t s) {
  if (n <= 0) return cudaErrorInvalidValue;
  DevBuf dP, dM1, dM2, dStep, dX, dZ, dIdx, dNorm, dG, dLoss;
  cudaError_t e;
  if ((e = dP.alloc(sizeof(float) * NPARAM)) || (e = dM1.alloc(sizeof(float) * NPARAM)) ||
      (e = dM2.alloc(sizeof(float) * NPARAM)) || (e = dStep.alloc(sizeof(int))) ||
      (e = dX.alloc(sizeof(float) * n * IN)) || (e = dZ.alloc(sizeof(float) * n)) ||
      (e = dIdx.alloc(sizeof(int) * n)) || (e = dNorm.alloc(sizeof(float) * 2 * IN)) ||
      (e = dG.alloc(sizeof(float) * NPARAM)) || (e = dLoss.alloc(sizeof(float))))
    return e;
  std::vector<int> idx(n);
  for (int64_t i = 0; i < n; ++i) idx[i] = (int)i;
  float* norm = (float*)dNorm.p;
  if ((e = cudaMemcpyAsync(dP.p, m, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemsetAsync(dM1.p, 0, sizeof(float) * NPARAM, s)) ||
      (e = cudaMemsetAsync(dM2.p, 0, sizeof(float) * NPARAM, s)) ||
      (e = cudaMemsetAsync(dStep.p, 0, sizeof(int), s)) ||
      (e = cudaMemcpyAsync(dX.p, X, sizeof(float) * n * IN, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(dZ.p, z, sizeof(float) * n, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(dIdx.p, idx.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(norm, m->mean, sizeof(float) * IN, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(norm + IN, m->scale, sizeof(float) * IN, cudaMemcpyHostToDevice, s)))
    return e;
  const size_t smem = sizeof(MlpShared);
  if ((e = cudaFuncSetAttribute(mlp_epoch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
    return e;
  mlp_epoch_kernel<<<1, MLP_THREADS, smem, s>>>((float*)dP.p, (float*)dM1.p, (float*)dM2.p, (int*)dStep.p,
                                                (const float*)dX.p, (const float*)dZ.p, (const int*)dIdx.p,
                                                (int)n, (int)n, 0.f, norm, norm + IN, (float*)dLoss.p,
                                                (float*)dG.p);
  CHFSI_COUNT_LAUNCH();
  if ((e = cudaGetLastError())) return e;
  if ((e = cudaMemcpyAsync(grad, dG.p, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(loss_out, dLoss.p, sizeof(float), cudaMemcpyDeviceToHost, s)))
    return e;
  return cudaStreamSynchronize(s);
}

cudaError_t mlp_predict(const chfsi_mlp* m, const float* X, int64_t n, float* y, cudaStream_t s) {
  if (n <= 0) return cudaErrorInvalidValue;
  DevBuf dP, dX, dIdx, dNorm, dY;
  cudaError_t e;
  if ((e = dP.alloc(sizeof(float) * NPARAM)) || (e = dX.alloc(sizeof(float) * n * IN)) ||
      (e = dIdx.alloc(sizeof(int) * n)) || (e = dNorm.alloc(sizeof(float) * 2 * IN)) ||
      (e = dY.alloc(sizeof(float) * n)))
    return e;
  std::vector<int> idx(n);
  for (int64_t i = 0; i < n; ++i) idx[i] = (int)i;
  float* norm = (float*)dNorm.p;
  if ((e = cudaMemcpyAsync(dP.p, m, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(dX.p, X, sizeof(float) * n * IN, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(dIdx.p, idx.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(norm, m->mean, sizeof(float) * IN, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(norm + IN, m->scale, sizeof(float) * IN, cudaMemcpyHostToDevice, s)))
    return e;
  const size_t smem = sizeof(MlpShared);
  if ((e = cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
    return e;
  mlp_forward_kernel<<<1, MLP_THREADS, smem, s>>>((const float*)dP.p, (const float*)dX.p, (const int*)dIdx.p,
                                                  (int)n, norm, norm + IN, (float*)dY.p);
  CHFSI_COUNT_LAUNCH();
  if ((e = cudaGetLastError())) return e;
  if ((e = cudaMemcpyAsync(y, dY.p, sizeof(float) * n, cudaMemcpyDeviceToHost, s))) return e;
  return cudaStreamSynchronize(s);
}
