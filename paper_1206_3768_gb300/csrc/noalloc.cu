// Allocation-free variant of the Rayleigh-Ritz eigensolver (chfsi_heev_noalloc).
//
// Some callers cannot call cudaMalloc: a host application that hands all device memory
// to its own pool allocator (a raw cudaMalloc outside the pool breaks its budget and
// accounting), or a latency-critical path that must not risk the implicit device-wide
// synchronisation cudaMalloc and cudaFree can cause.  Such callers cannot create a
// context either, because chfsi_create allocates the workspace.  This entry point runs the
// same cooperative Jacobi solver as chfsi_heev with its scratch in a fixed-size
// file-scope device array instead: 3 * 128 * 128 complex doubles for the two work copies
// of G and the rotated basis, plus the grid-barrier counters and the status word
// (786,688 bytes in all).  Every GPU that loads the library holds this array until the
// process exits.
#include <mutex>

#include "internal.cuh"

namespace {

constexpr int kMaxM = CHFSI_HEEV_NOALLOC_MAX;
constexpr size_t kWorkBytes = 3ull * kMaxM * kMaxM * sizeof(zd);
constexpr size_t kCtrlBytes = 256;  // barrier[4] (unsigned) then status[2] (int)

static __device__ __align__(256) unsigned char g_heev_scratch[kWorkBytes + kCtrlBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array for the current device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per device (with
// that device current) and cached.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_heev_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int chfsi_heev_noalloc(int32_t m, const chfsi_z* G, int64_t ldg, double* w,
                                  chfsi_z* V, int64_t ldv, void* cuda_stream) {
  if (m <= 0 || m > kMaxM || !G || !w || !V || ldg < m || ldv < m) return CHFSI_EINVAL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaGetLastError();  // report only this call's errors
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return CHFSI_ECUDA;
  zd* work = static_cast<zd*>(base);
  unsigned* barrier = reinterpret_cast<unsigned*>(static_cast<unsigned char*>(base) + kWorkBytes);
  int* status = reinterpret_cast<int*>(barrier + 4);
  // The array keeps the previous call's contents: the status word must start at zero (the
  // solver clears its own barrier counters).
  if (cudaMemsetAsync(status, 0, 2 * sizeof(int), s) != cudaSuccess) return CHFSI_ECUDA;
  if (jacobi_heev(reinterpret_cast<const zd*>(G), ldg, m, w, reinterpret_cast<zd*>(V), ldv, work,
                  barrier, status, s) != cudaSuccess)
    return CHFSI_ECUDA;
  int st[2] = {0, 0};
  if (cudaMemcpyAsync(st, status, sizeof st, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CHFSI_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CHFSI_ECUDA;
  if (st[0] & DEV_TIMEOUT) return CHFSI_ETIMEOUT;
  if (st[0] & DEV_NOCONV) return CHFSI_ENOCONV;
  return st[0] ? CHFSI_ECUDA : CHFSI_OK;
}
