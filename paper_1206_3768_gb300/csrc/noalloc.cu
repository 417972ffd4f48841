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
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.cuh"

namespace {

constexpr int kMaxM = CHFSI_HEEV_NOALLOC_MAX;
constexpr size_t kWorkBytes = 3ull * kMaxM * kMaxM * sizeof(zd);
constexpr size_t kCtrlBytes = 256;  // barrier[4] (unsigned) then status[2] (int)

static __device__ __align__(256) unsigned char g_heev_scratch[kWorkBytes + kCtrlBytes];

constexpr int kMaxDevices = 64;
struct ScratchSlot {
  unsigned long long ctx_id = 0;  // unique id of the context the address belongs to (0: none)
  void* addr = nullptr;
};
std::mutex g_mu;
ScratchSlot g_slot[kMaxDevices];

// Unique id of the calling thread's current context (0 if there is none yet or the driver
// entry points are unavailable).  Context ids are never reused within a process, so a
// context that was destroyed and created again (cudaDeviceReset, or the host application
// resetting the primary context) has a new id.
unsigned long long current_context_id() {
  static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
    fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(fn);
  });
  if (!get_current || !get_id) return 0;
  CUcontext c = nullptr;
  if (get_current(&c) != CUDA_SUCCESS || !c) return 0;
  unsigned long long id = 0;
  if (get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Device address of the scratch array for the current device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up with cudaGetSymbolAddress
// (with that device current) at set-up and cached for the device together with the id of
// its context; a later call under another context (after a reset) looks it up again.  When
// the context id cannot be read, every call looks the address up.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  ScratchSlot& slot = g_slot[dev];
  const unsigned long long id = current_context_id();
  if (id != 0 && slot.ctx_id == id && slot.addr) {
    *out = slot.addr;
    return cudaSuccess;
  }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_heev_scratch);  // also creates the context if needed
  if (e != cudaSuccess) return e;
  slot.addr = p;
  slot.ctx_id = current_context_id();
  *out = p;
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
