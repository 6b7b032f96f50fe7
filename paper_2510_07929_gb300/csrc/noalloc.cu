// FP32 Gram product that allocates no device memory.
//
// Its scratch (the FP32 copy of V and the per-split partial row sums) lives in
// one file-scope __device__ array of kNoAllocScratchBytes.  Every GPU that loads
// this library reserves that array until the process exits.  Host code cannot
// use the array's name as a device address, so the address is looked up with
// cudaGetSymbolAddress once per device (with that device current) and cached.
#include <mutex>

#include "kqr_internal.h"

namespace kqr {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

cudaError_t gram_f32_scratch(Handle* h, const double* V, double* U, int m, unsigned char* scratch, size_t cap,
                             size_t* need, cudaStream_t st);

static std::mutex g_scratch_mu;
static unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};
static unsigned long long g_scratch_ctx[kMaxDevices] = {0};

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique ID of the current CUDA context (cuCtxGetId), 0 if unavailable.  A
// device reset destroys the primary context and the next one gets a new ID,
// which invalidates the cached address below.
static unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (CtxGetCurrentFn)p;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (CtxGetIdFn)p;
    looked_up = true;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS) return id;
  return 0;
}

// Device address of g_noalloc_scratch on `device` (the current device), looked
// up with cudaGetSymbolAddress once per device and context.
static cudaError_t scratch_address(int device, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  const unsigned long long ctx = current_context_id();
  if (!g_scratch_addr[device] || g_scratch_ctx[device] != ctx) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = static_cast<unsigned char*>(p);
    g_scratch_ctx[device] = ctx;
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

}  // namespace kqr

using namespace kqr;

extern "C" kqr_status kqr_kmatvec_fp32_noalloc_dev(kqr_handle* kh, const double* V, double* U, int64_t m,
                                                   void* stream) {
  if (!kh) return KQR_INVALID_ARG;
  Handle* h = &kh->h;
  KQR_SINGLE(h);
  if (!V || !U) return fail(h, KQR_INVALID_ARG, "V and U must be non-null");
  if (m < 1 || m > kMaxRhs) return fail(h, KQR_INVALID_ARG, "m must be in [1, 8]");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetDevice");
  if (dev != h->device) return fail(h, KQR_INVALID_ARG, "the handle's device must be the current device");
  if (dev < 0 || dev >= kMaxDevices) return fail(h, KQR_INVALID_ARG, "device index out of range");
  unsigned char* scratch = nullptr;
  if ((e = scratch_address(dev, &scratch)) != cudaSuccess) return cuda_fail(h, e, "cudaGetSymbolAddress");
  size_t need = 0;
  e = gram_f32_scratch(h, V, U, (int)m, scratch, kNoAllocScratchBytes, &need, pick_stream(h, stream));
  if (e == cudaErrorInvalidValue && need > kNoAllocScratchBytes)
    return fail(h, KQR_INVALID_ARG,
                "no-allocation Gram product needs " + std::to_string(need) + " bytes of scratch; the static array holds " +
                    std::to_string(kNoAllocScratchBytes));
  if (e != cudaSuccess) return cuda_fail(h, e, "no-allocation Gram product");
  return KQR_OK;
}
