// tt_full_noalloc: tt_full with its scratch in a fixed device array, for
// callers that cannot allocate device memory during the call.
//
// The scratch lives in a file-scope __device__ array of kNoAllocScratchBytes.
// The CUDA runtime loads this file's module (and so reserves the array on a
// device) when the module is first used on that device -- with the default
// lazy module loading, that is the first tt_full_noalloc call there, not the
// loading of the library.  From then on the device holds the array until the
// process exits.  In host code the array's name is only a host-side stand-in,
// so its device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached.  That first
// call on a device may therefore allocate device memory and synchronize: make
// it before another allocator's pool takes the device's memory and before
// capturing work on that device into a stream.
#include <stdio.h>

#include <mutex>

#include "internal.h"
#include "ttutv.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

cudaError_t scratch_for_current_device(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" {

size_t tt_full_noalloc_max_work_bytes(void) { return kNoAllocScratchBytes; }

tt_status tt_full_noalloc(int32_t d, const int64_t* dims, const int64_t* ranks,
                          const void* const* cores, int32_t dtype, void* out, void* stream) {
  char msg[256];
  if (d < 2 || d > TT_MAXD || !dims || !ranks || !cores || !out ||
      (dtype != TT_F32 && dtype != TT_F64)) {
    ttk::set_last_error("tt_full_noalloc: bad argument");
    return TT_EINVAL;
  }
  const size_t need = tt_full_work_bytes(d, dims, ranks, dtype);
  if (need == 0 || need > kNoAllocScratchBytes) {
    snprintf(msg, sizeof(msg),
             "tt_full_noalloc: this contraction needs %zu bytes of scratch, above the fixed %zu",
             need, kNoAllocScratchBytes);
    ttk::set_last_error(msg);
    return TT_EINVAL;
  }
  void* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "tt_full_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    ttk::set_last_error(msg);
    return TT_ECUDA;
  }
  // Every intermediate and split-K partial in the scratch is written before it
  // is read, so nothing needs clearing between calls.
  return tt_full(d, dims, ranks, cores, dtype, out, scratch, stream);
}

}  // extern "C"
