// Allocation-free evaluation: the workspace is a static device array.
//
// For callers that cannot allocate device memory once they run: a real-time
// control loop under a no-allocation rule (an allocation can block for an
// unbounded time), or a plugin whose host application owns all device memory
// and hands it only input and output buffers.  The
// array below is reserved on every GPU that loads this library and stays until
// the process exits.  In host code its name is only a host-side stand-in, so
// its device address is looked up once per device with cudaGetSymbolAddress.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>

#include "internal.h"

static __device__ __align__(256) unsigned char cs_noalloc_scratch[CUSADI_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_scratch_mu;
std::map<int, void*> g_scratch_addr;  // device ordinal -> device address of the array
}  // namespace

extern "C" cusadi_status cusadi_eval_noalloc(cusadi_fn fn, const void* in, int64_t ld_in,
                                             void* out, int64_t ld_out, int64_t N,
                                             cusadi_stream stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return cusadi::report(CUSADI_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    auto it = g_scratch_addr.find(dev);
    if (it == g_scratch_addr.end()) {
      // set-up, once per device, with that device current
      e = cudaGetSymbolAddress(&scratch, cs_noalloc_scratch);
      if (e != cudaSuccess || scratch == nullptr)
        return cusadi::report(CUSADI_E_CUDA, std::string("cudaGetSymbolAddress of the scratch "
                                                         "region: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = scratch;
    } else {
      scratch = it->second;
    }
  }
  return cusadi::eval_in_scratch(fn, in, ld_in, out, ld_out, N, scratch,
                                 CUSADI_NOALLOC_SCRATCH_BYTES, stream);
}
