// Allocation-free variant of irk_mg_restrict (declared in include/irk.h).
//
// Some callers cannot allocate device memory at the point where they restrict a
// residual: a serving process that has already handed every byte of its device
// memory budget to resident request state, or a latency-critical loop in which
// a cudaMalloc/cudaFree (which may synchronise the device) is not acceptable.
// For them, irk_mg_restrict_noalloc performs the same restriction as
// irk_mg_restrict but places the two intermediate grids of its axis-by-axis
// passes in one file-scope device array instead of the handle's buffers, and
// calls no allocating routine.
//
// * The array is kNoAllocScratchBytes (24 MiB) per device; every GPU on which
//   the library's kernels are loaded holds it until the process exits.
// * Its device address is resolved once per device, with that device current,
//   by the first call made on that device (cudaGetSymbolAddress; the host-side
//   name of the array is not a device address).  That first call should come
//   before any stream capture.
// * Every call shares the array and it keeps the last call's contents; each
//   call clears the part it uses first.  Calls whose work overlaps on the GPU
//   (different streams, different handles) race on the array: serialise them.
#include <cuda_runtime.h>

#include <mutex>

#include "irk.h"

irk_status irk_restrict_scratch_impl(irk_handle h, int level, const void* r, void* bc, void* scratch, size_t bytes);

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(24) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

}  // namespace

extern "C" irk_status irk_mg_restrict_noalloc(irk_handle h, int level, const void* r_fine, void* b_coarse) {
  if (!h) return IRK_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return IRK_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return IRK_EINVAL;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return IRK_ECUDA;
      }
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  return irk_restrict_scratch_impl(h, level, r_fine, b_coarse, scratch, kNoAllocScratchBytes);
}
