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
// * Its device address is resolved once per device, for the GPU the handle was
//   created on and with that GPU current (cudaGetSymbolAddress; the host-side
//   name of the array is not a device address), by the first call that uses
//   that GPU; the caller's current device is restored afterwards.  That first
//   call should come before any stream capture.  The address is cached for the
//   life of the process: a cudaDeviceReset of that GPU invalidates it, as it
//   invalidates every handle created there.
// * Every call shares the array and it keeps the last call's contents; each
//   call clears the part it uses first.  Calls whose work overlaps on the GPU
//   (different streams, different handles) race on the array: serialise them.
#include <cuda_runtime.h>

#include <mutex>

#include "irk.h"

using ScratchResolver = irk_status (*)(int device, void** addr, size_t* bytes, const char** why);
irk_status irk_restrict_scratch_impl(irk_handle h, int level, const void* r, void* bc, ScratchResolver resolve);

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(24) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the array on `device`, which the caller has made current.
irk_status resolve_scratch(int device, void** addr, size_t* bytes, const char** why) {
  if (device < 0 || device >= kMaxDevices) {
    *why = "device index beyond the 64 devices the address table holds";
    return IRK_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      *why = "cudaGetSymbolAddress failed (make the first call on a device outside stream capture)";
      return IRK_ECUDA;
    }
    g_scratch_addr[device] = p;
  }
  *addr = g_scratch_addr[device];
  *bytes = kNoAllocScratchBytes;
  return IRK_OK;
}

}  // namespace

extern "C" irk_status irk_mg_restrict_noalloc(irk_handle h, int level, const void* r_fine, void* b_coarse) {
  return irk_restrict_scratch_impl(h, level, r_fine, b_coarse, resolve_scratch);
}
