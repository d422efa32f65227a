// launch.cu -- the dynamic shared-memory cap of the library's kernels.
//
// A kernel that takes more than 48 KB of dynamic shared memory needs its cap raised
// (cudaFuncAttributeMaxDynamicSharedMemorySize) before the launch.  The cap is a property of the
// function on a device, shared by every context and host thread of the process: setting it to each
// launch's own size lets a concurrent launch on another thread (another context, another lattice)
// lower it between this thread's set and launch, which then fails with "invalid argument".  So the
// cap is raised once per (kernel, device) to the device's opt-in maximum, under a lock; occupancy
// and residency still follow the size each launch asks for.
#include <mutex>
#include <set>
#include <utility>

#include "internal.h"

namespace jtr {

cudaError_t allow_dyn_smem(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> raised;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes at{};
  if ((e = cudaFuncGetAttributes(&at, func)) != cudaSuccess) return e;
  int optin = 0;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  const size_t cap = (size_t)optin > at.sharedSizeBytes ? (size_t)optin - at.sharedSizeBytes : 0;
  if (bytes > cap) return cudaErrorInvalidValue;   // too large for any launch of this kernel
  std::lock_guard<std::mutex> lock(mu);
  if (raised.count({func, dev})) return cudaSuccess;
  if ((e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap)) != cudaSuccess) return e;
  raised.insert({func, dev});
  return cudaSuccess;
}

}  // namespace jtr
