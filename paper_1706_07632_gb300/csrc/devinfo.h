// Per-device launch facts shared by the launchers: the SM count (grids are sized in multiples of
// it) and the per-kernel state the CUDA runtime keeps per device.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <mutex>

namespace fhmg {

// Launch state that the CUDA runtime keeps per device is cached per device (one slot per device
// index below kDevSlots; devices beyond that are queried on every launch), under a mutex, since
// host threads may launch concurrently.
constexpr int kDevSlots = 64;

// Streaming multiprocessors of the current device (grids are sized in multiples of it).
inline int device_sms() {
  static std::atomic<int> cache[kDevSlots];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  const bool slot = dev >= 0 && dev < kDevSlots;
  if (slot) {
    const int v = cache[dev].load(std::memory_order_acquire);
    if (v > 0) return v;
  }
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 1;
  }
  if (slot) cache[dev].store(n, std::memory_order_release);
  return n;
}

// Per-kernel, per-device launch state: the raised dynamic shared-memory limit and the resident
// CTAs per SM at the last shared-memory size.
struct KernelCache {
  std::mutex mu;
  size_t smem_limit[kDevSlots] = {};
  size_t occ_smem[kDevSlots] = {};
  int occ[kDevSlots] = {};
};

// Raises kern's dynamic shared-memory limit to smem on the current device (when above the 48 KB
// default) and returns the resident CTAs per SM of a launch with `block` threads and smem bytes.
template <typename K>
inline cudaError_t prepare_launch(K kern, int block, size_t smem, KernelCache& c, int* occ_out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool slot = dev >= 0 && dev < kDevSlots;
  std::lock_guard<std::mutex> lock(c.mu);
  if (smem > 48 * 1024 && (!slot || smem > c.smem_limit[dev])) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (slot) c.smem_limit[dev] = smem;
  }
  if (slot && c.occ[dev] > 0 && c.occ_smem[dev] == smem) {
    *occ_out = c.occ[dev];
    return cudaSuccess;
  }
  int o = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, block, smem) != cudaSuccess || o < 1) {
    cudaGetLastError();  // not sticky; keep it out of the launch check that follows
    o = 1;
  }
  if (slot) {
    c.occ_smem[dev] = smem;
    c.occ[dev] = o;
  }
  *occ_out = o;
  return cudaSuccess;
}

// Grid of a grid-stride elementwise kernel over n items with 256-thread blocks: enough blocks for
// every item, at most per_sm blocks per SM of the current device.
inline int grid_for(long long n, int per_sm) {
  const long long b = (n + 255) / 256;
  const long long cap = (long long)device_sms() * per_sm;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace fhmg
