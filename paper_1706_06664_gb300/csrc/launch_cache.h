// Per-process caches for launch set-up that does not change between launches: a kernel's
// dynamic shared-memory limit (an attribute that stays with the function in the device's
// context) and its resident blocks per SM for a block shape.  Without them every launch pays a
// driver call for the attribute and an occupancy query, which matters for small batches where
// the host's calls, not the kernels, set the rate.  Keys carry the device, so a process that
// drives several devices sets each one's attribute once.  (A context torn down with
// cudaDeviceReset loses the attributes; the library's handles are invalid after that anyway.)
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>

namespace ace {

namespace launch_cache_detail {
inline std::mutex& mu() {
  static std::mutex m;
  return m;
}
// (kernel, device) -> the limit last set
inline std::map<std::pair<const void*, int>, int>& limits() {
  static std::map<std::pair<const void*, int>, int> m;
  return m;
}
// (kernel, device, threads, dynamic shared bytes) -> resident blocks per SM
inline std::map<std::tuple<const void*, int, int, size_t>, int>& occupancy() {
  static std::map<std::tuple<const void*, int, int, size_t>, int> m;
  return m;
}
}  // namespace launch_cache_detail

// Sets kern's dynamic shared-memory limit to `bytes` on the current device unless it already is.
template <typename Kern>
inline cudaError_t smem_limit(Kern kern, int bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const auto key = std::make_pair(reinterpret_cast<const void*>(kern), dev);
  {
    std::lock_guard<std::mutex> lk(launch_cache_detail::mu());
    auto it = launch_cache_detail::limits().find(key);
    if (it != launch_cache_detail::limits().end() && it->second == bytes) return cudaSuccess;
  }
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(launch_cache_detail::mu());
  launch_cache_detail::limits()[key] = bytes;
  return cudaSuccess;
}

// Resident blocks of kern per SM with `threads` threads and `smem` dynamic shared bytes.
template <typename Kern>
inline cudaError_t blocks_per_sm(int* out, Kern kern, int threads, size_t smem) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const auto key = std::make_tuple(reinterpret_cast<const void*>(kern), dev, threads, smem);
  {
    std::lock_guard<std::mutex> lk(launch_cache_detail::mu());
    auto it = launch_cache_detail::occupancy().find(key);
    if (it != launch_cache_detail::occupancy().end()) {
      *out = it->second;
      return cudaSuccess;
    }
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(launch_cache_detail::mu());
  launch_cache_detail::occupancy()[key] = per_sm;
  *out = per_sm;
  return cudaSuccess;
}

}  // namespace ace
