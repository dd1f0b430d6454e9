// Process-wide cache of the device and pinned host blocks that contexts release.
//
// A context allocates a few dozen device buffers (the per-mode arena, the split copy of X, tree
// nodes, work areas) and one small pinned host buffer.  cudaMalloc costs ~30 us a call and
// cudaFree 30-260 us (it also waits for the device), cudaMallocHost / cudaFreeHost ~100 us each,
// so a short solve through cp_als_qr_run_host spent about 1 ms of its set-up and tear-down in
// them.  Blocks freed here stay cached, keyed by device and exact size, and the next request of
// that size on that device takes one back: repeated solves of one shape allocate nothing after
// the first.  The cached bytes of a device are capped at a quarter of its memory (a block that
// would exceed the cap is freed at once); cpqr_release_cached_memory() returns everything.
// A block's contents are whatever its last user left, like fresh cudaMalloc memory: users clear
// what must start at zero.  Before a cached block is handed out its pointer is checked with
// cudaPointerGetAttributes, so blocks lost to a cudaDeviceReset are dropped, not reused.
#include <cuda_runtime.h>

#include <cstddef>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "cpqr.h"

namespace cpqr {

namespace {

struct Cache {
  std::mutex mu;
  std::multimap<std::pair<int, size_t>, void*> dev;  // (device, bytes) -> block
  std::map<int, size_t> dev_bytes;                   // cached bytes per device
  std::map<int, size_t> dev_cap;                     // cap per device
  std::multimap<size_t, void*> host;                 // pinned host blocks by size
};

// Never destroyed: at process exit the driver reclaims the blocks, and freeing them from a static
// destructor could run after the runtime has shut down.
Cache& cache() {
  static Cache* c = new Cache();
  return *c;
}

constexpr size_t kHostCacheMax = 64;  // pinned blocks kept (each a few bytes)

// p is still a live device allocation of device d
bool still_device_memory(void* p, int d) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice && a.device == d;
}

}  // namespace

cudaError_t cache_malloc(void** p, size_t bytes) {
  int d = 0;
  cudaError_t e = cudaGetDevice(&d);
  if (e != cudaSuccess) return e;
  Cache& c = cache();
  {
    std::lock_guard<std::mutex> g(c.mu);
    for (;;) {
      auto it = c.dev.find({d, bytes});
      if (it == c.dev.end()) break;
      void* q = it->second;
      c.dev.erase(it);
      c.dev_bytes[d] -= bytes;
      if (still_device_memory(q, d)) {
        *p = q;
        return cudaSuccess;
      }
    }
  }
  e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    // cached blocks of other sizes may be what stands in the way
    cudaGetLastError();
    cpqr_release_cached_memory();
    e = cudaMalloc(p, bytes);
  }
  return e;
}

void cache_free(void* p, size_t bytes) {
  if (!p) return;
  // the block's own device (the current one may have changed since it was allocated)
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess || a.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    cudaFree(p);
    return;
  }
  const int d = a.device;
  Cache& c = cache();
  std::lock_guard<std::mutex> g(c.mu);
  auto cap = c.dev_cap.find(d);
  if (cap == c.dev_cap.end()) {
    // total memory of device d, read without making it current
    size_t tot = 0;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, d) == cudaSuccess) tot = prop.totalGlobalMem;
    else cudaGetLastError();
    cap = c.dev_cap.emplace(d, tot / 4).first;
  }
  if (c.dev_bytes[d] + bytes > cap->second) {
    cudaFree(p);
    return;
  }
  c.dev.emplace(std::make_pair(d, bytes), p);
  c.dev_bytes[d] += bytes;
}

cudaError_t cache_malloc_host(void** p, size_t bytes) {
  Cache& c = cache();
  {
    std::lock_guard<std::mutex> g(c.mu);
    auto it = c.host.find(bytes);
    if (it != c.host.end()) {
      *p = it->second;
      c.host.erase(it);
      return cudaSuccess;
    }
  }
  return cudaMallocHost(p, bytes);
}

void cache_free_host(void* p, size_t bytes) {
  if (!p) return;
  Cache& c = cache();
  std::lock_guard<std::mutex> g(c.mu);
  if (c.host.size() >= kHostCacheMax) {
    cudaFreeHost(p);
    return;
  }
  c.host.emplace(bytes, p);
}

}  // namespace cpqr

extern "C" cpqr_status cpqr_release_cached_memory(void) {
  using namespace cpqr;
  Cache& c = cache();
  std::vector<std::pair<int, void*>> dev;
  std::vector<void*> host;
  {
    std::lock_guard<std::mutex> g(c.mu);
    for (auto& kv : c.dev) dev.emplace_back(kv.first.first, kv.second);
    for (auto& kv : c.host) host.push_back(kv.second);
    c.dev.clear();
    c.dev_bytes.clear();
    c.host.clear();
  }
  int cur = 0;
  const bool have_cur = cudaGetDevice(&cur) == cudaSuccess;
  cpqr_status s = CPQR_OK;
  for (auto& b : dev) {
    if (cudaSetDevice(b.first) != cudaSuccess || cudaFree(b.second) != cudaSuccess) {
      cudaGetLastError();
      s = CPQR_ECUDA;
    }
  }
  if (have_cur) cudaSetDevice(cur);
  for (void* p : host)
    if (cudaFreeHost(p) != cudaSuccess) {
      cudaGetLastError();
      s = CPQR_ECUDA;
    }
  return s;
}
