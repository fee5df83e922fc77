// Device memory of the library: a caching allocator in front of cudaMalloc.
//
// Handles, plans and workspaces are created and destroyed per solve by many
// callers (one handle per medium and step in an end-to-end loop), and
// cudaMalloc / cudaFree cost tens of microseconds each, cudaFree with an
// implicit device synchronisation.  Freed blocks are kept per (device, size
// class) and handed out again to a request of the same class.
//
// * Size classes: 512-byte multiples up to 1 MiB, 2 MiB multiples above.
// * A block goes back to the cache only after the device has finished with
//   it: vie_free synchronises the device first (what cudaFree does
//   implicitly), unless the caller declared the device idle (DeviceIdle).
// * At most kCacheCap bytes are kept; larger blocks, and blocks past the
//   cap, are released at once.  A cudaMalloc that fails releases the whole
//   cache and tries again.
// * Pinned host buffers (cudaMallocHost: the solvers' read-back scalars) are
//   cached the same way under the pseudo-device kHost.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "vie_internal.cuh"

namespace vie {

namespace {

constexpr size_t kCacheCap = 4ull << 30;
constexpr int kHost = -1;

struct Block {
  int device;
  size_t bytes;
};

std::mutex g_mu;
std::unordered_map<void *, Block> g_live;                 // blocks handed out
std::map<std::pair<int, size_t>, std::vector<void *>> g_free;  // cached, by (device, class)
size_t g_cached = 0;
thread_local int t_device_idle = 0;

size_t size_class(size_t bytes) {
  if (bytes == 0) bytes = 1;
  if (bytes <= (1u << 20)) return (bytes + 511) & ~(size_t)511;
  return (bytes + (2u << 20) - 1) & ~(((size_t)2 << 20) - 1);
}

// release every cached block (caller holds g_mu)
void release_cached() {
  int cur = 0;
  cudaGetDevice(&cur);
  for (auto &kv : g_free) {
    if (kv.second.empty()) continue;
    if (kv.first.first == kHost) {
      for (void *p : kv.second) cudaFreeHost(p);
      kv.second.clear();
      continue;
    }
    cudaSetDevice(kv.first.first);
    for (void *p : kv.second) cudaFree(p);
    kv.second.clear();
  }
  g_free.clear();
  g_cached = 0;
  cudaSetDevice(cur);
}

}  // namespace

DeviceIdle::DeviceIdle() { ++t_device_idle; }
DeviceIdle::~DeviceIdle() { --t_device_idle; }

namespace {

cudaError_t cached_alloc(void **p, size_t bytes, bool host) {
  int dev = kHost;
  cudaError_t e = host ? cudaSuccess : cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const size_t cls = size_class(bytes);
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_free.find({dev, cls});
  if (it != g_free.end() && !it->second.empty()) {
    *p = it->second.back();
    it->second.pop_back();
    g_cached -= cls;
    g_live[*p] = {dev, cls};
    return cudaSuccess;
  }
  e = host ? cudaMallocHost(p, cls) : cudaMalloc(p, cls);
  if (e != cudaSuccess) {
    cudaGetLastError();  // the failed allocation's error is not sticky
    release_cached();
    e = host ? cudaMallocHost(p, cls) : cudaMalloc(p, cls);
    if (e != cudaSuccess) return e;
  }
  g_live[*p] = {dev, cls};
  return cudaSuccess;
}

cudaError_t cached_free(void *p, bool host) {
  if (!p) return cudaSuccess;
  Block b;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_live.find(p);
    if (it == g_live.end()) return host ? cudaFreeHost(p) : cudaFree(p);  // not ours
    b = it->second;
    g_live.erase(it);
  }
  int cur = 0;
  cudaGetDevice(&cur);
  if (b.device != kHost && b.device != cur) cudaSetDevice(b.device);
  cudaError_t e = cudaSuccess;
  // no kernel or copy still uses the block (what cudaFree / cudaFreeHost wait for)
  if (!t_device_idle) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (b.bytes <= kCacheCap && g_cached + b.bytes <= kCacheCap) {
      g_free[{b.device, b.bytes}].push_back(p);
      g_cached += b.bytes;
      p = nullptr;
    }
  }
  if (p) e = host ? cudaFreeHost(p) : cudaFree(p);
  if (b.device != kHost && b.device != cur) cudaSetDevice(cur);
  return e;
}

}  // namespace

cudaError_t vie_malloc(void **p, size_t bytes) { return cached_alloc(p, bytes, false); }
cudaError_t vie_free(void *p) { return cached_free(p, false); }
cudaError_t vie_malloc_host(void **p, size_t bytes) { return cached_alloc(p, bytes, true); }
cudaError_t vie_free_host(void *p) { return cached_free(p, true); }

void vie_release_cached_memory() {
  std::lock_guard<std::mutex> lock(g_mu);
  cudaDeviceSynchronize();
  release_cached();
}

}  // namespace vie

extern "C" vie_status vie_release_memory(void) {
  vie::vie_release_cached_memory();
  return VIE_OK;
}
