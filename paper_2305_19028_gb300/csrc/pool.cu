// Device and pinned-host memory of the library's contexts and batches.
//
// Every device buffer goes through hook_alloc / hook_free, which serve it from one of three
// sources, remembered per pointer so that it returns to the one it came from:
//   - the caller's allocator (tls_set_allocator), when one is set;
//   - else the library's process-wide block cache (on by default): blocks freed by a destroyed
//     context or batch are kept per device and size class and handed to the next context that
//     asks for a block of that class, so that repeated create / solve / destroy cycles (a
//     server answering one problem per request) neither call cudaMalloc nor pay for cudaFree,
//     which synchronises the whole device;
//   - else cudaMalloc / cudaFree.
// The small pinned host blocks (read-back scalars) are cached the same way (cudaMallocHost and
// cudaFreeHost are costly calls). A block enters the cache only after the stream that used it
// has been synchronised, so a cached block is never still in use on the device. When cudaMalloc
// fails, the cache of that device is released and the allocation retried once. The state is
// heap-allocated and never destroyed: nothing is freed from static destructors, which may run
// after the CUDA runtime has shut down.
#include "../../include/tls.h"
#include "../../include/tls_debug.h"
#include "tls_internal.h"

#include <cstring>
#include <cstdint>
#include <map>
#include <mutex>
#include <unordered_map>
#include <utility>

namespace {

enum Source : int { kCuda = 0, kCache = 1, kUser = 2 };

struct Live {
  Source src;
  size_t bytes;          // size of the block as allocated (the cache's size class)
  int device;
  tls_free_fn release;   // caller's release function for kUser blocks
  void* user;
};

struct State {
  std::mutex mu;
  bool enabled = true;
  tls_alloc_fn alloc = nullptr;
  tls_free_fn release = nullptr;
  void* user = nullptr;
  std::unordered_map<void*, Live> live;                   // device blocks handed out
  std::multimap<std::pair<int, size_t>, void*> dev_free;  // (device, bytes) -> cached block
  std::multimap<size_t, void*> host_free;                 // bytes -> cached pinned block
  std::unordered_map<void*, size_t> host_live;            // pinned blocks handed out
  uint64_t cached_dev = 0, cached_host = 0, live_dev = 0;
  int poison = -1;                                        // fill byte for new blocks, or -1
};

State& st() {
  static State* s = new State();   // never destroyed (see the file comment)
  return *s;
}

// Size class: multiples of 512 B up to 1 MiB, of 2 MiB above.
size_t size_class(size_t bytes) {
  if (bytes == 0) bytes = 16;
  const size_t g = bytes <= ((size_t)1 << 20) ? 512 : ((size_t)2 << 20);
  return (bytes + g - 1) / g * g;
}

// Release every cached device block of `device` (all devices for -1); caller holds the lock.
uint64_t trim_device_locked(State& s, int device) {
  uint64_t freed = 0;
  int cur = -1;
  cudaGetDevice(&cur);
  for (auto it = s.dev_free.begin(); it != s.dev_free.end();) {
    if (device >= 0 && it->first.first != device) { ++it; continue; }
    if (it->first.first != cur) {
      cudaSetDevice(it->first.first);
      cur = it->first.first;
    }
    cudaFree(it->second);
    freed += it->first.second;
    it = s.dev_free.erase(it);
  }
  s.cached_dev -= freed;
  return freed;
}

// The block, filled with the poison byte when one is set (tls_pool_poison).
void* fill(const State& s, void* p, size_t bytes, cudaStream_t stream) {
  if (s.poison >= 0 && cudaMemsetAsync(p, s.poison, bytes, stream) != cudaSuccess)
    (void)cudaGetLastError();
  return p;
}

// Release every cached block (device and pinned host); caller holds the lock.
uint64_t trim_all_locked(State& s) {
  int cur = 0;
  cudaGetDevice(&cur);
  uint64_t freed = trim_device_locked(s, -1);
  cudaSetDevice(cur);
  for (auto& h : s.host_free) {
    cudaFreeHost(h.second);
    freed += h.first;
  }
  s.host_free.clear();
  s.cached_host = 0;
  (void)cudaGetLastError();
  return freed;
}

void sync_unless_capturing(cudaStream_t stream) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone)
    cudaStreamSynchronize(stream);
  (void)cudaGetLastError();
}

}  // namespace

namespace tls {

void* hook_alloc(size_t bytes, cudaStream_t stream) {
  State& s = st();
  std::lock_guard<std::mutex> lk(s.mu);
  int dev = 0;
  cudaGetDevice(&dev);
  void* p = nullptr;
  if (s.alloc) {
    if (bytes == 0) bytes = 16;
    p = s.alloc((uint64_t)bytes, (void*)stream, s.user);
    if (p) s.live[p] = {kUser, bytes, dev, s.release, s.user};
    return p;
  }
  if (!s.enabled) {
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      (void)cudaGetLastError();
      return nullptr;
    }
    s.live[p] = {kCuda, bytes, dev, nullptr, nullptr};
    s.live_dev += bytes;
    return fill(s, p, bytes, stream);
  }
  const size_t cls = size_class(bytes);
  // the smallest cached block of this device whose class is at least `cls` and at most a
  // quarter larger
  auto it = s.dev_free.lower_bound({dev, cls});
  if (it != s.dev_free.end() && it->first.first == dev && it->first.second <= cls + cls / 4) {
    p = it->second;
    const size_t got = it->first.second;
    s.dev_free.erase(it);
    s.cached_dev -= got;
    s.live[p] = {kCache, got, dev, nullptr, nullptr};
    s.live_dev += got;
    return fill(s, p, got, stream);
  }
  if (cudaMalloc(&p, cls) != cudaSuccess) {
    (void)cudaGetLastError();
    trim_device_locked(s, dev);
    cudaSetDevice(dev);
    if (cudaMalloc(&p, cls) != cudaSuccess) {
      (void)cudaGetLastError();
      return nullptr;
    }
  }
  s.live[p] = {kCache, cls, dev, nullptr, nullptr};
  s.live_dev += cls;
  return fill(s, p, cls, stream);
}

void hook_free(void* p, size_t /*bytes*/, cudaStream_t stream) {
  if (!p) return;
  State& s = st();
  std::unique_lock<std::mutex> lk(s.mu);
  auto it = s.live.find(p);
  if (it == s.live.end()) return;   // not ours
  const Live b = it->second;
  s.live.erase(it);
  if (b.src == kUser) {
    lk.unlock();
    if (b.release) b.release(p, (uint64_t)b.bytes, (void*)stream, b.user);
    return;
  }
  s.live_dev -= b.bytes;
  if (b.src == kCuda || !s.enabled) {
    cudaFree(p);
    return;
  }
  lk.unlock();
  sync_unless_capturing(stream);   // nothing on the device uses the block any more
  lk.lock();
  s.dev_free.insert({{b.device, b.bytes}, p});
  s.cached_dev += b.bytes;
}

void* host_alloc(size_t bytes) {
  State& s = st();
  std::lock_guard<std::mutex> lk(s.mu);
  const size_t cls = size_class(bytes);
  void* p = nullptr;
  if (s.enabled) {
    auto it = s.host_free.find(cls);
    if (it != s.host_free.end()) {
      p = it->second;
      s.host_free.erase(it);
      s.cached_host -= cls;
      s.host_live[p] = cls;
      if (s.poison >= 0) std::memset(p, s.poison, cls);
      return p;
    }
  }
  if (cudaMallocHost(&p, cls) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  s.host_live[p] = cls;
  if (s.poison >= 0) std::memset(p, s.poison, cls);
  return p;
}

void host_free(void* p) {
  if (!p) return;
  State& s = st();
  std::lock_guard<std::mutex> lk(s.mu);
  auto it = s.host_live.find(p);
  if (it == s.host_live.end()) return;
  const size_t cls = it->second;
  s.host_live.erase(it);
  if (!s.enabled) {
    cudaFreeHost(p);
    return;
  }
  s.host_free.insert({cls, p});
  s.cached_host += cls;
}

}  // namespace tls

extern "C" {

void tls_set_allocator(tls_alloc_fn alloc, tls_free_fn release, void* user) {
  State& s = st();
  std::lock_guard<std::mutex> lk(s.mu);
  s.alloc = alloc;
  s.release = release;
  s.user = user;
}

void tls_pool_enable(int on) {
  State& s = st();
  std::lock_guard<std::mutex> lk(s.mu);
  s.enabled = on != 0;
  if (!s.enabled) trim_all_locked(s);
}

uint64_t tls_pool_trim(void) {
  State& s = st();
  std::lock_guard<std::mutex> lk(s.mu);
  return trim_all_locked(s);
}

void tls_pool_stats(uint64_t* cached_device, uint64_t* cached_host, uint64_t* live_device) {
  State& s = st();
  std::lock_guard<std::mutex> lk(s.mu);
  if (cached_device) *cached_device = s.cached_dev;
  if (cached_host) *cached_host = s.cached_host;
  if (live_device) *live_device = s.live_dev;
}

void tls_pool_poison(int value) {
  State& s = st();
  std::lock_guard<std::mutex> lk(s.mu);
  s.poison = value < 0 ? -1 : (value & 0xFF);
}

}  // extern "C"
