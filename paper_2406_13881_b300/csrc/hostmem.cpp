// Host blocks that hold the arrays of host results.
//
// A result copied to the host lives in one block: one allocation, one DMA
// target per array.  Blocks of at least kCacheMin bytes are rounded up to
// a size class and, once released, kept per class up to a byte cap, so a
// caller that analyses again (or a serving loop whose batches differ in
// size) reuses memory whose pages are already there.  Two kinds:
//   page-locked (a plan's result: one large block, copied back at link
//     speed; pinning new pages is slow, about 1 GB/s, so only reuse pays,
//     and freeing them waits for the device, so it happens past the cap);
//   pageable (batches and serving: many blocks of varying size, copied
//     through the driver's staging buffers).
// Smaller blocks are plain heap memory.  A block is reference counted: the
// results of a batch are views into their arena's block and the last one
// freed releases it.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdlib>
#include <map>
#include <mutex>

#include "solver.h"

namespace ompdart {

struct HostBlock {
  void *ptr = nullptr;
  size_t bytes = 0;
  bool pinned = false;
  bool cached = false;  // returns to the cache of its kind when released
  std::atomic<int> refs{1};
};

namespace {

constexpr size_t kCacheMin = size_t(1) << 20;

struct Cache {
  std::mutex mu;
  std::multimap<size_t, void *> free_blocks[2];  // [pageable, page-locked], by size class
  size_t cached[2] = {0, 0};
  size_t cap = 0;
};

// four classes per power of two (at most 25% over the size asked for)
size_t size_class(size_t bytes) {
  size_t p = kCacheMin;
  while (2 * p < bytes) p <<= 1;
  for (size_t m = 4; m <= 8; ++m)
    if (p / 4 * m >= bytes) return p / 4 * m;
  return 2 * p;
}

// never destroyed: releases may come from static destructors of callers
Cache &cache() {
  static Cache *c = [] {
    Cache *x = new Cache();
    size_t mb = 4096;
    if (const char *e = std::getenv("OMPDART_HOST_CACHE_MB")) mb = (size_t)std::strtoull(e, nullptr, 10);
    x->cap = mb << 20;
    return x;
  }();
  return *c;
}

}  // namespace

HostBlock *host_block_new(size_t bytes, bool pin) {
  HostBlock *b = new (std::nothrow) HostBlock();
  if (!b) return nullptr;
  b->bytes = bytes ? bytes : 1;
  // a small block is not worth page-locking: cudaHostAlloc costs far more
  // than the staged copy it saves, and it serialises concurrent callers
  if (b->bytes < kCacheMin) pin = false;
  if (b->bytes >= kCacheMin) {
    Cache &c = cache();
    b->bytes = size_class(b->bytes);
    b->cached = true;
    {
      std::lock_guard<std::mutex> lk(c.mu);
      auto &fb = c.free_blocks[pin];
      auto it = fb.find(b->bytes);
      if (it != fb.end()) {
        b->ptr = it->second;
        b->pinned = pin;
        c.cached[pin] -= it->first;
        fb.erase(it);
        return b;
      }
    }
    if (pin) {
      TraceScope trace("page-locked alloc", (long long)b->bytes);
      if (cudaHostAlloc(&b->ptr, b->bytes, cudaHostAllocPortable) == cudaSuccess) {
        b->pinned = true;
        return b;
      }
      cudaGetLastError();  // fall back to pageable memory
      b->ptr = nullptr;
    }
  }
  b->ptr = std::malloc(b->bytes);
  if (!b->ptr) {
    delete b;
    return nullptr;
  }
  return b;
}

void *host_block_ptr(HostBlock *b) { return b ? b->ptr : nullptr; }

void host_block_ref(HostBlock *b) {
  if (b) b->refs.fetch_add(1, std::memory_order_relaxed);
}

void host_block_release(HostBlock *b) {
  if (!b || b->refs.fetch_sub(1, std::memory_order_acq_rel) != 1) return;
  bool keep = false;
  if (b->cached) {
    Cache &c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    if (c.cached[b->pinned] + b->bytes <= c.cap) {
      c.free_blocks[b->pinned].emplace(b->bytes, b->ptr);
      c.cached[b->pinned] += b->bytes;
      keep = true;
    }
  }
  if (!keep) {
    if (b->pinned) {
      TraceScope trace("page-locked free", (long long)b->bytes);
      cudaFreeHost(b->ptr);
    } else {
      std::free(b->ptr);
    }
  }
  delete b;
}

}  // namespace ompdart

extern "C" {

size_t ompdart_host_cache_trim(void) {
  using namespace ompdart;
  Cache &c = cache();
  std::lock_guard<std::mutex> lk(c.mu);
  const size_t n = c.cached[0] + c.cached[1];
  for (auto &kv : c.free_blocks[0]) std::free(kv.second);
  for (auto &kv : c.free_blocks[1]) cudaFreeHost(kv.second);
  for (int k = 0; k < 2; ++k) {
    c.free_blocks[k].clear();
    c.cached[k] = 0;
  }
  return n;
}

}  // extern "C"
