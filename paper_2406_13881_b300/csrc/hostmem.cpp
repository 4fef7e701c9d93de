// Host blocks that hold the arrays of host results.
//
// A result copied to the host lives in one block: one allocation, one DMA
// target per array.  Blocks of at least kPinMin bytes are page-locked
// (device->host copies then run at link speed instead of through the
// driver's staging buffers and first-touch page faults) and, once released,
// kept in a size-keyed cache up to a byte cap, so a caller that analyses
// again reuses them without pinning new pages.  Smaller blocks are plain
// heap memory.  A block is reference counted: the results of a batch are
// views into their arena's block and the last one freed releases it.
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
  std::atomic<int> refs{1};
};

namespace {

constexpr size_t kPinMin = size_t(1) << 20;

struct Cache {
  std::mutex mu;
  std::multimap<size_t, void *> free_blocks;  // pinned, by size
  size_t cached = 0;
  size_t cap = 0;
};

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

HostBlock *host_block_new(size_t bytes) {
  HostBlock *b = new (std::nothrow) HostBlock();
  if (!b) return nullptr;
  b->bytes = bytes ? bytes : 1;
  if (b->bytes >= kPinMin) {
    Cache &c = cache();
    {
      // best fit among cached blocks no more than twice the size asked for
      std::lock_guard<std::mutex> lk(c.mu);
      auto it = c.free_blocks.lower_bound(b->bytes);
      if (it != c.free_blocks.end() && it->first <= 2 * b->bytes) {
        b->ptr = it->second;
        b->bytes = it->first;
        c.cached -= it->first;
        c.free_blocks.erase(it);
        b->pinned = true;
        return b;
      }
    }
    if (cudaHostAlloc(&b->ptr, b->bytes, cudaHostAllocPortable) == cudaSuccess) {
      b->pinned = true;
      return b;
    }
    cudaGetLastError();  // fall back to pageable memory
    b->ptr = nullptr;
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
  if (b->pinned) {
    Cache &c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    if (c.cached + b->bytes <= c.cap) {
      c.free_blocks.emplace(b->bytes, b->ptr);
      c.cached += b->bytes;
    } else {
      cudaFreeHost(b->ptr);
    }
  } else {
    std::free(b->ptr);
  }
  delete b;
}

}  // namespace ompdart

extern "C" {

size_t ompdart_host_cache_trim(void) {
  using namespace ompdart;
  Cache &c = cache();
  std::lock_guard<std::mutex> lk(c.mu);
  const size_t n = c.cached;
  for (auto &kv : c.free_blocks) cudaFreeHost(kv.second);
  c.free_blocks.clear();
  c.cached = 0;
  return n;
}

}  // extern "C"
