// classify.cu -- directive classification and consolidation (Table II;
// Sec. IV-D data region; Sec. IV-F one directive per insertion point), run
// after the emission when the data-region mode is on.
//
// From the per-access flags, the transfers the emission left on the data
// region's boundary edges and the exit sets:
//   k_cls_writes  which variables each kernel writes on the host / device;
//   k_cls_access  one thread per access: the variables each kernel touches
//                 on the device; a `to' (`from') flagged inside kernel k is
//                 made right before k (no host code runs in a kernel) unless
//                 k writes the variable on the host (device); any other
//                 flagged transfer gets its consolidated insertion point --
//                 just after the previous access of the same variable in
//                 its block, or the block's first access (a call is a
//                 barrier and keeps its own point);
//   k_cls_bounds  one thread per (CFG, word): map(to:) = `to's on every edge
//                 into the region (the region does not start at the CFG's
//                 entry) and the lifted `to's of the kernel whose entry
//                 edges are the region's; map(from:) = `from's on every edge
//                 leaving it and at every exit inside it; map(alloc:) = what
//                 a kernel touches on the device with neither.
#include <cuda_runtime.h>

#include "common.cuh"
#include "solver.h"

namespace ompdart {

namespace {

__device__ __forceinline__ void or_bit(uint64_t *row, int v) {
  atomicOr(reinterpret_cast<unsigned long long *>(row) + (v >> 6), 1ull << (v & 63));
}
// OR bit v into word w of `row' for every lane with key >= 0, one atomic per
// distinct (key, word) in the warp: many accesses of one CFG or kernel hit
// the same few words, so lanes with the same target combine their bits
// first.  Every lane of the warp must call it (inactive ones with key -1).
__device__ __forceinline__ void or_bit_warp(uint64_t *base, long long key, int v) {
  const long long target = key < 0 ? -1 : key + (v >> 6);
  const unsigned grp = __match_any_sync(0xffffffffu, target);
  if (target < 0) return;
  unsigned long long bits = 0;
  for (unsigned m = grp; m; m &= m - 1) bits |= __shfl_sync(grp, 1ull << (v & 63), __ffs(m) - 1);
  if ((threadIdx.x & 31) == __ffs(grp) - 1) atomicOr(reinterpret_cast<unsigned long long *>(base) + target, bits);
}
__device__ __forceinline__ bool has_bit(const uint64_t *row, int v) { return (row[v >> 6] >> (v & 63)) & 1ull; }

__global__ void k_cls_writes(ClsDev c) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long kh = -1, kd = -1;
  int v = 0;
  if (i < c.A) {
    const uint32_t a = c.acc[i];
    const int k = (a >> 31) ? -1 : c.kern[c.acc_blk[i]];
    if (k >= 0 && (acc_kind(a) & 2)) {
      v = acc_var(a);
      (acc_space(a) ? kd : kh) = (long long)k * c.W;
    }
  }
  or_bit_warp(c.kw_h, kh, v);
  or_bit_warp(c.kw_d, kd, v);
}

__global__ void k_cls_access(ClsDev c) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  // variables the kernels touch on the device (reachable blocks)
  {
    long long key = -1;
    int v = 0;
    if (i < c.A) {
      const int b = c.acc_blk[i];
      const uint32_t a = c.acc[i];
      if (c.pos[b] >= 0 && !(a >> 31) && c.kern[b] >= 0 && acc_space(a)) {
        key = (long long)c.blk_cfg[b] * c.W;
        v = acc_var(a);
      }
    }
    or_bit_warp(c.dev_touched, key, v);
  }
  if (i >= c.A) return;
  const int b = c.acc_blk[i];
  if (c.pos[b] < 0) {  // unreachable: no transfer
    c.acc_point[i] = -1;
    return;
  }
  const uint32_t a = c.acc[i];
  const int cfg = c.blk_cfg[b], k = c.kern[b], W = c.W;
  const bool call = (a >> 31) != 0;
  const int v = acc_var(a);
  const int f = c.acc_flag[i];
  if (!f) {
    c.acc_point[i] = -1;
    return;
  }
  if (call) {
    c.acc_point[i] = (int32_t)(i - c.acc_base[cfg]);
    return;
  }
  if (k >= 0) {
    if (f == 1 && !has_bit(c.kw_h + (size_t)k * W, v)) {
      or_bit(c.kernel_to + (size_t)k * W, v);
      c.acc_point[i] = -1;
      return;
    }
    if (f == 2 && !has_bit(c.kw_d + (size_t)k * W, v)) {
      or_bit(c.kernel_from + (size_t)k * W, v);
      c.acc_point[i] = -1;
      return;
    }
  }
  long long j = i;
  const int lo = c.acc_off[b];
  while (j > lo) {
    const uint32_t x = c.acc[j - 1];
    if ((x >> 31) || acc_var(x) == v) break;
    --j;
  }
  c.acc_point[i] = (int32_t)(j - c.acc_base[cfg]);
}

__global__ void k_cls_bounds(ClsDev c) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)c.n_cfg * c.W) return;
  const int cfg = (int)(t / c.W), w = (int)(t % c.W), W = c.W;
  uint64_t mt = 0, mf = 0;
  if (c.has_r[cfg]) {
    const int r0 = c.rin_off[cfg], r1 = c.rin_off[cfg + 1];
    if (r1 > r0 && !c.entry_in_r[cfg]) {
      uint64_t u = ~0ull;
      for (int r = r0; r < r1; ++r) u &= c.bnd_to[(size_t)r * W + w];
      mt = u;
    }
    const int sk = c.start_k[cfg];
    if (sk >= 0) {
      mt |= c.kernel_to[(size_t)sk * W + w];
      c.kernel_to[(size_t)sk * W + w] = 0;
    }
    const int x0 = c.rout_off[cfg], x1 = c.rout_off[cfg + 1], e0 = c.xin_off[cfg], e1 = c.xin_off[cfg + 1];
    if (x1 > x0 || e1 > e0) {
      uint64_t u = ~0ull;
      for (int r = x0; r < x1; ++r) u &= c.bnd_from[(size_t)(c.n_rin + r) * W + w];
      for (int e = e0; e < e1; ++e) u &= c.from_exit[(size_t)c.xin[e] * W + w];
      mf = u;
    }
  }
  c.map_to[t] = mt;
  c.map_from[t] = mf;
  c.map_alloc[t] = c.has_r[cfg] ? c.dev_touched[t] & ~mt & ~mf : 0ull;
}

inline int grid1(long long n, int b) {
  long long g = (n + b - 1) / b;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

int enqueue_classify(const ClsDev &c, cudaStream_t s, Prof *pf) {
  int n = 0;
  if (pf) pf->mark(s, "classify");
  if (c.n_k) {
    cudaMemsetAsync(c.kw_h, 0, sizeof(uint64_t) * (size_t)c.n_k * c.W, s);
    cudaMemsetAsync(c.kw_d, 0, sizeof(uint64_t) * (size_t)c.n_k * c.W, s);
    cudaMemsetAsync(c.kernel_to, 0, sizeof(uint64_t) * (size_t)c.n_k * c.W, s);
    cudaMemsetAsync(c.kernel_from, 0, sizeof(uint64_t) * (size_t)c.n_k * c.W, s);
  }
  cudaMemsetAsync(c.dev_touched, 0, sizeof(uint64_t) * (size_t)c.n_cfg * c.W, s);
  if (c.A) {
    k_cls_writes<<<grid1(c.A, 256), 256, 0, s>>>(c); ++n;
    k_cls_access<<<grid1(c.A, 256), 256, 0, s>>>(c); ++n;
  }
  k_cls_bounds<<<grid1((long long)c.n_cfg * c.W, 128), 128, 0, s>>>(c); ++n;
  return n;
}

}  // namespace ompdart
