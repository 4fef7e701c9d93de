// noalloc.cu -- liveness of one CFG without any memory allocation.
//
// Some callers cannot allocate device memory: code that runs while another
// runtime owns the device allocator (an application's own memory pool, a
// framework that forbids cudaMalloc inside its step), or code that must not
// synchronise the device the way cudaMalloc/cudaFree can.  This file gives
// them ompdart_liveness_noalloc: the caller passes its CFG and the output
// plane already in device memory, and every scratch byte the kernel needs
// lives in one file-scope static device array (NOALLOC_SCRATCH_WORDS words,
// 4.5 MiB, resident on every device that loads the library until the
// process exits).
//
// The host code may not hand the array's name to a kernel (on the host it
// is only a stand-in for the symbol): with the device current, the entry
// point asks cudaGetSymbolAddress for the device address and keeps it once
// the lookup has succeeded (a failed lookup is tried again by the next
// call).  That lookup happens on the first call on each device, which
// should therefore come before any stream capture.  Every call waits for
// `stream' before it returns.  Every call shares the array: calls whose
// kernels overlap on the GPU race and must be ordered by the caller (one
// stream, or events).
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/ompdart.h"
#include "common.cuh"

namespace ompdart {
void set_last_error_text(const std::string &msg);  // api.cu

namespace {

constexpr int NA_MAX_BLOCKS = 65536;
constexpr int NA_MAX_WORDS = 64;          // 4096 variables
constexpr int NA_MAX_ACC = 1 << 20;       // accesses
constexpr int NA_STATUS_WORDS = 32;
// layout (uint64 words): [status 32][reach flags, int32 per block]
// [breadth-first order, int32 per block][summary records, uint32 per access]
constexpr size_t NA_REACH_WORDS = NA_MAX_BLOCKS / 2;
constexpr size_t NA_ORDER_WORDS = NA_MAX_BLOCKS / 2;
constexpr size_t NA_REC_WORDS = NA_MAX_ACC / 2;
constexpr size_t NOALLOC_SCRATCH_WORDS = NA_STATUS_WORDS + NA_REACH_WORDS + NA_ORDER_WORDS + NA_REC_WORDS;
// device time a call may take before it gives up (OMPDART_E_TIMEOUT);
// valid inputs within the limits above finish in well under a second
constexpr unsigned long long NA_TIME_LIMIT_NS = 20ull * 1000 * 1000 * 1000;

static __device__ __align__(256) uint64_t g_noalloc_scratch[NOALLOC_SCRATCH_WORDS];

enum { NA_OK = 0, NA_BAD_CSR = 1, NA_TOO_MANY_ACC = 2, NA_NOCONVERGE = 3, NA_TIMEOUT = 4 };

__device__ __forceinline__ unsigned long long na_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// One CTA does everything (the sizes are bounded), with block-wide
// barriers between the steps:
//   1. validate the CSR offsets and ids, clear the reach flags and output
//   2. summary records of every block (one warp per block)
//   3. breadth-first search from the entry, level by level: the blocks
//      reachable from the entry in order of their distance from it
//   4. liveness, one thread per 64-variable word, Gauss-Seidel sweeps over
//      the reachable blocks farthest first (a block after the successors it
//      reaches by tree edges, so a chain settles in one sweep), until
//      nothing changes (<= n + 2 sweeps):
//        Live_in[b] = UE[b] | (Live_out[b] & ~Def[b]),
//        Live_out[b] = OR of the successors' Live_in, or exit_host_live;
//      UE = a read in either space before any write (Sec. II-B liveness,
//      Sec. IV-D region-exit liveness); unreachable blocks stay zero.
// Steps 3 and 4 stop with NA_TIMEOUT once the call has run for
// NA_TIME_LIMIT_NS of device time.
__global__ void __launch_bounds__(1024) k_live_noalloc(int n, int nv, int entry, const int32_t *so,
                                                       const int32_t *su, const int32_t *ao, const uint32_t *acc,
                                                       const uint64_t *xl, uint64_t *live, uint64_t *scratch) {
  int32_t *status = reinterpret_cast<int32_t *>(scratch);
  int32_t *reach = reinterpret_cast<int32_t *>(scratch + NA_STATUS_WORDS);
  int32_t *order = reinterpret_cast<int32_t *>(scratch + NA_STATUS_WORDS + NA_REACH_WORDS);
  uint32_t *rec = reinterpret_cast<uint32_t *>(scratch + NA_STATUS_WORDS + NA_REACH_WORDS + NA_ORDER_WORDS);
  __shared__ int bad, tail, stop;
  const int t = threadIdx.x, T = blockDim.x, lane = t & 31, warp = t >> 5, nwarp = T >> 5;
  const int W = (nv + 63) / 64;
  const unsigned long long t0 = na_now();
  if (t == 0) {
    bad = NA_OK;
    stop = 0;
  }
  __syncthreads();
  // ---- 1. validation and clearing
  const int E = so[n], A = ao[n];
  if (so[0] != 0 || ao[0] != 0 || E < 0 || A < 0) bad = NA_BAD_CSR;
  if (A > NA_MAX_ACC) bad = NA_TOO_MANY_ACC;
  for (int b = t; b < n; b += T) {
    if (so[b + 1] < so[b] || ao[b + 1] < ao[b] || so[b + 1] > E || ao[b + 1] > A) bad = NA_BAD_CSR;
    reach[b] = 0;
  }
  __syncthreads();
  if (bad == NA_OK) {
    for (int e = t; e < E; e += T)
      if (su[e] < 0 || su[e] >= n || su[e] == entry) bad = NA_BAD_CSR;
    for (int i = t; i < A; i += T) {
      const uint32_t a = acc[i];
      if ((a >> 27) || acc_var(a) >= nv || acc_kind(a) == 0) bad = NA_BAD_CSR;
    }
  }
  for (long long i = t; i < (long long)n * W; i += T) live[i] = 0;
  __syncthreads();
  if (bad != NA_OK) {
    if (t == 0) status[0] = bad;
    return;
  }
  // ---- 2. summary records
  for (int b = warp; b < n; b += nwarp) summarize_block(acc, rec, ao[b], ao[b + 1], lane);
  // ---- 3. breadth-first order of the reachable blocks (each block enters
  // the order once: the thread that flips its flag appends it)
  if (t == 0) {
    reach[entry] = 1;
    order[0] = entry;
    tail = 1;
  }
  __syncthreads();
  int head = 0;
  while (true) {
    const int hi = tail;  // this level: order[head, hi)
    __syncthreads();      // every thread has read the level's end before any appends
    if (head == hi) break;
    for (int i = head + t; i < hi; i += T) {
      const int b = order[i];
      for (int e = so[b]; e < so[b + 1]; ++e) {
        const int s = su[e];
        if (atomicCAS(&reach[s], 0, 1) == 0) order[atomicAdd(&tail, 1)] = s;
      }
    }
    if (t == 0 && na_now() - t0 > NA_TIME_LIMIT_NS) stop = 1;
    __syncthreads();
    if (stop) break;
    head = hi;
  }
  const int nr = tail;  // reachable blocks
  __syncthreads();
  if (stop) {
    if (t == 0) status[0] = NA_TIMEOUT;
    return;
  }
  // ---- 4. liveness, one thread per word, farthest blocks first
  int result = NA_OK;
  if (t < W) {
    const int w = t;
    const uint64_t top = (w == W - 1 && nv % 64) ? ((1ull << (nv % 64)) - 1) : ~0ull;
    const uint64_t x = (xl ? xl[w] : ~0ull) & top;
    bool again = true;
    int sweeps = 0;
    while (again) {
      if (sweeps++ > n + 2) {
        result = NA_NOCONVERGE;
        break;
      }
      if (na_now() - t0 > NA_TIME_LIMIT_NS) {
        result = NA_TIMEOUT;
        break;
      }
      again = false;
      for (int k = nr - 1; k >= 0; --k) {
        const int b = order[k];
        uint64_t z = so[b] == so[b + 1] ? x : 0;
        for (int e = so[b]; e < so[b + 1]; ++e) z |= live[(size_t)su[e] * W + w];
        for (int r = ao[b]; r < ao[b + 1]; ++r) {
          const uint32_t rc = rec[r];
          if (rc == REC_NONE || (acc_var(rc) >> 6) != w) continue;
          const uint64_t bit = 1ull << (acc_var(rc) & 63);
          if (rc & (R_UH | R_UD)) z |= bit;
          else if (rc & R_DF) z &= ~bit;
        }
        if (z != live[(size_t)b * W + w]) {
          live[(size_t)b * W + w] = z;
          again = true;
        }
      }
    }
  }
  if (result != NA_OK) atomicMax(&status[0], result);
}

// the scratch array's device address per device, once a lookup succeeded
struct DeviceSlot {
  std::mutex mu;
  uint64_t *ptr = nullptr;
};
DeviceSlot g_slots[64];

int na_fail(int code, const char *msg) {
  set_last_error_text(msg);
  return code;
}

}  // namespace

}  // namespace ompdart

using namespace ompdart;

extern "C" int ompdart_liveness_noalloc(int32_t n_blocks, int32_t n_vars, int32_t entry, const int32_t *succ_off,
                                        const int32_t *succ, const int32_t *acc_off, const uint32_t *acc,
                                        const uint64_t *exit_host_live, uint64_t *live_in, void *stream) {
  set_last_error_text("");
  if (n_blocks < 1 || n_blocks > NA_MAX_BLOCKS)
    return na_fail(OMPDART_E_BUDGET, "n_blocks must be in [1, 65536] for the no-allocation entry point");
  if (n_vars < 1 || (n_vars + 63) / 64 > NA_MAX_WORDS)
    return na_fail(OMPDART_E_BUDGET, "n_vars must be in [1, 4096] for the no-allocation entry point");
  if (entry < 0 || entry >= n_blocks) return na_fail(OMPDART_E_INVALID, "entry out of range");
  if (!succ_off || !acc_off || !live_in) return na_fail(OMPDART_E_INVALID, "NULL device pointer");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return na_fail(OMPDART_E_CUDA, "cudaGetDevice failed");
  DeviceSlot &slot = g_slots[dev];
  uint64_t *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(slot.mu);
    if (!slot.ptr) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();  // not sticky: the next call tries again
        return na_fail(OMPDART_E_CUDA, "cudaGetSymbolAddress of the scratch failed");
      }
      slot.ptr = static_cast<uint64_t *>(p);
    }
    scratch = slot.ptr;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // status words start at zero for every call
  if (cudaMemsetAsync(scratch, 0, NA_STATUS_WORDS * sizeof(uint64_t), s) != cudaSuccess)
    return na_fail(OMPDART_E_CUDA, "clearing the status words failed");
  k_live_noalloc<<<1, 1024, 0, s>>>(n_blocks, n_vars, entry, succ_off, succ, acc_off, acc, exit_host_live, live_in,
                                    scratch);
  if (cudaGetLastError() != cudaSuccess) return na_fail(OMPDART_E_CUDA, "kernel launch failed");
  int32_t st = 0;
  if (cudaMemcpyAsync(&st, scratch, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return na_fail(OMPDART_E_CUDA, "device run failed");
  switch (st) {
    case NA_OK: return OMPDART_OK;
    case NA_BAD_CSR: return na_fail(OMPDART_E_INVALID, "malformed CSR, id out of range or entry with predecessors");
    case NA_TOO_MANY_ACC: return na_fail(OMPDART_E_BUDGET, "more than 2^20 accesses for the no-allocation entry point");
    case NA_TIMEOUT: return na_fail(OMPDART_E_TIMEOUT, "the no-allocation liveness ran past its device time limit");
    default: return na_fail(OMPDART_E_NOCONVERGE, "liveness sweeps did not converge");
  }
}
