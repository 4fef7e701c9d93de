// plan.cuh -- the device-side view of one ingested CFG (internal).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

namespace ompdart {

// Device memory of plans comes from the stream-ordered allocator (the
// device's default memory pool, allocations and frees ordered on the
// calling thread's default stream): freeing a finished plan does not
// synchronise the device, so other plans' kernels keep running.  Callers
// synchronise cudaStreamPerThread before another stream touches new
// memory, and free only memory no stream still uses.
void pool_setup();  // once per process: keep freed pool memory for reuse
inline void *dev_malloc(size_t bytes) {
  pool_setup();
  void *p = nullptr;
  if (cudaMallocAsync(&p, bytes ? bytes : 1, cudaStreamPerThread) != cudaSuccess) return nullptr;
  return p;
}
inline void dev_free(void *p) {
  if (p) cudaFreeAsync(p, cudaStreamPerThread);
}

// Plain struct of device pointers, passed by value to every kernel.
// Planes are row-major [rows][W] uint64, rows indexed by block id unless
// stated otherwise.
struct DevPlan {
  int N, M, E, A, W, V, L, K, X, entry;
  int n_cfg;  // CFGs in this plan (a batch); boundary rows below are per CFG
  int max_sweeps;
  // traversal order (reachable blocks only)
  const int32_t *order;    // [M] block at position
  const int32_t *pos;      // [N] position or -1
  const int32_t *fin_off;  // [M+1] in-edges of each position
  const int32_t *fin_src;  // source block
  const int32_t *fin_eid;  // edge id
  const int32_t *fin_ent;  // loop-entry edge index or -1
  const int32_t *fin_dst;  // target block (= order[position])
  const int32_t *out_off;  // [M+1] out-edges of each position
  const int32_t *out_dst;  // target block
  const uint8_t *is_exit;  // [M]
  const int32_t *exit_blocks;  // [X]
  const int32_t *unreach;      // [N - M] blocks not reachable from the entry
  const int32_t *unreach_cfg;  // [N - M] CFG of each (a batch), or null: CFG 0
  int n_unreach;
  // accesses
  const int32_t *acc_off;  // [N+1]
  const uint32_t *acc;     // [A]
  uint32_t *rec;           // [A] local summary records
  // loops
  const int32_t *loop_head;  // [L]
  const int32_t *body_off;   // [L+1]
  const int32_t *body_blk;   // blocks of each body, ascending position
  const int32_t *ent_loop;   // [K] loop of a loop-entry edge, -1 for a region-exit-only edge
  const int32_t *ent_src;    // [K]
  const uint8_t *ent_rx;     // [K] the edge leaves the data region, or null (no region)
  const int32_t *ent_dst;    // [K] target block
  // data region: boundary row of each in-edge (fin index) or -1, and the
  // transfers the emission leaves on those edges ([rows][W]); null without
  const int32_t *fin_bnd;
  uint64_t *bnd_to, *bnd_from;
  // boundary conditions and valid-variable masks, [n_cfg][W] each
  const uint64_t *entry_h, *entry_d, *exit_live, *top;
  // state planes [N*W]
  uint64_t *h_in, *d_in, *h_out, *d_out;
  uint64_t *hp_out, *live;
  uint64_t *ant_h, *ant_d;
  // eager `to' placement (sweep solver): AntDm at block entry, or null
  uint64_t *ant_dm;
  // loop planes [L*W], loop-entry edge constants [K*W]
  uint64_t *mask_h, *mask_d;
  uint64_t *ec_h, *ec_d;
  uint64_t *lant;  // scratch [body_blk.size()*W*2] (sweep solver)
  // outputs
  uint8_t *acc_flag;       // [A]
  EdgeXfer *xfer;          // [xfer_cap]
  int xfer_cap;
  uint64_t *from_exit;     // [X*W]
  int32_t *status;         // [ST_COUNT]
  // call sites (Sec. IV-C), in access order; call blocks: reachable blocks
  // holding at least one call pseudo-access
  int n_sites, n_cblk;
  const uint64_t *calls;        // [rows][7][W] call table
  const int32_t *site_acc;      // [n_sites] access index
  const int32_t *cblk;          // [n_cblk] block
  const int32_t *cblk_site0;    // [n_cblk] its first call site
  const int32_t *cblk_rowbase;  // [n_cblk] first table row of its CFG
  const int32_t *cblk_cfg;      // [n_cblk] its CFG (boundary rows)
  uint64_t *call_to, *call_from, *call_entry_h, *call_entry_d, *call_exit_live;  // [n_sites][W]
};

// Optional per-launch timing: a CUDA event is recorded on the launch stream
// before every kernel and once after the last; the time between two events
// is charged to the kernel launched between them.
struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> kid;
  std::vector<std::string> names;
  std::vector<double> ms;
  std::vector<int> cnt;
  int used = 0;
  bool collect_pending = false;
  void mark(cudaStream_t s, const char *name) {
    if (!on) return;
    if (used + 1 >= (int)ev.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      ev.push_back(e);
      cudaEventCreate(&e);
      ev.push_back(e);
    }
    int k = 0;
    while (k < (int)names.size() && names[k] != name) ++k;
    if (k == (int)names.size()) {
      names.push_back(name);
      ms.push_back(0.0);
      cnt.push_back(0);
    }
    kid.resize(used + 1);
    kid[used] = k;
    cudaEventRecord(ev[used], s);
    ++used;
  }
  void close(cudaStream_t s) {
    if (!on || !used) return;
    if (used >= (int)ev.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      ev.push_back(e);
    }
    cudaEventRecord(ev[used], s);
  }
  // after the stream finished
  void collect() {
    for (int i = 0; i < used; ++i) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ev[i], ev[i + 1]) == cudaSuccess) {
        ms[kid[i]] += t;
        cnt[kid[i]] += 1;
      }
    }
    used = 0;
  }
  ~Prof() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

}  // namespace ompdart
