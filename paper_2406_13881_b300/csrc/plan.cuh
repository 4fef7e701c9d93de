// plan.cuh -- the device-side view of one ingested CFG (internal).
#pragma once
#include <cstdint>

#include "common.cuh"

namespace ompdart {

// Plain struct of device pointers, passed by value to every kernel.
// Planes are row-major [rows][W] uint64, rows indexed by block id unless
// stated otherwise.
struct DevPlan {
  int N, M, E, A, W, V, L, K, X, entry;
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
  // accesses
  const int32_t *acc_off;  // [N+1]
  const uint32_t *acc;     // [A]
  uint32_t *rec;           // [A] local summary records
  // loops
  const int32_t *loop_head;  // [L]
  const int32_t *body_off;   // [L+1]
  const int32_t *body_blk;   // blocks of each body, ascending position
  const int32_t *ent_loop;   // [K]
  const int32_t *ent_src;    // [K]
  // boundary conditions [W]
  const uint64_t *entry_h, *entry_d, *exit_live, *top;
  // state planes [N*W]
  uint64_t *h_in, *d_in, *h_out, *d_out;
  uint64_t *hp_out, *live;
  uint64_t *ant_h, *ant_d;
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
};

}  // namespace ompdart
