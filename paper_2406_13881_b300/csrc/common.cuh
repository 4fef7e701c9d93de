// common.cuh -- device-side definitions shared by the libompdart kernels.
#pragma once
#include <cstdint>

namespace ompdart {

// ---- packed access words (input format, ompdart.h) ------------------------
__host__ __device__ inline int acc_var(uint32_t a) { return (int)(a & 0xFFFFFFu); }
__host__ __device__ inline int acc_kind(uint32_t a) { return (int)((a >> 24) & 3u); }
__host__ __device__ inline int acc_space(uint32_t a) { return (int)((a >> 26) & 1u); }
__host__ __device__ inline bool acc_is_call(uint32_t a) { return (a >> 31) != 0u; }

// ---- local summary records ---------------------------------------------------
// One record per (block, variable touched): the net effect of the block's
// accesses on that variable (Sec. IV-D validity rules), written at the slot
// of the variable's first access in the block; other slots hold REC_NONE.
//   bits 0-23 variable
//   bit 24 GH  host copy valid at block exit whatever it was at entry
//   bit 25 KH  host copy stale at block exit whatever it was at entry
//   bit 26 GD  device copy valid at exit
//   bit 27 KD  device copy stale at exit
//   bit 28 UH  a host read sees the value from before the block
//   bit 29 UD  a device read sees the value from before the block
//   bit 30 DF  the block writes the variable
constexpr uint32_t REC_NONE = 0xFFFFFFFFu;
constexpr uint32_t R_GH = 1u << 24, R_KH = 1u << 25, R_GD = 1u << 26, R_KD = 1u << 27;
constexpr uint32_t R_UH = 1u << 28, R_UD = 1u << 29, R_DF = 1u << 30;

// Summary record of access i of a block with accesses acc[a0, a1): if i is
// the block's first access to its variable, the variable's net effect on
// the host and device copies, whether a host/device read sees the value
// from before the block, and whether the block writes it (Sec. IV-D);
// REC_NONE for later accesses to the same variable.
__device__ inline void summarize_one(const uint32_t *acc, uint32_t *rec, int a0, int a1, int i) {
  const int v = acc_var(acc[i]);
  for (int j = a0; j < i; ++j)
    if (acc_var(acc[j]) == v) {
      rec[i] = REC_NONE;
      return;
    }
  // the last event touching each copy (1 made valid, 2 made stale); the
  // ordinal of the first read per space and of the first write
  int last_h = 0, last_d = 0;
  int first_rh = 0, first_rd = 0, first_w = 0, t = 0;
  for (int j = i; j < a1; ++j) {
    const uint32_t a = acc[j];
    if (acc_var(a) != v) continue;
    const int kind = acc_kind(a), dev = acc_space(a);
    if (kind & 1) {  // read: it gets a valid copy in its space
      ++t;
      if (dev) { last_d = 1; if (!first_rd) first_rd = t; }
      else     { last_h = 1; if (!first_rh) first_rh = t; }
    }
    if (kind & 2) {  // write: own copy valid, the other stale
      ++t;
      if (dev) { last_d = 1; last_h = 2; } else { last_h = 1; last_d = 2; }
      if (!first_w) first_w = t;
    }
  }
  uint32_t r = (uint32_t)v;
  if (last_h == 1) r |= R_GH;
  if (last_h == 2) r |= R_KH;
  if (last_d == 1) r |= R_GD;
  if (last_d == 2) r |= R_KD;
  if (first_rh && (!first_w || first_rh < first_w)) r |= R_UH;
  if (first_rd && (!first_w || first_rd < first_w)) r |= R_UD;
  if (first_w) r |= R_DF;
  rec[i] = r;
}

// the same for all accesses of one block, one warp (lane j takes j, j+32, ...)
__device__ inline void summarize_block(const uint32_t *acc, uint32_t *rec, int a0, int a1, int lane) {
  for (int i = a0 + lane; i < a1; i += 32) summarize_one(acc, rec, a0, a1, i);
}

// ---- device status words -------------------------------------------------------
enum StatusSlot { ST_ERROR = 0, ST_SWEEPS = 1, ST_NREC = 2, ST_OVERFLOW = 3, ST_COUNT = 8 };
constexpr int ERR_NOCONVERGE = 1;

struct EdgeXfer {
  int32_t edge, word;
  uint64_t to_bits, from_bits;
};

}  // namespace ompdart
