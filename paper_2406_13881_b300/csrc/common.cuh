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

// ---- device status words -------------------------------------------------------
enum StatusSlot { ST_ERROR = 0, ST_SWEEPS = 1, ST_NREC = 2, ST_OVERFLOW = 3, ST_COUNT = 8 };
constexpr int ERR_NOCONVERGE = 1;

struct EdgeXfer {
  int32_t edge, word;
  uint64_t to_bits, from_bits;
};

}  // namespace ompdart
