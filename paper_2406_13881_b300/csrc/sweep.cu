// sweep.cu -- local summaries and the general sweep solver.
//
// The sweep solver accepts any CFG (irreducible ones included): every phase
// repeats Gauss-Seidel sweeps in the loop-ordered reverse post-order until
// nothing changes, bounded by max_sweeps.  Each thread owns one 64-variable
// word column for the whole graph (variables are independent bit-vector
// problems; the host/device coupling is per variable, so per word).  It is
// the fallback for CFGs the chunked scan solver cannot take and the
// cross-check for it; the scan solver is the fast path.
#include "plan.cuh"

namespace ompdart {

// ---- local summary (Sec. IV-D validity rules per block) ---------------------
// One warp per block (see summarize_block).
__global__ void k_local_summary(DevPlan p) {
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < p.N; b += nwarps)
    summarize_block(p.acc, p.rec, p.acc_off[b], p.acc_off[b + 1], lane);
}

// fill every row of a plane with `top` (all variables set, padding clear)
__global__ void k_fill_top(uint64_t *plane, int rows, int W, const uint64_t *top) {
  const long long n = (long long)rows * W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    plane[i] = top[i % W];
}

// rows of blocks unreachable from the entry: every state plane all-ones,
// liveness zero
__global__ void k_fill_unreachable(DevPlan p, int keep_states) {
  const long long n = (long long)p.n_unreach * p.W;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const int w = (int)(t % p.W);
    const long long u = t / p.W;
    const size_t o = (size_t)p.unreach[u] * p.W + w;
    const uint64_t top = p.top[(size_t)(p.unreach_cfg ? p.unreach_cfg[u] : 0) * p.W + w];
    p.h_in[o] = top;
    p.d_in[o] = top;
    p.live[o] = 0;
    if (keep_states) {
      p.h_out[o] = top;
      p.d_out[o] = top;
    }
  }
}

// ---- backward anticipation (Sec. II-B liveness, Sec. IV-D region exit) -------
// AntS_in[b] = UES[b] | (AntS_out[b] & ~Def[b]); AntS_out[b] = OR of the
// successors' AntS_in, or the region-exit value (host: exit_host_live,
// device: nothing) for a block without successors.  Least fixed point over
// reachable blocks; Live = AntH | AntD.
__global__ void k_sweep_ant(DevPlan p) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= p.W) return;
  const int W = p.W;
  const uint64_t xl = p.exit_live[w];
  int sweeps = 0;
  bool changed = true;
  while (changed) {
    if (sweeps >= p.max_sweeps) { atomicExch(&p.status[ST_ERROR], ERR_NOCONVERGE); break; }
    changed = false;
    ++sweeps;
    for (int i = p.M - 1; i >= 0; --i) {
      const int b = p.order[i];
      uint64_t oh = p.is_exit[i] ? xl : 0, od = 0;
      for (int k = p.out_off[i]; k < p.out_off[i + 1]; ++k) {
        const int s = p.out_dst[k];
        oh |= p.ant_h[(size_t)s * W + w];
        od |= p.ant_d[(size_t)s * W + w];
      }
      for (int r = p.acc_off[b]; r < p.acc_off[b + 1]; ++r) {
        const uint32_t rc = p.rec[r];
        if (rc == REC_NONE || (acc_var(rc) >> 6) != w) continue;
        const uint64_t bit = 1ull << (acc_var(rc) & 63);
        if (rc & R_UH) oh |= bit; else if (rc & R_DF) oh &= ~bit;
        if (rc & R_UD) od |= bit; else if (rc & R_DF) od &= ~bit;
      }
      const size_t o = (size_t)b * W + w;
      if (oh != p.ant_h[o] || od != p.ant_d[o]) { p.ant_h[o] = oh; p.ant_d[o] = od; changed = true; }
    }
  }
  atomicMax(&p.status[ST_SWEEPS], sweeps);
  for (int i = 0; i < p.M; ++i) {
    const size_t o = (size_t)p.order[i] * W + w;
    p.live[o] = p.ant_h[o] | p.ant_d[o];
  }
}

// ---- eager `to': must-anticipation of device reads (Sec. IV-E) --------------------
// AntDm_in[b] = UED[b] | (AntDm_out[b] & ~Def[b]); AntDm_out[b] = AND of the
// successors' AntDm_in, nothing for a block without successors.  Greatest
// fixed point from all ones: v is in it where every path reads v on the
// device before any write of v.
__global__ void k_sweep_antm(DevPlan p) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= p.W) return;
  const int W = p.W;
  const uint64_t top = p.top[w];
  for (int i = 0; i < p.M; ++i) p.ant_dm[(size_t)p.order[i] * W + w] = top;
  int sweeps = 0;
  bool changed = true;
  while (changed) {
    if (sweeps >= p.max_sweeps) { atomicExch(&p.status[ST_ERROR], ERR_NOCONVERGE); break; }
    changed = false;
    ++sweeps;
    for (int i = p.M - 1; i >= 0; --i) {
      const int b = p.order[i];
      uint64_t x = p.out_off[i] == p.out_off[i + 1] ? 0ull : top;
      for (int k = p.out_off[i]; k < p.out_off[i + 1]; ++k) x &= p.ant_dm[(size_t)p.out_dst[k] * W + w];
      for (int r = p.acc_off[b]; r < p.acc_off[b + 1]; ++r) {
        const uint32_t rc = p.rec[r];
        if (rc == REC_NONE || (acc_var(rc) >> 6) != w) continue;
        const uint64_t bit = 1ull << (acc_var(rc) & 63);
        if (rc & R_UD) x |= bit; else if (rc & R_DF) x &= ~bit;
      }
      const size_t o = (size_t)b * W + w;
      if (x != p.ant_dm[o]) { p.ant_dm[o] = x; changed = true; }
    }
  }
  atomicMax(&p.status[ST_SWEEPS], sweeps);
}

// ---- forward must problems (Sec. IV-D) -------------------------------------------
// PH_HP: plain host validity (host access -> valid, device write -> stale)
// PH_D : device validity; loop-entry edges add the hoisted `to' set; with
//        eager placement every edge p->b adds AntDm_in[b] & Hp_out[p] (what
//        every path on reads on the device first, from the latest host copy)
// PH_H : host validity; loop-entry edges add the hoisted `from' set, and a
//        live variable valid in neither space after the join is resolved
//        toward the host (a `from' on the disagreeing in-edges).
enum Phase { PH_HP = 0, PH_D = 1, PH_H = 2 };

template <int PH>
__global__ void k_sweep_fwd(DevPlan p) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= p.W) return;
  const int W = p.W;
  const uint32_t GEN = PH == PH_D ? R_GD : R_GH, KILL = PH == PH_D ? R_KD : R_KH;
  uint64_t *out = PH == PH_HP ? p.hp_out : PH == PH_D ? p.d_out : p.h_out;
  uint64_t *in = PH == PH_HP ? nullptr : PH == PH_D ? p.d_in : p.h_in;
  const uint64_t *ec = PH == PH_D ? p.ec_d : p.ec_h;
  const uint64_t init = (PH == PH_D ? p.entry_d[w] : p.entry_h[w]) & p.top[w];
  const uint64_t top = p.top[w];
  int sweeps = 0;
  bool changed = true;
  while (changed) {
    if (sweeps >= p.max_sweeps) { atomicExch(&p.status[ST_ERROR], ERR_NOCONVERGE); break; }
    changed = false;
    ++sweeps;
    for (int i = 0; i < p.M; ++i) {
      const int b = p.order[i];
      uint64_t x;
      if (b == p.entry) {
        x = init;
      } else {
        x = top;
        for (int k = p.fin_off[i]; k < p.fin_off[i + 1]; ++k) {
          uint64_t v = out[(size_t)p.fin_src[k] * W + w];
          if (PH != PH_HP && p.fin_ent[k] >= 0) v |= ec[(size_t)p.fin_ent[k] * W + w];
          if (PH == PH_D && p.ant_dm) v |= p.ant_dm[(size_t)b * W + w] & p.hp_out[(size_t)p.fin_src[k] * W + w];
          x &= v;
        }
      }
      const size_t o = (size_t)b * W + w;
      if (PH == PH_H) x |= p.live[o] & ~p.d_in[o];
      if (in) in[o] = x;
      for (int r = p.acc_off[b]; r < p.acc_off[b + 1]; ++r) {
        const uint32_t rc = p.rec[r];
        if (rc == REC_NONE || (acc_var(rc) >> 6) != w) continue;
        const uint64_t bit = 1ull << (acc_var(rc) & 63);
        if (rc & GEN) x |= bit; else if (rc & KILL) x &= ~bit;
      }
      if (x != out[o]) { out[o] = x; changed = true; }
    }
  }
  atomicMax(&p.status[ST_SWEEPS], sweeps);
}

// ---- loop masks (Sec. IV-D loop rule, Algorithm 1) ---------------------------------
// One thread per (loop, word).  LantS = what a node of the loop reads in S
// before any write, on a path from the header inside the body during one
// iteration (edges back to the header and out of the body dropped);
// MaskS = LantS & ~(OR of KillS over the body).
__device__ int body_index(const DevPlan &p, int lo, int hi, int blk) {
  const int key = p.pos[blk];
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int pm = p.pos[p.body_blk[mid]];
    if (pm == key) return mid;
    if (pm < key) lo = mid + 1; else hi = mid;
  }
  return -1;
}

__global__ void k_sweep_masks(DevPlan p) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)p.L * p.W) return;
  const int l = (int)(t / p.W), w = (int)(t % p.W), W = p.W;
  const int b0 = p.body_off[l], b1 = p.body_off[l + 1], head = p.loop_head[l];
  uint64_t koh = 0, kod = 0;
  for (int j = b0; j < b1; ++j) {
    const int b = p.body_blk[j];
    for (int r = p.acc_off[b]; r < p.acc_off[b + 1]; ++r) {
      const uint32_t rc = p.rec[r];
      if (rc == REC_NONE || (acc_var(rc) >> 6) != w) continue;
      const uint64_t bit = 1ull << (acc_var(rc) & 63);
      if (rc & R_KH) koh |= bit;
      if (rc & R_KD) kod |= bit;
    }
    p.lant[((size_t)j * W + w) * 2 + 0] = 0;
    p.lant[((size_t)j * W + w) * 2 + 1] = 0;
  }
  int sweeps = 0;
  bool changed = true;
  while (changed) {
    if (sweeps >= p.max_sweeps) { atomicExch(&p.status[ST_ERROR], ERR_NOCONVERGE); break; }
    changed = false;
    ++sweeps;
    for (int j = b1 - 1; j >= b0; --j) {
      const int b = p.body_blk[j], i = p.pos[b];
      uint64_t oh = 0, od = 0;
      for (int k = p.out_off[i]; k < p.out_off[i + 1]; ++k) {
        const int s = p.out_dst[k];
        if (s == head) continue;
        const int js = body_index(p, b0, b1, s);
        if (js < 0) continue;
        oh |= p.lant[((size_t)js * W + w) * 2 + 0];
        od |= p.lant[((size_t)js * W + w) * 2 + 1];
      }
      for (int r = p.acc_off[b]; r < p.acc_off[b + 1]; ++r) {
        const uint32_t rc = p.rec[r];
        if (rc == REC_NONE || (acc_var(rc) >> 6) != w) continue;
        const uint64_t bit = 1ull << (acc_var(rc) & 63);
        if (rc & R_UH) oh |= bit; else if (rc & R_DF) oh &= ~bit;
        if (rc & R_UD) od |= bit; else if (rc & R_DF) od &= ~bit;
      }
      uint64_t *lh = &p.lant[((size_t)j * W + w) * 2];
      if (oh != lh[0] || od != lh[1]) { lh[0] = oh; lh[1] = od; changed = true; }
    }
  }
  p.mask_h[(size_t)l * W + w] = p.lant[((size_t)b0 * W + w) * 2 + 0] & ~koh;
  p.mask_d[(size_t)l * W + w] = p.lant[((size_t)b0 * W + w) * 2 + 1] & ~kod;
}

// edge constants: on a loop-entry edge, device side = mask_d of the loop &
// host valid (plain) at the source, host side = mask_h & device valid at
// the source; on an edge leaving the data region the host side also holds
// what is live at its target (made valid on the host there)
template <int PH>
__global__ void k_edge_const(DevPlan p) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)p.K * p.W) return;
  const int k = (int)(t / p.W), w = (int)(t % p.W), W = p.W;
  const int l = p.ent_loop[k], src = p.ent_src[k];
  if (PH == PH_D) {
    p.ec_d[t] = l >= 0 ? p.mask_d[(size_t)l * W + w] & p.hp_out[(size_t)src * W + w] : 0ull;
  } else {
    uint64_t x = l >= 0 ? p.mask_h[(size_t)l * W + w] & p.d_out[(size_t)src * W + w] : 0ull;
    if (p.ent_rx && p.ent_rx[k]) x |= p.live[(size_t)p.ent_dst[k] * W + w];
    p.ec_h[t] = x;
  }
}

// ---- emission (Table II) ------------------------------------------------------------
// Access flags: replay each reachable block from its entry states; a read
// that finds its space stale gets `update to' (device read) or `update from'
// (host read) right before it.
__global__ void k_emit_flags(DevPlan p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.M) return;
  const int b = p.order[i], W = p.W;
  const int a0 = p.acc_off[b], a1 = p.acc_off[b + 1];
  for (int j = a0; j < a1; ++j) {
    const uint32_t a = p.acc[j];
    const int v = acc_var(a);
    const uint64_t bit = 1ull << (v & 63);
    bool h = (p.h_in[(size_t)b * W + (v >> 6)] & bit) != 0;
    bool d = (p.d_in[(size_t)b * W + (v >> 6)] & bit) != 0;
    uint8_t flag = 0;
    for (int q = a0; q <= j; ++q) {
      const uint32_t x = p.acc[q];
      if (acc_var(x) != v) continue;
      const int kind = acc_kind(x), dev = acc_space(x);
      if (kind & 1) {
        if (dev && !d) { d = true; if (q == j) flag = 1; }
        if (!dev && !h) { h = true; if (q == j) flag = 2; }
      }
      if (kind & 2) { if (dev) { d = true; h = false; } else { h = true; d = false; } }
    }
    p.acc_flag[j] = flag;
  }
}

// Edge transfers: hoisted `to'/`from' on loop-entry edges; eager `to' on
// any edge (AntDm at the target, the host copy the latest at the source,
// the device copy stale); `from' on any in-edge where a live variable valid
// in neither space after the join is not host-valid on that edge.
__global__ void k_emit_edges(DevPlan p, int n_fin) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)n_fin * p.W) return;
  const int k = (int)(t / p.W), w = (int)(t % p.W), W = p.W;
  const int src = p.fin_src[k], dst = p.fin_dst[k], ent = p.fin_ent[k];
  uint64_t hedge = p.h_out[(size_t)src * W + w], to = 0, fr = 0;
  if (p.ant_dm)
    to = p.ant_dm[(size_t)dst * W + w] & p.hp_out[(size_t)src * W + w] & ~p.d_out[(size_t)src * W + w];
  if (ent >= 0) {
    to |= p.ec_d[(size_t)ent * W + w] & ~p.d_out[(size_t)src * W + w];
    fr = p.ec_h[(size_t)ent * W + w] & ~p.h_out[(size_t)src * W + w];
    hedge |= p.ec_h[(size_t)ent * W + w];
  }
  fr |= p.live[(size_t)dst * W + w] & ~p.d_in[(size_t)dst * W + w] & ~hedge;
  if (p.fin_bnd && p.fin_bnd[k] >= 0) {  // an edge on the data region's boundary
    p.bnd_to[(size_t)p.fin_bnd[k] * W + w] = to;
    p.bnd_from[(size_t)p.fin_bnd[k] * W + w] = fr;
  }
  if (to | fr) {
    const int slot = atomicAdd(&p.status[ST_NREC], 1);
    if (slot < p.xfer_cap) p.xfer[slot] = EdgeXfer{p.fin_eid[k], w, to, fr};
  }
}

__global__ void k_emit_exit(DevPlan p) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)p.X * p.W) return;
  const int x = (int)(t / p.W), w = (int)(t % p.W);
  p.from_exit[t] = p.exit_live[w] & ~p.h_out[(size_t)p.exit_blocks[x] * p.W + w];
}

// explicit instantiations used by api.cu
template __global__ void k_sweep_fwd<PH_HP>(DevPlan);
template __global__ void k_sweep_fwd<PH_D>(DevPlan);
template __global__ void k_sweep_fwd<PH_H>(DevPlan);
template __global__ void k_edge_const<PH_D>(DevPlan);
template __global__ void k_edge_const<PH_H>(DevPlan);

}  // namespace ompdart

namespace ompdart {

static int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > (1 << 20)) g = 1 << 20;
  return (int)g;
}

// Enqueue the local summary kernel.  Returns the number of launches.
int enqueue_local_summary(const DevPlan &p, cudaStream_t s, Prof *pf) {
  const int threads = 256;
  if (pf) pf->mark(s, "local_summary");
  k_local_summary<<<grid_for((long long)p.N * 32, threads), threads, 0, s>>>(p);
  return 1;
}

#define PROF(name) if (pf) pf->mark(s, name)

// Enqueue the whole sweep solver (after the local summary): anticipation,
// plain host validity, masks, device validity, host validity, emission.
int enqueue_sweep_solver(const DevPlan &p, cudaStream_t s, int n_fin, Prof *pf) {
  const int T = 128;
  int n = 0;
  const long long NW = (long long)p.N * p.W;
  for (uint64_t *pl : {p.hp_out, p.d_in, p.d_out, p.h_in, p.h_out}) {
    PROF("fill_top");
    k_fill_top<<<grid_for(NW, 256), 256, 0, s>>>(pl, p.N, p.W, p.top);
    ++n;
  }
  cudaMemsetAsync(p.ant_h, 0, NW * sizeof(uint64_t), s);
  cudaMemsetAsync(p.ant_d, 0, NW * sizeof(uint64_t), s);
  cudaMemsetAsync(p.acc_flag, 0, (size_t)p.A, s);
  PROF("sweep_ant");
  k_sweep_ant<<<grid_for(p.W, T), T, 0, s>>>(p); ++n;
  if (p.ant_dm) { PROF("sweep_antm"); k_sweep_antm<<<grid_for(p.W, T), T, 0, s>>>(p); ++n; }
  PROF("sweep_hp");
  k_sweep_fwd<PH_HP><<<grid_for(p.W, T), T, 0, s>>>(p); ++n;
  if (p.L) { PROF("sweep_masks"); k_sweep_masks<<<grid_for((long long)p.L * p.W, T), T, 0, s>>>(p); ++n; }
  if (p.K) { PROF("edge_const_d"); k_edge_const<PH_D><<<grid_for((long long)p.K * p.W, T), T, 0, s>>>(p); ++n; }
  PROF("sweep_d");
  k_sweep_fwd<PH_D><<<grid_for(p.W, T), T, 0, s>>>(p); ++n;
  if (p.K) { PROF("edge_const_h"); k_edge_const<PH_H><<<grid_for((long long)p.K * p.W, T), T, 0, s>>>(p); ++n; }
  PROF("sweep_h");
  k_sweep_fwd<PH_H><<<grid_for(p.W, T), T, 0, s>>>(p); ++n;
  PROF("emit_flags");
  k_emit_flags<<<grid_for(p.M, T), T, 0, s>>>(p); ++n;
  if (n_fin) { PROF("emit_edges"); k_emit_edges<<<grid_for((long long)n_fin * p.W, T), T, 0, s>>>(p, n_fin); ++n; }
  if (p.X) { PROF("emit_exit"); k_emit_exit<<<grid_for((long long)p.X * p.W, T), T, 0, s>>>(p); ++n; }
  return n;
}

int enqueue_fill_unreachable(const DevPlan &p, cudaStream_t s, int keep_states, Prof *pf) {
  if (!p.n_unreach) return 0;
  PROF("fill_unreachable");
  k_fill_unreachable<<<grid_for((long long)p.n_unreach * p.W, 256), 256, 0, s>>>(p, keep_states);
  return 1;
}

// Re-run the edge emission alone (after the record buffer was enlarged).
int enqueue_sweep_edges(const DevPlan &p, cudaStream_t s, int n_fin) {
  if (n_fin) k_emit_edges<<<grid_for((long long)n_fin * p.W, 128), 128, 0, s>>>(p, n_fin);
  return n_fin ? 1 : 0;
}

}  // namespace ompdart
