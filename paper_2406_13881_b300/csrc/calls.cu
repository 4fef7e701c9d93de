// calls.cu -- the call-site pass: per-access flags of blocks holding call
// pseudo-accesses and the call-site rows (Sec. IV-C side effects applied at
// call sites; Sec. IV-D transfers).
//
// Runs after the host-validity pass, from the final entry states of each
// call block.  One warp per (call block, 64-word group), each lane owning
// two words of the variable planes:
//   forward, access by access from (H_in, D_in): a plain read finds its
//     space stale -> `to' (device) / `from' (host) flag, then valid; a write
//     makes its space valid and the other stale; a call first meets the
//     callee's requirements (call_to = ReqD & ~D, call_from = ReqH & ~H),
//     records the state the callee starts from, then applies GenS / KillS;
//   backward, from Live at the block exit (OR of the successors' Live_in,
//     or the region-exit row): a call records Live after it, then
//     Live = ReqH | ReqD | (Live & ~MustDef); a write ends liveness, a read
//     starts it.
// A second kernel turns each call site's rows into its access flag.
#include <cuda_runtime.h>

#include "solver.h"

namespace ompdart {
namespace {

constexpr int PLANES = 7;  // ReqH, ReqD, GenH, KillH, GenD, KillD, MustDef

__device__ __forceinline__ uint64_t wd(const uint64_t *row, int W, int w) { return w < W ? row[w] : 0ull; }

__global__ void k_call_blocks(DevPlan p) {
  const int gw = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int G = (p.W + 63) / 64;
  if (gw >= p.n_cblk * G) return;
  const int k = gw / G, wg = gw % G, lane = threadIdx.x & 31, W = p.W;
  const int b = p.cblk[k], a0 = p.acc_off[b], a1 = p.acc_off[b + 1];
  const int rowbase = p.cblk_rowbase[k];
  int w[2] = {wg * 64 + 2 * lane, wg * 64 + 2 * lane + 1};
  uint64_t h[2], d[2];
  for (int q = 0; q < 2; ++q) {
    h[q] = wd(p.h_in + (size_t)b * W, W, w[q]);
    d[q] = wd(p.d_in + (size_t)b * W, W, w[q]);
  }
  int site = p.cblk_site0[k];
  for (int i = a0; i < a1; ++i) {
    const uint32_t a = p.acc[i];
    if (a >> 31) {
      const uint64_t *row = p.calls + (size_t)(rowbase + (int)(a & 0x7FFFFFFFu)) * PLANES * W;
      for (int q = 0; q < 2; ++q) {
        if (w[q] >= W) continue;
        const uint64_t rqh = row[w[q]], rqd = row[W + w[q]];
        const size_t o = (size_t)site * W + w[q];
        p.call_from[o] = rqh & ~h[q];
        p.call_to[o] = rqd & ~d[q];
        h[q] |= rqh;
        d[q] |= rqd;
        p.call_entry_h[o] = h[q];
        p.call_entry_d[o] = d[q];
        h[q] = row[2 * W + w[q]] | (h[q] & ~row[3 * W + w[q]]);
        d[q] = row[4 * W + w[q]] | (d[q] & ~row[5 * W + w[q]]);
      }
      ++site;
      continue;
    }
    const int v = (int)(a & 0xFFFFFFu), kind = (int)((a >> 24) & 3u), dev = (int)((a >> 26) & 1u);
    const int lw = (v >> 6) - wg * 64;
    if (lw < 0 || lw >= 64 || (lw >> 1) != lane) continue;  // not this lane's word
    const int q = lw & 1;
    const uint64_t bit = 1ull << (v & 63);
    uint64_t &own = dev ? d[q] : h[q], &oth = dev ? h[q] : d[q];
    uint8_t flag = 0;
    if ((kind & 1) && !(own & bit)) {
      flag = dev ? 1 : 2;
      own |= bit;
    }
    if (kind & 2) {
      own |= bit;
      oth &= ~bit;
    }
    p.acc_flag[i] = flag;
  }
  // ---- backward: Live right after each call
  const int pos = p.pos[b];
  uint64_t x[2] = {0, 0};
  if (p.is_exit[pos]) {
    for (int q = 0; q < 2; ++q) x[q] = wd(p.exit_live + (size_t)p.cblk_cfg[k] * W, W, w[q]);
  } else {
    for (int e = p.out_off[pos]; e < p.out_off[pos + 1]; ++e)
      for (int q = 0; q < 2; ++q) x[q] |= wd(p.live + (size_t)p.out_dst[e] * W, W, w[q]);
  }
  for (int i = a1 - 1; i >= a0; --i) {
    const uint32_t a = p.acc[i];
    if (a >> 31) {
      --site;
      const uint64_t *row = p.calls + (size_t)(rowbase + (int)(a & 0x7FFFFFFFu)) * PLANES * W;
      for (int q = 0; q < 2; ++q) {
        if (w[q] >= W) continue;
        p.call_exit_live[(size_t)site * W + w[q]] = x[q];
        x[q] = row[w[q]] | row[W + w[q]] | (x[q] & ~row[6 * W + w[q]]);
      }
      continue;
    }
    const int v = (int)(a & 0xFFFFFFu), kind = (int)((a >> 24) & 3u);
    const int lw = (v >> 6) - wg * 64;
    if (lw < 0 || lw >= 64 || (lw >> 1) != lane) continue;
    const uint64_t bit = 1ull << (v & 63);
    if (kind & 2) x[lw & 1] &= ~bit;
    if (kind & 1) x[lw & 1] |= bit;
  }
}

// access flag of each call site: 1 if anything goes to the device, 2 if
// anything comes back to the host, 3 both
__global__ void k_call_flags(DevPlan p) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= p.n_sites) return;
  uint64_t to = 0, fr = 0;
  for (int w = 0; w < p.W; ++w) {
    to |= p.call_to[(size_t)s * p.W + w];
    fr |= p.call_from[(size_t)s * p.W + w];
  }
  p.acc_flag[p.site_acc[s]] = (uint8_t)((to ? 1 : 0) | (fr ? 2 : 0));
}

}  // namespace

int enqueue_call_sites(const DevPlan &p, cudaStream_t s, Prof *pf) {
  if (!p.n_sites) return 0;
  if (pf) pf->mark(s, "call_sites");
  const size_t rows = (size_t)p.n_sites * p.W * sizeof(uint64_t);
  // sites in unreachable blocks keep zero rows
  cudaMemsetAsync(p.call_to, 0, rows, s);
  cudaMemsetAsync(p.call_from, 0, rows, s);
  cudaMemsetAsync(p.call_entry_h, 0, rows, s);
  cudaMemsetAsync(p.call_entry_d, 0, rows, s);
  cudaMemsetAsync(p.call_exit_live, 0, rows, s);
  int n = 0;
  if (p.n_cblk) {
    const long long threads = (long long)p.n_cblk * ((p.W + 63) / 64) * 32;
    k_call_blocks<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(p);
    ++n;
  }
  if (pf) pf->mark(s, "call_flags");
  k_call_flags<<<(p.n_sites + 255) / 256, 256, 0, s>>>(p);
  return n + 1;
}

}  // namespace ompdart
