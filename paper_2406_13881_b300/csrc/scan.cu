// scan.cu -- chunked scan solver: the fast path for reducible CFGs whose
// loop bodies are contiguous in the loop-ordered reverse post-order.
//
// Every phase of the analysis (Sec. IV-D) is, per variable, a bit problem
// whose block functions have the form x -> g | (x & p) (in the "stale"
// domain for the forward must problems, in the anticipation domain for the
// backward one), closed under composition and union.  The order is cut at
// single-entry points (all edges crossing a cut enter the same block, none
// goes back), so the influence of one chunk on the next is one bit plane
// and a chunk's effect on it is one affine map  carry' = G | (carry & P).
// Each phase therefore runs as
//   summary  (one warp per chunk and 64-variable word group: G and P),
//   scan     (compose the maps over the chunks: every chunk's carry),
//   apply    (one warp per chunk: final values, outputs, emission).
// Inside a chunk the warp walks positions in order; a loop body (a
// contiguous run starting at its header) is walked again only when the
// value entering its header grew (closed form of a loop: header = entry |
// what the body contributes along its back edges, so one more pass is
// exact; Kam-Ullman rapidity).  Values a later position still needs live
// in slots assigned on the host by interval colouring (16 per plane in
// shared memory, the rest spilled to global scratch).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <functional>
#include <queue>
#include <string>
#include <vector>

#include "ingest.h"
#include "plan.cuh"

namespace ompdart {

namespace {

constexpr int CARRY = -2;      // slot id: the chunk's incoming carry
constexpr int SH_SLOTS = 16;   // slots per plane kept in shared memory
constexpr int MAX_DEPTH = 31;  // loop nesting depth the chain handles
// bound on loop re-runs per chunk walk: each loop of a reducible CFG needs
// at most one re-run per entry, so 8 per position is far beyond any valid
// walk; hitting it reports OMPDART_E_NOCONVERGE instead of spinning
__host__ __device__ inline int rerun_cap(int len) { return 8 * len + 64; }

enum PhaseKind { K_ANT = 0, K_HP = 1, K_D = 2, K_H = 3 };
enum ModeKind { M_SUM = 0, M_APPLY = 1, M_LANT = 2 };

struct PosMeta {  // one per position, 64 B
  int32_t blk;
  int32_t fin_beg, out_beg, acc_beg, srcent_beg, bend_beg;
  int16_t nfin, nout, nacc, nsrcent, nbend, fslot, bslot, pad0;
  int32_t head_loop;      // loop whose header is this position, else -1
  uint32_t latch_levels;  // bit d: back edge to the header of the level-d loop
  int32_t exit_idx;       // index in exit_blocks, else -1
  int32_t pad1, pad2, pad3;
};
static_assert(sizeof(PosMeta) == 64, "PosMeta layout");

struct LoopMeta {
  int32_t ph, pend;   // body = positions [ph, pend)
  int16_t hslot, depth;
  int32_t lat_beg;    // latch slots to clear on a fresh entry
  int32_t lat_cnt;
  int32_t pad;
};

struct ChunkMeta {
  int32_t s, e;             // positions [s, e)
  int32_t carry_beg, carry_cnt;
  int32_t loop_beg, loop_end;
  int32_t pad0, pad1;
};

struct CarrySrc {  // an edge from this chunk into the next chunk's first block
  int32_t slot, ent, fin_k, pad;
};

struct ScanDev {
  int C, G;           // chunks, word groups
  int fslots, bslots; // max slots (forward, backward)
  const PosMeta *meta;
  const LoopMeta *loops;
  const ChunkMeta *chunks;
  const CarrySrc *csrc;
  const int32_t *fin_slot, *fin_ent;
  const int32_t *out_slot, *out_pos;
  const int32_t *lat_slot;
  const int32_t *bend_loop;
  const int32_t *srcent;
  uint64_t *spill;     // per warp spill area
  int spill_stride;    // words per warp
  uint64_t *gsum, *psum;   // [planes][C][W] chunk maps
  uint64_t *carry;         // [planes][C][W] carry into each chunk
  uint64_t *hp_src, *d_src;  // [K][W] plain host / device validity at loop-entry sources
  uint64_t *xval;      // [n_carry_src][W] host-stale sets of crossing-edge sources
  int32_t *rec_cnt;    // [streams]
  const int32_t *rec_base, *rec_cap;  // [streams]
  EdgeXfer *stream;    // record streams
  int n_streams;
  int keep_states;
};

// ---- host side: per-chunk metadata and slot colouring -------------------------------

struct Interval {
  int a, b, id;
};

// Interval colouring: intervals sharing no position may share a slot.
int colour(std::vector<Interval> &iv, std::vector<int32_t> &slot_of) {
  std::sort(iv.begin(), iv.end(), [](const Interval &x, const Interval &y) { return x.a < y.a; });
  std::priority_queue<std::pair<int, int>, std::vector<std::pair<int, int>>, std::greater<>> active;
  std::priority_queue<int, std::vector<int>, std::greater<>> freeq;
  int n = 0;
  for (const Interval &x : iv) {
    while (!active.empty() && active.top().first < x.a) {
      freeq.push(active.top().second);
      active.pop();
    }
    int s;
    if (freeq.empty()) {
      s = n++;
    } else {
      s = freeq.top();
      freeq.pop();
    }
    slot_of[x.id] = s;
    active.push({x.b, s});
  }
  return n;
}

}  // namespace

struct ScanState {
  int C = 0, G = 0, fslots = 0, bslots = 0, n_streams = 0, n_apply_streams = 0;
  int n_csrc = 0;
  long long total_cap = 0;
  long long h2d = 0;
  std::vector<void *> allocs;
  ScanDev sd{};
  std::vector<int32_t> h_rec_cap;  // host copy of capacities
  int32_t *d_rec_cap = nullptr, *d_rec_base = nullptr;
  int32_t *offs = nullptr;         // stream offsets in the gathered result
  uint64_t *init = nullptr;        // [W] stale set entering the first chunk
  EdgeXfer *stream_buf = nullptr;
  ~ScanState() {
    for (void *p : allocs) cudaFree(p);
  }
  template <class T>
  T *alloc(size_t n) {
    void *p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return nullptr;
    allocs.push_back(p);
    return (T *)p;
  }
  template <class T>
  T *up(const std::vector<T> &v) {
    T *d = alloc<T>(v.size());
    if (d && !v.empty() && cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
      return nullptr;
    h2d += (long long)(v.size() * sizeof(T));
    return d;
  }
};

int scan_supported(const Ingest &g) {
  if (!g.reducible || !g.contiguous || g.M < 1) return 0;
  for (int l = 0; l < g.L; ++l)
    if (g.loop_depth[l] > MAX_DEPTH) return 0;
  return 1;
}

namespace {

bool build_meta(const Ingest &g, int target, ScanState *st, std::vector<PosMeta> &meta, std::vector<LoopMeta> &loops,
                std::vector<ChunkMeta> &chunks, std::vector<CarrySrc> &csrc, std::vector<int32_t> &fin_slot,
                std::vector<int32_t> &out_slot, std::vector<int32_t> &out_pos, std::vector<int32_t> &lat_slot,
                std::vector<int32_t> &bend_loop, std::vector<int32_t> &srcent, std::string *err) {
  Ingest &gm = const_cast<Ingest &>(g);
  make_chunks(&gm, target);
  const int M = g.M, C = (int)g.chunk_off.size() - 1, L = g.L;
  meta.assign(M, PosMeta{});
  loops.assign(L, LoopMeta{});
  chunks.assign(C, ChunkMeta{});
  std::vector<int32_t> head_loop_of_pos(M, -1);
  for (int l = 0; l < L; ++l) head_loop_of_pos[g.pos[g.loop_head[l]]] = l;
  std::vector<int32_t> exit_idx(g.N, -1);
  for (size_t x = 0; x < g.exit_blocks.size(); ++x) exit_idx[g.exit_blocks[x]] = (int32_t)x;
  // loop-entry edges by source block
  std::vector<std::vector<int32_t>> ent_by_src(g.N);
  for (int k = 0; k < g.K; ++k) ent_by_src[g.ent_src[k]].push_back(k);
  // loops ending at each position, outer first
  std::vector<std::vector<int32_t>> ends(M);
  for (int l = 0; l < L; ++l) ends[g.loop_end[l] - 1].push_back(l);
  for (auto &v : ends)
    std::sort(v.begin(), v.end(), [&](int a, int b) { return g.loop_depth[a] < g.loop_depth[b]; });

  fin_slot.assign(g.fin_src.size(), -1);
  out_slot.assign(g.out_dst.size(), -1);
  out_pos.assign(g.out_dst.size(), -1);
  std::vector<int32_t> fslot(M, -1), bslot(M, -1), hslot(L, -1);
  int max_f = 0, max_b = 0;
  // loop containing a block but not another: outermost such
  auto contains = [&](int l, int p) { return p >= g.pos[g.loop_head[l]] && p < g.loop_end[l]; };
  for (int c = 0; c < C; ++c) {
    const int s = g.chunk_off[c], e = g.chunk_off[c + 1];
    ChunkMeta &cm = chunks[c];
    cm.s = s;
    cm.e = e;
    // ---- forward values
    std::vector<Interval> iv;
    const int nval = e - s;  // ids: [0, nval) positions, [nval, nval + nloops) header in-values
    int lb = L, le = -1;
    for (int i = s; i < e; ++i) {
      const int b = g.order[i];
      int a = i, z = -1;
      for (int k = g.out_off[i]; k < g.out_off[i + 1]; ++k) {
        const int pt = g.pos[g.out_dst[k]];
        if (pt >= e) {
          z = std::max(z, e);
        } else if (pt > i) {
          const int l = head_loop_of_pos[pt];
          z = std::max(z, l >= 0 ? g.loop_end[l] - 1 : pt);
        } else {
          const int l = head_loop_of_pos[pt];
          if (l < 0) {
            if (err) *err = "retreating edge into a non-header";
            return false;
          }
          a = std::min(a, pt);
          z = std::max(z, g.loop_end[l] - 1);
        }
      }
      (void)b;
      if (z >= 0) iv.push_back({a, z, i - s});
      const int l = head_loop_of_pos[i];
      if (l >= 0) {
        lb = std::min(lb, l);
        le = std::max(le, l);
      }
    }
    std::vector<int32_t> loc_loops;
    if (le >= 0)
      for (int l = lb; l <= le; ++l) {
        loc_loops.push_back(l);
        iv.push_back({g.pos[g.loop_head[l]], g.loop_end[l] - 1, nval + (int)loc_loops.size() - 1});
      }
    cm.loop_beg = le >= 0 ? lb : 0;
    cm.loop_end = le >= 0 ? le + 1 : 0;
    std::vector<int32_t> so(nval + loc_loops.size(), -1);
    max_f = std::max(max_f, colour(iv, so));
    for (int i = s; i < e; ++i) fslot[i] = so[i - s];
    for (size_t q = 0; q < loc_loops.size(); ++q) hslot[loc_loops[q]] = so[nval + q];
    // ---- backward values
    iv.clear();
    for (int i = s; i < e; ++i) {
      int a = i, z = -1;
      const int b = g.order[i];
      for (int k = g.fin_off[i]; k < g.fin_off[i + 1]; ++k) {
        const int p = g.fin_src[k], pp = g.pos[p];
        if (pp < s) continue;  // crossing edge: read as the carry of chunk c-1
        if (pp < i) {
          int lo = pp;
          for (int x = g.inner_loop[p]; x >= 0; x = g.loop_parent[x]) {
            if (contains(x, i)) break;
            lo = std::min(lo, g.pos[g.loop_head[x]]);
          }
          a = std::min(a, lo);
          z = std::max(z, i);
        } else {
          const int l = head_loop_of_pos[i];
          a = std::min(a, i);
          z = std::max(z, g.loop_end[l] - 1);
        }
      }
      (void)b;
      if (z >= 0) iv.push_back({a, z, i - s});
    }
    std::vector<int32_t> sb(nval, -1);
    max_b = std::max(max_b, colour(iv, sb));
    for (int i = s; i < e; ++i) bslot[i] = sb[i - s];
  }
  // ---- per position records
  for (int i = 0; i < M; ++i) {
    const int b = g.order[i];
    PosMeta &m = meta[i];
    m.blk = b;
    m.fin_beg = g.fin_off[i];
    m.nfin = (int16_t)(g.fin_off[i + 1] - g.fin_off[i]);
    m.out_beg = g.out_off[i];
    m.nout = (int16_t)(g.out_off[i + 1] - g.out_off[i]);
    m.acc_beg = 0;  // filled from acc_off by the caller
    m.fslot = (int16_t)fslot[i];
    m.bslot = (int16_t)bslot[i];
    m.head_loop = head_loop_of_pos[i];
    m.exit_idx = exit_idx[b];
    m.srcent_beg = (int32_t)srcent.size();
    for (int k : ent_by_src[b]) srcent.push_back(k);
    m.nsrcent = (int16_t)(srcent.size() - m.srcent_beg);
    m.bend_beg = (int32_t)bend_loop.size();
    for (int l : ends[i]) bend_loop.push_back(l);
    m.nbend = (int16_t)(bend_loop.size() - m.bend_beg);
    m.latch_levels = 0;
    // find chunk of i for the slot ids of in-edges
  }
  for (int c = 0; c < C; ++c) {
    const int s = chunks[c].s, e = chunks[c].e;
    for (int i = s; i < e; ++i) {
      for (int k = g.fin_off[i]; k < g.fin_off[i + 1]; ++k) {
        const int pp = g.pos[g.fin_src[k]];
        fin_slot[k] = pp < s ? CARRY : fslot[pp];
        if (pp >= i) {  // back edge: the source is a latch of loop head_loop_of_pos[i]
          const int l = head_loop_of_pos[i];
          meta[pp].latch_levels |= 1u << (g.loop_depth[l] - 1);
        }
      }
      for (int k = g.out_off[i]; k < g.out_off[i + 1]; ++k) {
        const int pt = g.pos[g.out_dst[k]];
        out_pos[k] = pt;
        out_slot[k] = pt >= e ? CARRY : bslot[pt];
      }
    }
    // carry sources: edges into position e from this chunk
    chunks[c].carry_beg = (int32_t)csrc.size();
    if (e < M)
      for (int k = g.fin_off[e]; k < g.fin_off[e + 1]; ++k) {
        const int pp = g.pos[g.fin_src[k]];
        if (pp < e) csrc.push_back(CarrySrc{fslot[pp], g.fin_ent[k], k, 0});
      }
    chunks[c].carry_cnt = (int32_t)csrc.size() - chunks[c].carry_beg;
  }
  for (int l = 0; l < L; ++l) {
    LoopMeta &lm = loops[l];
    lm.ph = g.pos[g.loop_head[l]];
    lm.pend = g.loop_end[l];
    lm.hslot = (int16_t)hslot[l];
    lm.depth = (int16_t)g.loop_depth[l];
    lm.lat_beg = (int32_t)lat_slot.size();
    const int i = lm.ph;
    for (int k = g.fin_off[i]; k < g.fin_off[i + 1]; ++k) {
      const int pp = g.pos[g.fin_src[k]];
      if (pp >= i && std::find(lat_slot.begin() + lm.lat_beg, lat_slot.end(), fslot[pp]) == lat_slot.end())
        lat_slot.push_back(fslot[pp]);
    }
    lm.lat_cnt = (int32_t)lat_slot.size() - lm.lat_beg;
  }
  st->C = C;
  st->fslots = std::max(max_f, 1);
  st->bslots = std::max(max_b, 1);
  if (max_f > 32000 || max_b > 32000) {
    if (err) *err = "too many live values in one chunk";
    return false;
  }
  for (int i = 0; i < M; ++i)
    if (g.fin_off[i + 1] - g.fin_off[i] > 32000 || g.out_off[i + 1] - g.out_off[i] > 32000) {
      if (err) *err = "block degree too large for the scan solver";
      return false;
    }
  return true;
}

}  // namespace

// ==================================================================================
// device side
// ==================================================================================

namespace {

struct Lane {
  int lane, wg, w0;     // w0: first of the lane's two words (global word index)
  uint64_t top0, top1;  // valid-variable masks of the two words
};

template <int NP>
struct Slots {
  uint64_t *sh;     // [SH_SLOTS][NP][64]
  uint64_t *spill;  // [extra][NP][64]
  __device__ ulonglong2 *at(int slot, int plane, int lane) const {
    if (slot < SH_SLOTS) return reinterpret_cast<ulonglong2 *>(sh + ((size_t)(slot * NP + plane) * 64) + 2 * lane);
    return reinterpret_cast<ulonglong2 *>(spill + ((size_t)((slot - SH_SLOTS) * NP + plane) * 64) + 2 * lane);
  }
};

__device__ __forceinline__ uint64_t ld_word(const uint64_t *plane, size_t row, int W, int w) {
  return w < W ? plane[row * W + w] : 0ull;
}
__device__ __forceinline__ void st_word(uint64_t *plane, size_t row, int W, int w, uint64_t v) {
  if (w < W) plane[row * W + w] = v;
}

// Apply a block's summary records to the lane's two words of each plane.
//   ANT planes (H, D): local: UE -> 1, else write -> 0; coefficient: both -> 0
//   forward planes (stale sets): local: GEN -> 0 (valid), KILL -> 1 (stale);
//   coefficient: both -> 0.
template <int PH, int MODE, int NP>
__device__ __forceinline__ void apply_records(const DevPlan &p, const PosMeta &m, const Lane &L, uint64_t (&z)[NP][2],
                                              uint64_t &koh0, uint64_t &koh1, uint64_t &kod0, uint64_t &kod1) {
  const uint32_t *rec = p.rec + p.acc_off[m.blk];
  const int na = p.acc_off[m.blk + 1] - p.acc_off[m.blk];
  for (int r = 0; r < na; ++r) {
    const uint32_t rc = __ldg(rec + r);
    if (rc == REC_NONE) continue;
    const int lw = (int)((rc & 0xFFFFFFu) >> 6) - L.wg * 64;
    if ((unsigned)lw >= 64u || (lw >> 1) != L.lane) continue;
    const uint64_t bit = 1ull << (rc & 63u);
    const int j = lw & 1;
    if (PH == K_ANT) {
      // planes: SUM: [H local, H coef, D local, D coef]; APPLY/LANT: [H, D]
      const bool uh = rc & R_UH, ud = rc & R_UD, df = rc & R_DF;
      if (MODE == M_SUM) {
        z[0][j] = uh ? (z[0][j] | bit) : df ? (z[0][j] & ~bit) : z[0][j];
        if (uh || df) z[1][j] &= ~bit;
        z[2][j] = ud ? (z[2][j] | bit) : df ? (z[2][j] & ~bit) : z[2][j];
        if (ud || df) z[3][j] &= ~bit;
      } else {
        z[0][j] = uh ? (z[0][j] | bit) : df ? (z[0][j] & ~bit) : z[0][j];
        z[1][j] = ud ? (z[1][j] | bit) : df ? (z[1][j] & ~bit) : z[1][j];
        if (MODE == M_LANT) {
          if (rc & R_KH) { if (j) koh1 |= bit; else koh0 |= bit; }
          if (rc & R_KD) { if (j) kod1 |= bit; else kod0 |= bit; }
        }
      }
    } else {
      const uint32_t GEN = PH == K_D ? R_GD : R_GH, KILL = PH == K_D ? R_KD : R_KH;
      if (rc & GEN) z[0][j] &= ~bit;
      else if (rc & KILL) z[0][j] |= bit;
      if (MODE == M_SUM && (rc & (GEN | KILL))) z[1][j] &= ~bit;
    }
  }
}

// The H-phase emission for one position (apply mode): per-access flags,
// in-chunk edge records, exit transfers.
__device__ void emit_position(const DevPlan &p, const ScanDev &sd, const Lane &L, const PosMeta &m,
                              const Slots<1> &sl, const uint64_t zin[2], const uint64_t zout[2],
                              const uint64_t din[2], const uint64_t live[2], uint64_t *hd, int stream,
                              int &rec_count) {
  const int W = p.W, lane = L.lane;
  // ---- access flags: replay the block from its entry states
  hd[2 * lane] = ~zin[0] & L.top0;
  hd[2 * lane + 1] = ~zin[1] & L.top1;
  hd[64 + 2 * lane] = din[0];
  hd[64 + 2 * lane + 1] = din[1];
  __syncwarp();
  const int a0 = p.acc_off[m.blk], a1 = p.acc_off[m.blk + 1];
  for (int j = a0 + lane; j < a1; j += 32) {
    const uint32_t a = p.acc[j];
    const int v = acc_var(a), lw = (v >> 6) - L.wg * 64;
    if ((unsigned)lw >= 64u) continue;
    const uint64_t bit = 1ull << (v & 63);
    bool h = (hd[lw] & bit) != 0, d = (hd[64 + lw] & bit) != 0;
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
  __syncwarp();
  // ---- edge transfers on in-chunk in-edges
  const uint64_t c0 = live[0] & ~din[0], c1 = live[1] & ~din[1];
  for (int q = 0; q < m.nfin; ++q) {
    const int k = m.fin_beg + q;
    const int slot = sd.fin_slot[k];
    if (slot == CARRY) continue;
    const int ent = sd.fin_ent[k];
    const ulonglong2 zs = *sl.at(slot, 0, lane);
    uint64_t to0 = 0, to1 = 0, fr0, fr1;
    uint64_t e0 = zs.x, e1 = zs.y;
    if (ent >= 0) {
      const uint64_t eh0 = ld_word(p.ec_h, ent, W, L.w0), eh1 = ld_word(p.ec_h, ent, W, L.w0 + 1);
      const uint64_t ed0 = ld_word(p.ec_d, ent, W, L.w0), ed1 = ld_word(p.ec_d, ent, W, L.w0 + 1);
      to0 = ed0 & ~ld_word(sd.d_src, ent, W, L.w0);
      to1 = ed1 & ~ld_word(sd.d_src, ent, W, L.w0 + 1);
      fr0 = eh0 & zs.x;
      fr1 = eh1 & zs.y;
      e0 &= ~eh0;
      e1 &= ~eh1;
    } else {
      fr0 = fr1 = 0;
    }
    fr0 |= c0 & e0;
    fr1 |= c1 & e1;
    const bool n0 = (to0 | fr0) != 0, n1 = (to1 | fr1) != 0;
    const unsigned b0 = __ballot_sync(0xffffffffu, n0), b1 = __ballot_sync(0xffffffffu, n1);
    if (b0 | b1) {
      const int eid = p.fin_eid[k];
      const unsigned below = (1u << lane) - 1u;
      const int off0 = __popc(b0 & below) + __popc(b1 & below);
      const int base = rec_count;
      const int cap = sd.rec_cap[stream];
      EdgeXfer *out = sd.stream + sd.rec_base[stream];
      int idx = base + off0;
      if (n0) { if (idx < cap) out[idx] = EdgeXfer{eid, L.w0, to0, fr0}; ++idx; }
      if (n1) { if (idx < cap) out[idx] = EdgeXfer{eid, L.w0 + 1, to1, fr1}; }
      rec_count = base + __popc(b0) + __popc(b1);
    }
  }
  // ---- region exit
  if (m.exit_idx >= 0) {
    st_word(p.from_exit, m.exit_idx, W, L.w0, p.exit_live[min(L.w0, W - 1)] & zout[0] & L.top0);
    if (L.w0 + 1 < W) st_word(p.from_exit, m.exit_idx, W, L.w0 + 1, p.exit_live[L.w0 + 1] & zout[1] & L.top1);
  }
}

// --------------------------------------------------------------------------------------
// forward chain (Hp, D, H): positions ascending
// --------------------------------------------------------------------------------------
template <int PH, int MODE>
__global__ void __launch_bounds__(128) k_fwd_chain(DevPlan p, ScanDev sd) {
  constexpr int NP = MODE == M_SUM ? 2 : 1;
  extern __shared__ __align__(16) uint64_t smem[];
  const int warp_in_cta = threadIdx.x >> 5;
  const int gw = blockIdx.x * (blockDim.x >> 5) + warp_in_cta;
  if (gw >= sd.C * sd.G) return;
  const int c = gw / sd.G, wg = gw % sd.G;
  const int W = p.W;
  Lane L;
  L.lane = threadIdx.x & 31;
  L.wg = wg;
  L.w0 = wg * 64 + 2 * L.lane;
  L.top0 = L.w0 < W ? p.top[L.w0] : 0;
  L.top1 = L.w0 + 1 < W ? p.top[L.w0 + 1] : 0;
  uint64_t *wsm = smem + (size_t)warp_in_cta * (SH_SLOTS * NP * 64 + 128);
  Slots<NP> sl{wsm, sd.spill + (size_t)gw * sd.spill_stride};
  uint64_t *hd = wsm + SH_SLOTS * NP * 64;
  const ChunkMeta cm = sd.chunks[c];
  const uint64_t *ec = PH == K_D ? p.ec_d : p.ec_h;
  // carry into this chunk, per plane
  uint64_t cin[NP][2];
  if (MODE == M_SUM) {
    cin[0][0] = cin[0][1] = 0;
    cin[1][0] = L.top0;
    cin[1][1] = L.top1;
  } else {
    cin[0][0] = ld_word(sd.carry, c, W, L.w0);
    cin[0][1] = ld_word(sd.carry, c, W, L.w0 + 1);
  }
  const int stream = c * sd.G + wg;
  int rec_count = 0;
  int st_loop[MAX_DEPTH + 1];
  int st_rec[MAX_DEPTH + 1];
  int depth = 0;
  uint32_t dirty = 0;
  int reruns = 0;
  uint64_t dummy = 0;
  uint64_t z[NP][2], zo[NP][2];
  uint64_t din[2] = {0, 0}, lv[2] = {0, 0};
  int i = cm.s;
  while (i < cm.e) {
    const PosMeta m = sd.meta[i];
    if (m.head_loop >= 0) {
      const LoopMeta lm = sd.loops[m.head_loop];
      if (lm.depth > depth) {  // fresh entry: latch values start from nothing
        st_loop[depth] = m.head_loop;
        st_rec[depth] = rec_count;
        dirty &= ~(1u << depth);
        ++depth;
        for (int q = 0; q < lm.lat_cnt; ++q) {
          const int s = sd.lat_slot[lm.lat_beg + q];
          for (int pl = 0; pl < NP; ++pl) *sl.at(s, pl, L.lane) = make_ulonglong2(0ull, 0ull);
        }
        __syncwarp();
      }
    }
    // ---- value entering the block
#pragma unroll
    for (int pl = 0; pl < NP; ++pl) z[pl][0] = z[pl][1] = 0;
    if (i == cm.s) {
#pragma unroll
      for (int pl = 0; pl < NP; ++pl) { z[pl][0] = cin[pl][0]; z[pl][1] = cin[pl][1]; }
    }
    for (int q = 0; q < m.nfin; ++q) {
      const int k = m.fin_beg + q;
      const int slot = sd.fin_slot[k];
      if (slot == CARRY) continue;  // already in z via cin
      uint64_t m0 = ~0ull, m1 = ~0ull;
      if (PH != K_HP) {
        const int ent = sd.fin_ent[k];
        if (ent >= 0) { m0 = ~ld_word(ec, ent, W, L.w0); m1 = ~ld_word(ec, ent, W, L.w0 + 1); }
      }
#pragma unroll
      for (int pl = 0; pl < NP; ++pl) {
        const ulonglong2 v = *sl.at(slot, pl, L.lane);
        z[pl][0] |= v.x & m0;
        z[pl][1] |= v.y & m1;
      }
    }
    // a header remembers the meet of its in-edges (before the node's own
    // mask): a latch that adds to it makes the loop body run again
    if (m.head_loop >= 0) {
      const int hs = sd.loops[m.head_loop].hslot;
#pragma unroll
      for (int pl = 0; pl < NP; ++pl) *sl.at(hs, pl, L.lane) = make_ulonglong2(z[pl][0], z[pl][1]);
    }
    if (PH == K_H) {  // live and stale on the device -> resolved toward the host
      const size_t row = (size_t)m.blk;
      lv[0] = ld_word(p.live, row, W, L.w0); lv[1] = ld_word(p.live, row, W, L.w0 + 1);
      din[0] = ld_word(p.d_in, row, W, L.w0); din[1] = ld_word(p.d_in, row, W, L.w0 + 1);
      const uint64_t b0 = ~(lv[0] & ~din[0]), b1 = ~(lv[1] & ~din[1]);
#pragma unroll
      for (int pl = 0; pl < NP; ++pl) { z[pl][0] &= b0; z[pl][1] &= b1; }
    }
#pragma unroll
    for (int pl = 0; pl < NP; ++pl) { zo[pl][0] = z[pl][0]; zo[pl][1] = z[pl][1]; }
    apply_records<PH, MODE, NP>(p, m, L, zo, dummy, dummy, dummy, dummy);
    // ---- a latch whose value adds to an open loop's header marks it dirty
    if (m.latch_levels) {
      uint32_t lvmask = m.latch_levels;
      while (lvmask) {
        const int lvl = __ffs(lvmask) - 1;
        lvmask &= lvmask - 1;
        if (lvl >= depth) continue;
        const int hs = sd.loops[st_loop[lvl]].hslot;
        bool grow = false;
#pragma unroll
        for (int pl = 0; pl < NP; ++pl) {
          const ulonglong2 h = *sl.at(hs, pl, L.lane);
          grow |= ((zo[pl][0] & ~h.x) | (zo[pl][1] & ~h.y)) != 0;
        }
        if (__any_sync(0xffffffffu, grow)) dirty |= 1u << lvl;
      }
    }
    if (m.fslot >= 0) {
#pragma unroll
      for (int pl = 0; pl < NP; ++pl) *sl.at(m.fslot, pl, L.lane) = make_ulonglong2(zo[pl][0], zo[pl][1]);
    }
    // ---- outputs
    if (MODE == M_APPLY) {
      const size_t row = (size_t)m.blk;
      if (PH == K_D) {
        st_word(p.d_in, row, W, L.w0, ~z[0][0] & L.top0);
        st_word(p.d_in, row, W, L.w0 + 1, ~z[0][1] & L.top1);
        if (sd.keep_states) {
          st_word(p.d_out, row, W, L.w0, ~zo[0][0] & L.top0);
          st_word(p.d_out, row, W, L.w0 + 1, ~zo[0][1] & L.top1);
        }
      }
      if (PH == K_H) {
        st_word(p.h_in, row, W, L.w0, ~z[0][0] & L.top0);
        st_word(p.h_in, row, W, L.w0 + 1, ~z[0][1] & L.top1);
        if (sd.keep_states) {
          st_word(p.h_out, row, W, L.w0, ~zo[0][0] & L.top0);
          st_word(p.h_out, row, W, L.w0 + 1, ~zo[0][1] & L.top1);
        }
        __syncwarp();
        emit_position(p, sd, L, m, *reinterpret_cast<Slots<1> *>(&sl), z[0], zo[0], din, lv, hd, stream, rec_count);
      }
      if ((PH == K_HP || PH == K_D) && m.nsrcent) {
        uint64_t *dst = PH == K_HP ? sd.hp_src : sd.d_src;
        for (int q = 0; q < m.nsrcent; ++q) {
          const int k = sd.srcent[m.srcent_beg + q];
          st_word(dst, k, W, L.w0, ~zo[0][0] & L.top0);
          st_word(dst, k, W, L.w0 + 1, ~zo[0][1] & L.top1);
        }
      }
    }
    __syncwarp();
    // ---- close loops ending here; walk a body again if its header grew
    bool jumped = false;
    while (depth > 0) {
      const LoopMeta lt = sd.loops[st_loop[depth - 1]];
      if (lt.pend - 1 != i) break;
      if (dirty & (1u << (depth - 1))) {
        dirty &= ~(1u << (depth - 1));
        rec_count = st_rec[depth - 1];
        i = lt.ph;
        jumped = true;
        break;
      }
      --depth;
    }
    if (jumped) {
      if (++reruns > rerun_cap(cm.e - cm.s)) {
        if (L.lane == 0) atomicExch(&p.status[ST_ERROR], ERR_NOCONVERGE);
        break;
      }
    } else {
      ++i;
    }
  }
  // ---- what leaves the chunk: the carry into the next chunk's first block
  if (MODE == M_SUM || (MODE == M_APPLY && PH == K_H)) {
    uint64_t co[NP][2];
#pragma unroll
    for (int pl = 0; pl < NP; ++pl) co[pl][0] = co[pl][1] = 0;
    for (int q = 0; q < cm.carry_cnt; ++q) {
      const CarrySrc cs = sd.csrc[cm.carry_beg + q];
      if (MODE == M_SUM) {
        uint64_t m0 = ~0ull, m1 = ~0ull;
        if (PH != K_HP && cs.ent >= 0) { m0 = ~ld_word(ec, cs.ent, W, L.w0); m1 = ~ld_word(ec, cs.ent, W, L.w0 + 1); }
#pragma unroll
        for (int pl = 0; pl < NP; ++pl) {
          const ulonglong2 v = *sl.at(cs.slot, pl, L.lane);
          co[pl][0] |= v.x & m0;
          co[pl][1] |= v.y & m1;
        }
      } else {
        const ulonglong2 v = *sl.at(cs.slot, 0, L.lane);
        st_word(sd.xval, cm.carry_beg + q, W, L.w0, v.x);
        st_word(sd.xval, cm.carry_beg + q, W, L.w0 + 1, v.y);
      }
    }
    if (MODE == M_SUM && cm.carry_cnt) {
      st_word(sd.gsum, c, W, L.w0, co[0][0]);
      st_word(sd.gsum, c, W, L.w0 + 1, co[0][1]);
      st_word(sd.psum, c, W, L.w0, co[1][0]);
      st_word(sd.psum, c, W, L.w0 + 1, co[1][1]);
    }
  }
  if (MODE == M_APPLY && PH == K_H && L.lane == 0) sd.rec_cnt[stream] = rec_count;
}

// --------------------------------------------------------------------------------------
// backward chain (anticipation; loop-restricted anticipation for the masks)
// --------------------------------------------------------------------------------------
template <int MODE>
__device__ void bwd_range(const DevPlan &p, const ScanDev &sd, const Lane &L, const Slots<(MODE == M_SUM ? 4 : 2)> &sl,
                          int s, int e, int base_depth, int lo_pos, bool use_carry,
                          const uint64_t (&cin)[(MODE == M_SUM ? 4 : 2)][2], uint64_t (&zlast)[(MODE == M_SUM ? 4 : 2)][2],
                          uint64_t &koh0, uint64_t &koh1, uint64_t &kod0, uint64_t &kod1) {
  constexpr int NP = MODE == M_SUM ? 4 : 2;
  const int W = p.W;
  const uint64_t xl0 = L.w0 < W ? p.exit_live[L.w0] : 0, xl1 = L.w0 + 1 < W ? p.exit_live[L.w0 + 1] : 0;
  int st_loop[MAX_DEPTH + 1];
  int depth = base_depth;
  uint32_t dirty = 0;
  int reruns = 0;
  uint64_t z[NP][2];
  int i = e - 1;
  while (i >= s) {
    const PosMeta m = sd.meta[i];
    // enter loops whose range ends here (outer first)
    for (int q = 0; q < m.nbend; ++q) {
      const int l = sd.bend_loop[m.bend_beg + q];
      const LoopMeta lm = sd.loops[l];
      if (lm.depth <= depth) continue;
      st_loop[lm.depth - 1] = l;
      dirty &= ~(1u << (lm.depth - 1));
      depth = lm.depth;
      const int hs = sd.meta[lm.ph].bslot;
      if (hs >= 0)
        for (int pl = 0; pl < NP; ++pl) *sl.at(hs, pl, L.lane) = make_ulonglong2(0ull, 0ull);
      __syncwarp();
    }
#pragma unroll
    for (int pl = 0; pl < NP; ++pl) z[pl][0] = z[pl][1] = 0;
    if (MODE != M_LANT && m.exit_idx >= 0) {  // region exit: the host may read what is live
      z[0][0] = xl0;
      z[0][1] = xl1;
    }
    for (int q = 0; q < m.nout; ++q) {
      const int k = m.out_beg + q;
      const int slot = sd.out_slot[k];
      if (MODE == M_LANT) {
        const int pt = sd.out_pos[k];
        if (pt <= lo_pos || pt >= e) continue;  // back to the loop header or out of the body
      }
      if (slot == CARRY) {
        if (use_carry) {
#pragma unroll
          for (int pl = 0; pl < NP; ++pl) { z[pl][0] |= cin[pl][0]; z[pl][1] |= cin[pl][1]; }
        }
        continue;
      }
#pragma unroll
      for (int pl = 0; pl < NP; ++pl) {
        const ulonglong2 v = *sl.at(slot, pl, L.lane);
        z[pl][0] |= v.x;
        z[pl][1] |= v.y;
      }
    }
    apply_records<K_ANT, MODE, NP>(p, m, L, z, koh0, koh1, kod0, kod1);
    if (m.bslot >= 0) {
      bool changed = false;
      const bool is_top_header = depth > base_depth && sd.loops[st_loop[depth - 1]].ph == i;
#pragma unroll
      for (int pl = 0; pl < NP; ++pl) {
        ulonglong2 *ptr = sl.at(m.bslot, pl, L.lane);
        if (is_top_header) {
          const ulonglong2 old = *ptr;
          changed |= (old.x != z[pl][0]) || (old.y != z[pl][1]);
        }
        *ptr = make_ulonglong2(z[pl][0], z[pl][1]);
      }
      if (is_top_header && __any_sync(0xffffffffu, changed)) dirty |= 1u << (depth - 1);
    }
    if (MODE == M_APPLY) {
      st_word(p.live, m.blk, W, L.w0, z[0][0] | z[1][0]);
      st_word(p.live, m.blk, W, L.w0 + 1, z[0][1] | z[1][1]);
    }
    __syncwarp();
#pragma unroll
    for (int pl = 0; pl < NP; ++pl) { zlast[pl][0] = z[pl][0]; zlast[pl][1] = z[pl][1]; }
    bool jumped = false;
    while (depth > base_depth) {
      const LoopMeta lt = sd.loops[st_loop[depth - 1]];
      if (lt.ph != i) break;
      if (dirty & (1u << (depth - 1))) {
        dirty &= ~(1u << (depth - 1));
        i = lt.pend - 1;
        jumped = true;
        break;
      }
      --depth;
    }
    if (jumped) {
      if (++reruns > rerun_cap(e - s)) {
        if (L.lane == 0) atomicExch(&p.status[ST_ERROR], ERR_NOCONVERGE);
        return;
      }
    } else {
      --i;
    }
  }
}

template <int MODE>
__global__ void __launch_bounds__(128) k_bwd_chain(DevPlan p, ScanDev sd) {
  constexpr int NP = MODE == M_SUM ? 4 : 2;
  extern __shared__ __align__(16) uint64_t smem[];
  const int warp_in_cta = threadIdx.x >> 5;
  const int gw = blockIdx.x * (blockDim.x >> 5) + warp_in_cta;
  if (gw >= sd.C * sd.G) return;
  const int c = gw / sd.G, wg = gw % sd.G;
  const int W = p.W;
  Lane L;
  L.lane = threadIdx.x & 31;
  L.wg = wg;
  L.w0 = wg * 64 + 2 * L.lane;
  L.top0 = L.w0 < W ? p.top[L.w0] : 0;
  L.top1 = L.w0 + 1 < W ? p.top[L.w0 + 1] : 0;
  uint64_t *wsm = smem + (size_t)warp_in_cta * (SH_SLOTS * NP * 64);
  Slots<NP> sl{wsm, sd.spill + (size_t)gw * sd.spill_stride};
  const ChunkMeta cm = sd.chunks[c];
  uint64_t cin[NP][2], zl[NP][2];
  uint64_t koh0 = 0, koh1 = 0, kod0 = 0, kod1 = 0;
  if (MODE == M_LANT) {
#pragma unroll
    for (int pl = 0; pl < NP; ++pl) cin[pl][0] = cin[pl][1] = 0;
    for (int l = cm.loop_beg; l < cm.loop_end; ++l) {
      const LoopMeta lm = sd.loops[l];
      koh0 = koh1 = kod0 = kod1 = 0;
      bwd_range<MODE>(p, sd, L, sl, lm.ph, lm.pend, lm.depth, lm.ph, false, cin, zl, koh0, koh1, kod0, kod1);
      st_word(p.mask_h, l, W, L.w0, zl[0][0] & ~koh0 & L.top0);
      st_word(p.mask_h, l, W, L.w0 + 1, zl[0][1] & ~koh1 & L.top1);
      st_word(p.mask_d, l, W, L.w0, zl[1][0] & ~kod0 & L.top0);
      st_word(p.mask_d, l, W, L.w0 + 1, zl[1][1] & ~kod1 & L.top1);
    }
    return;
  }
  // carry: anticipation entering the next chunk's first block
  if (MODE == M_SUM) {
    cin[0][0] = cin[0][1] = 0;
    cin[1][0] = L.top0; cin[1][1] = L.top1;
    cin[2][0] = cin[2][1] = 0;
    cin[3][0] = L.top0; cin[3][1] = L.top1;
  } else {
    const size_t CW = (size_t)sd.C;
    cin[0][0] = ld_word(sd.carry, c, W, L.w0);
    cin[0][1] = ld_word(sd.carry, c, W, L.w0 + 1);
    cin[1][0] = ld_word(sd.carry + CW * W, c, W, L.w0);
    cin[1][1] = ld_word(sd.carry + CW * W, c, W, L.w0 + 1);
  }
  bwd_range<MODE>(p, sd, L, sl, cm.s, cm.e, 0, -1, true, cin, zl, koh0, koh1, kod0, kod1);
  if (MODE == M_SUM) {
    const size_t CW = (size_t)sd.C * W;
    st_word(sd.gsum, c, W, L.w0, zl[0][0]);
    st_word(sd.gsum, c, W, L.w0 + 1, zl[0][1]);
    st_word(sd.psum, c, W, L.w0, zl[1][0]);
    st_word(sd.psum, c, W, L.w0 + 1, zl[1][1]);
    st_word(sd.gsum + CW, c, W, L.w0, zl[2][0]);
    st_word(sd.gsum + CW, c, W, L.w0 + 1, zl[2][1]);
    st_word(sd.psum + CW, c, W, L.w0, zl[3][0]);
    st_word(sd.psum + CW, c, W, L.w0 + 1, zl[3][1]);
  }
}

// --------------------------------------------------------------------------------------
// scan of the chunk maps: carry[c] for every chunk (one thread per word and plane)
// --------------------------------------------------------------------------------------
__global__ void k_scan_carry(ScanDev sd, int W, int planes, int backward, const uint64_t *init0,
                             const uint64_t *init1) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= planes * W) return;
  const int pl = t / W, w = t % W;
  const size_t off = (size_t)pl * sd.C * W;
  const uint64_t *G = sd.gsum + off, *P = sd.psum + off;
  uint64_t *car = sd.carry + off;
  uint64_t x = init0 ? (pl == 0 ? init0[w] : init1[w]) : 0ull;
  if (!backward) {
    for (int c = 0; c < sd.C; ++c) {
      car[(size_t)c * W + w] = x;
      x = G[(size_t)c * W + w] | (x & P[(size_t)c * W + w]);
    }
  } else {
    for (int c = sd.C - 1; c >= 0; --c) {
      car[(size_t)c * W + w] = x;
      x = G[(size_t)c * W + w] | (x & P[(size_t)c * W + w]);
    }
  }
}

// initial stale sets at the entry block (forward problems): ~valid & top
__global__ void k_entry_stale(const uint64_t *valid, const uint64_t *top, uint64_t *out, int W) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w < W) out[w] = ~valid[w] & top[w];
}

// loop-entry edge constants (hoisted transfers): device = mask_d & plain
// host valid at the source; host = mask_h & device valid at the source
__global__ void k_scan_edge_const(DevPlan p, ScanDev sd, int which) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)p.K * p.W) return;
  const int k = (int)(t / p.W), w = (int)(t % p.W);
  const int l = p.ent_loop[k];
  if (which == 0)
    p.ec_d[t] = p.mask_d[(size_t)l * p.W + w] & sd.hp_src[t];
  else
    p.ec_h[t] = p.mask_h[(size_t)l * p.W + w] & sd.d_src[t];
}

// edge transfers on edges that cross a chunk boundary (into the first block
// of chunk c from chunk c-1), from the sources' stored host-stale sets
__global__ void k_cross_emit(DevPlan p, ScanDev sd, int stream0) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= sd.C * sd.G) return;
  const int c = gw / sd.G, wg = gw % sd.G, lane = threadIdx.x & 31, W = p.W;
  const int stream = stream0 + gw;
  int cnt = 0;
  if (c + 1 < sd.C) {
    const ChunkMeta cm = sd.chunks[c];
    const int dst = sd.meta[cm.e].blk;
    const int w0 = wg * 64 + 2 * lane;
    const uint64_t lv0 = ld_word(p.live, dst, W, w0), lv1 = ld_word(p.live, dst, W, w0 + 1);
    const uint64_t di0 = ld_word(p.d_in, dst, W, w0), di1 = ld_word(p.d_in, dst, W, w0 + 1);
    const uint64_t c0 = lv0 & ~di0, c1 = lv1 & ~di1;
    EdgeXfer *out = sd.stream + sd.rec_base[stream];
    const int cap = sd.rec_cap[stream];
    for (int q = 0; q < cm.carry_cnt; ++q) {
      const CarrySrc cs = sd.csrc[cm.carry_beg + q];
      const uint64_t zs0 = ld_word(sd.xval, cm.carry_beg + q, W, w0), zs1 = ld_word(sd.xval, cm.carry_beg + q, W, w0 + 1);
      uint64_t to0 = 0, to1 = 0, fr0 = 0, fr1 = 0, e0 = zs0, e1 = zs1;
      if (cs.ent >= 0) {
        const uint64_t eh0 = ld_word(p.ec_h, cs.ent, W, w0), eh1 = ld_word(p.ec_h, cs.ent, W, w0 + 1);
        to0 = ld_word(p.ec_d, cs.ent, W, w0) & ~ld_word(sd.d_src, cs.ent, W, w0);
        to1 = ld_word(p.ec_d, cs.ent, W, w0 + 1) & ~ld_word(sd.d_src, cs.ent, W, w0 + 1);
        fr0 = eh0 & zs0;
        fr1 = eh1 & zs1;
        e0 &= ~eh0;
        e1 &= ~eh1;
      }
      fr0 |= c0 & e0;
      fr1 |= c1 & e1;
      const bool n0 = (to0 | fr0) != 0, n1 = (to1 | fr1) != 0;
      const unsigned b0 = __ballot_sync(0xffffffffu, n0), b1 = __ballot_sync(0xffffffffu, n1);
      if (b0 | b1) {
        const int eid = p.fin_eid[cs.fin_k];
        const unsigned below = (1u << lane) - 1u;
        int idx = cnt + __popc(b0 & below) + __popc(b1 & below);
        if (n0) { if (idx < cap) out[idx] = EdgeXfer{eid, w0, to0, fr0}; ++idx; }
        if (n1) { if (idx < cap) out[idx] = EdgeXfer{eid, w0 + 1, to1, fr1}; }
        cnt += __popc(b0) + __popc(b1);
      }
    }
  }
  if (lane == 0) sd.rec_cnt[stream] = cnt;
}

// gather the record streams into the result array (single CTA prefix, then copy)
__global__ void k_streams_prefix(ScanDev sd, int32_t *offs, int32_t *status) {
  __shared__ int32_t part[1024];
  __shared__ int overflow;
  const int t = threadIdx.x, n = sd.n_streams;
  if (t == 0) overflow = 0;
  __syncthreads();
  // each thread sums a contiguous range
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int b = t * per, e = min(n, b + per);
  int sum = 0;
  for (int i = b; i < e; ++i) {
    const int cnt = sd.rec_cnt[i];
    if (cnt > sd.rec_cap[i]) overflow = 1;
    sum += cnt;
  }
  part[t] = sum;
  __syncthreads();
  if (t == 0) {
    int run = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      const int x = part[i];
      part[i] = run;
      run += x;
    }
    status[ST_NREC] = run;
    if (overflow) status[ST_OVERFLOW] = 1;
  }
  __syncthreads();
  int run = part[t];
  for (int i = b; i < e; ++i) {
    offs[i] = run;
    run += sd.rec_cnt[i];
  }
}

__global__ void k_streams_copy(ScanDev sd, const int32_t *offs, EdgeXfer *dst, int cap) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (gw >= sd.n_streams) return;
  const int n = min(sd.rec_cnt[gw], sd.rec_cap[gw]);
  const EdgeXfer *src = sd.stream + sd.rec_base[gw];
  const int o = offs[gw];
  for (int i = lane; i < n; i += 32)
    if (o + i < cap) dst[o + i] = src[i];
}

int grid_of(long long n, int b) { return (int)std::max<long long>(1, std::min<long long>((n + b - 1) / b, 1 << 30)); }

template <class K>
void set_smem(K kern, size_t bytes) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

// ==================================================================================
// host interface
// ==================================================================================

// Upload stream capacities (and bases) and (re)allocate the stream buffer.
static bool scan_set_streams(ScanState *st) {
  std::vector<int32_t> base(st->n_streams);
  long long tot = 0;
  for (int i = 0; i < st->n_streams; ++i) {
    base[i] = (int32_t)tot;
    tot += st->h_rec_cap[i];
  }
  if (tot >= (1ll << 31)) return false;
  if (st->stream_buf) {
    cudaFree(st->stream_buf);
    st->allocs.erase(std::find(st->allocs.begin(), st->allocs.end(), (void *)st->stream_buf));
  }
  st->stream_buf = st->alloc<EdgeXfer>((size_t)tot);
  if (!st->stream_buf) return false;
  st->total_cap = tot;
  st->sd.stream = st->stream_buf;
  if (cudaMemcpy(st->d_rec_cap, st->h_rec_cap.data(), sizeof(int32_t) * st->n_streams, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(st->d_rec_base, base.data(), sizeof(int32_t) * st->n_streams, cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  return true;
}

ScanState *scan_create(const Ingest &g, DevPlan &p, int chunk_target, int keep_states, std::string *err) {
  ScanState *st = new ScanState();
  std::vector<PosMeta> meta;
  std::vector<LoopMeta> loops;
  std::vector<ChunkMeta> chunks;
  std::vector<CarrySrc> csrc;
  std::vector<int32_t> fin_slot, out_slot, out_pos, lat_slot, bend_loop, srcent;
  if (chunk_target <= 0) chunk_target = g.M <= 4096 ? std::max(64, g.M / 8) : 512;
  if (!build_meta(g, chunk_target, st, meta, loops, chunks, csrc, fin_slot, out_slot, out_pos, lat_slot, bend_loop,
                  srcent, err)) {
    delete st;
    return nullptr;
  }
  std::vector<int32_t> acc_off_h(g.N + 1);
  if (cudaMemcpy(acc_off_h.data(), p.acc_off, sizeof(int32_t) * (g.N + 1), cudaMemcpyDeviceToHost) != cudaSuccess) {
    if (err) *err = "copy of access offsets failed";
    delete st;
    return nullptr;
  }
  for (int i = 0; i < g.M; ++i) {
    meta[i].acc_beg = acc_off_h[meta[i].blk];
    meta[i].nacc = (int16_t)std::min(32767, acc_off_h[meta[i].blk + 1] - acc_off_h[meta[i].blk]);
  }
  const int W = p.W, C = st->C, G = (W + 63) / 64;
  st->G = G;
  ScanDev &sd = st->sd;
  sd.C = C;
  sd.G = G;
  sd.fslots = st->fslots;
  sd.bslots = st->bslots;
  sd.keep_states = keep_states;
  bool ok = true;
  auto chk = [&](const void *x) { ok = ok && x; };
  chk(sd.meta = st->up(meta));
  chk(sd.loops = st->up(loops));
  chk(sd.chunks = st->up(chunks));
  chk(sd.csrc = st->up(csrc));
  chk(sd.fin_slot = st->up(fin_slot));
  std::vector<int32_t> fin_ent(g.fin_ent.begin(), g.fin_ent.end());
  chk(sd.fin_ent = st->up(fin_ent));
  chk(sd.out_slot = st->up(out_slot));
  chk(sd.out_pos = st->up(out_pos));
  chk(sd.lat_slot = st->up(lat_slot));
  chk(sd.bend_loop = st->up(bend_loop));
  chk(sd.srcent = st->up(srcent));
  const int max_slots = std::max(st->fslots, st->bslots);
  const int extra = std::max(0, max_slots - SH_SLOTS);
  sd.spill_stride = extra * 4 * 64;  // room for up to 4 planes
  chk(sd.spill = st->alloc<uint64_t>((size_t)std::max(1, sd.spill_stride) * C * G));
  chk(sd.gsum = st->alloc<uint64_t>((size_t)2 * C * W));
  chk(sd.psum = st->alloc<uint64_t>((size_t)2 * C * W));
  chk(sd.carry = st->alloc<uint64_t>((size_t)2 * C * W));
  chk(sd.hp_src = st->alloc<uint64_t>((size_t)std::max(1, g.K) * W));
  chk(sd.d_src = st->alloc<uint64_t>((size_t)std::max(1, g.K) * W));
  st->n_csrc = (int)csrc.size();
  chk(sd.xval = st->alloc<uint64_t>((size_t)std::max(1, st->n_csrc) * W));
  // record streams: one per apply warp, then one per crossing warp
  st->n_apply_streams = C * G;
  st->n_streams = 2 * C * G;
  sd.n_streams = st->n_streams;
  st->h_rec_cap.assign(st->n_streams, 0);
  for (int c = 0; c < C; ++c)
    for (int wg = 0; wg < G; ++wg) {
      const int len = chunks[c].e - chunks[c].s;
      st->h_rec_cap[c * G + wg] = 64 + len;
      st->h_rec_cap[C * G + c * G + wg] = 8 + 2 * chunks[c].carry_cnt * 64;
    }
  chk(st->d_rec_cap = st->alloc<int32_t>(st->n_streams));
  chk(st->d_rec_base = st->alloc<int32_t>(st->n_streams));
  chk(sd.rec_cnt = st->alloc<int32_t>(st->n_streams + 1));
  chk(st->offs = st->alloc<int32_t>(st->n_streams + 1));
  chk(st->init = st->alloc<uint64_t>((size_t)W));
  if (ok) ok = scan_set_streams(st);
  sd.rec_cap = st->d_rec_cap;
  sd.rec_base = st->d_rec_base;
  if (!ok) {
    if (err) *err = "device allocation for the scan solver failed";
    delete st;
    return nullptr;
  }
  set_smem(k_fwd_chain<K_HP, M_SUM>, 4 * (SH_SLOTS * 2 * 64 + 128) * 8);
  set_smem(k_fwd_chain<K_D, M_SUM>, 4 * (SH_SLOTS * 2 * 64 + 128) * 8);
  set_smem(k_fwd_chain<K_H, M_SUM>, 4 * (SH_SLOTS * 2 * 64 + 128) * 8);
  set_smem(k_fwd_chain<K_HP, M_APPLY>, 4 * (SH_SLOTS * 1 * 64 + 128) * 8);
  set_smem(k_fwd_chain<K_D, M_APPLY>, 4 * (SH_SLOTS * 1 * 64 + 128) * 8);
  set_smem(k_fwd_chain<K_H, M_APPLY>, 4 * (SH_SLOTS * 1 * 64 + 128) * 8);
  set_smem(k_bwd_chain<M_SUM>, 4 * (SH_SLOTS * 4 * 64) * 8);
  set_smem(k_bwd_chain<M_APPLY>, 4 * (SH_SLOTS * 2 * 64) * 8);
  set_smem(k_bwd_chain<M_LANT>, 4 * (SH_SLOTS * 2 * 64) * 8);
  return st;
}

// After a run whose record streams overflowed: size every stream to what
// it needed (plus slack).  Returns false on allocation failure.
bool scan_grow_streams(ScanState *st) {
  std::vector<int32_t> cnt(st->n_streams);
  if (cudaMemcpy(cnt.data(), st->sd.rec_cnt, sizeof(int32_t) * st->n_streams, cudaMemcpyDeviceToHost) != cudaSuccess)
    return false;
  for (int i = 0; i < st->n_streams; ++i)
    if (cnt[i] > st->h_rec_cap[i]) st->h_rec_cap[i] = cnt[i] + cnt[i] / 4 + 16;
  return scan_set_streams(st);
}

#define PROF(name) if (pf) pf->mark(s, name)

static int run_emission_tail(ScanState *st, const DevPlan &p, cudaStream_t s, Prof *pf) {
  ScanDev &sd = st->sd;
  int32_t *offs = st->offs;
  const int nw = sd.C * sd.G;
  PROF("cross_emit");
  k_cross_emit<<<grid_of((long long)nw * 32, 128), 128, 0, s>>>(p, sd, st->n_apply_streams);
  PROF("streams_prefix");
  k_streams_prefix<<<1, 1024, 0, s>>>(sd, offs, p.status);
  PROF("streams_copy");
  k_streams_copy<<<grid_of((long long)sd.n_streams * 32, 256), 256, 0, s>>>(sd, offs, p.xfer, p.xfer_cap);
  return 3;
}

int enqueue_scan_solver(ScanState *st, const DevPlan &p, cudaStream_t s, Prof *pf) {
  ScanDev &sd = st->sd;
  const int W = p.W, nw = sd.C * sd.G;
  const int wpc = 4;  // warps per CTA
  const int grid = (nw + wpc - 1) / wpc;
  uint64_t *init = st->init;
  int n = 0;
  const size_t sm1 = wpc * (SH_SLOTS * 1 * 64 + 128) * 8, sm2 = wpc * (SH_SLOTS * 2 * 64 + 128) * 8;
  const size_t smb4 = wpc * (SH_SLOTS * 4 * 64) * 8, smb2 = wpc * (SH_SLOTS * 2 * 64) * 8;
  cudaMemsetAsync(p.acc_flag, 0, (size_t)p.A, s);
  // ---- anticipation and liveness (backward)
  PROF("ant_summary");
  k_bwd_chain<M_SUM><<<grid, 128, smb4, s>>>(p, sd); ++n;
  PROF("ant_scan");
  k_scan_carry<<<grid_of(2 * W, 128), 128, 0, s>>>(sd, W, 2, 1, nullptr, nullptr); ++n;
  PROF("ant_apply");
  k_bwd_chain<M_APPLY><<<grid, 128, smb2, s>>>(p, sd); ++n;
  // ---- loop masks: need within the loop body, kills anywhere in it
  if (p.L) { PROF("loop_masks"); k_bwd_chain<M_LANT><<<grid, 128, smb2, s>>>(p, sd); ++n; }
  // ---- plain host validity
  PROF("entry_stale");
  k_entry_stale<<<grid_of(W, 128), 128, 0, s>>>(p.entry_h, p.top, init, W); ++n;
  PROF("hp_summary");
  k_fwd_chain<K_HP, M_SUM><<<grid, 128, sm2, s>>>(p, sd); ++n;
  PROF("fwd_scan");
  k_scan_carry<<<grid_of(W, 128), 128, 0, s>>>(sd, W, 1, 0, init, init); ++n;
  PROF("hp_apply");
  k_fwd_chain<K_HP, M_APPLY><<<grid, 128, sm1, s>>>(p, sd); ++n;
  if (p.K) { PROF("edge_const"); k_scan_edge_const<<<grid_of((long long)p.K * W, 256), 256, 0, s>>>(p, sd, 0); ++n; }
  // ---- device validity
  PROF("entry_stale");
  k_entry_stale<<<grid_of(W, 128), 128, 0, s>>>(p.entry_d, p.top, init, W); ++n;
  PROF("d_summary");
  k_fwd_chain<K_D, M_SUM><<<grid, 128, sm2, s>>>(p, sd); ++n;
  PROF("fwd_scan");
  k_scan_carry<<<grid_of(W, 128), 128, 0, s>>>(sd, W, 1, 0, init, init); ++n;
  PROF("d_apply");
  k_fwd_chain<K_D, M_APPLY><<<grid, 128, sm1, s>>>(p, sd); ++n;
  if (p.K) { PROF("edge_const"); k_scan_edge_const<<<grid_of((long long)p.K * W, 256), 256, 0, s>>>(p, sd, 1); ++n; }
  // ---- host validity and emission
  PROF("entry_stale");
  k_entry_stale<<<grid_of(W, 128), 128, 0, s>>>(p.entry_h, p.top, init, W); ++n;
  PROF("h_summary");
  k_fwd_chain<K_H, M_SUM><<<grid, 128, sm2, s>>>(p, sd); ++n;
  PROF("fwd_scan");
  k_scan_carry<<<grid_of(W, 128), 128, 0, s>>>(sd, W, 1, 0, init, init); ++n;
  PROF("h_apply_emit");
  k_fwd_chain<K_H, M_APPLY><<<grid, 128, sm1, s>>>(p, sd); ++n;
  n += run_emission_tail(st, p, s, pf);
  return n;
}

int enqueue_scan_edges(ScanState *st, const DevPlan &p, cudaStream_t s, Prof *pf) {
  // after the record buffers grew: redo the host-validity apply pass and the gather
  ScanDev &sd = st->sd;
  const int nw = sd.C * sd.G, wpc = 4, grid = (nw + wpc - 1) / wpc;
  const size_t sm1 = wpc * (SH_SLOTS * 1 * 64 + 128) * 8;
  PROF("h_apply_emit");
  k_fwd_chain<K_H, M_APPLY><<<grid, 128, sm1, s>>>(p, sd);
  return 1 + run_emission_tail(st, p, s, pf);
}

void scan_destroy(ScanState *st) { delete st; }

long long scan_h2d_bytes(const ScanState *st) { return st ? st->h2d : 0; }

}  // namespace ompdart
