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
//   summary  (one warp per chunk and 64-variable word group: the chunk's
//            map and every position's affine pair),
//   scan     (compose the maps over the chunks: every chunk's carry),
//   resolve  (every position's pair with its carry: the final plane),
// and the emission reads the final planes.  Inside a chunk the warp walks
// positions in order.  A loop body is a contiguous run starting at its
// header; its header's value has a closed form (entry | what the body
// contributes along its back edges: Kam-Ullman rapidity), so the forward
// walks take every body once relative to the header's value and compose
// at its end, and the backward walks take their outermost open loops once
// with extra planes for the header's value (deeper loops are walked again
// when their header's value grew).  Values a later position still needs
// live in slots assigned on the host by interval colouring (a few in
// shared memory, the rest spilled to global scratch).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <queue>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "ingest.h"
#include "parallel.h"
#include "plan.cuh"
#include "solver.h"

namespace ompdart {

namespace {

constexpr int CARRY = -2;      // slot id: the chunk's incoming carry
constexpr int PREV = -3;       // slot id: the value of the position walked just before
constexpr int BACK = -4;       // slot id (forward in-edges): a back edge, closed at the loop's end
// Occupancy of the chain kernels (latency-bound walks: more warps per SM
// help until registers spill).  They are compiled for at most 4 warps per
// CTA and at least 6 (forward) / 5 (backward) CTAs per SM, which caps
// registers at 85 and 102 per thread, and keep 128 / 256 shared-memory
// words per warp for slots, so 24 / 20 warps fit on an SM.  Measured on the
// 2^20-block CFG: 16 warps per SM made the host-validity walk 20% slower,
// 7 forward CTAs (73 registers, spilling) 20% slower too; the liveness walk
// loses with 6 CTAs (85 registers) or with no slot in shared memory.
#ifndef OMPDART_FWD_SH_WORDS
#define OMPDART_FWD_SH_WORDS 128
#endif
#ifndef OMPDART_BWD_SH_WORDS
#define OMPDART_BWD_SH_WORDS 256
#endif
#ifndef OMPDART_FWD_MIN_CTAS
#define OMPDART_FWD_MIN_CTAS 6
#endif
#ifndef OMPDART_LANT_SH_WORDS  // the loop-mask walk (four planes): no slot in shared memory, 5 CTAs
#define OMPDART_LANT_SH_WORDS 0
#endif
#ifndef OMPDART_BWD_MIN_CTAS
#define OMPDART_BWD_MIN_CTAS 5
#endif
#ifndef OMPDART_MAX_WPC
#define OMPDART_MAX_WPC 4  // warps per CTA a chain kernel is compiled for at most
#endif
constexpr int FWD_SH_WORDS = OMPDART_FWD_SH_WORDS;  // shared-memory words per warp for slots
constexpr int BWD_SH_WORDS = OMPDART_BWD_SH_WORDS;
constexpr int WPC = 4;         // warps per CTA of the chain kernels
constexpr int MAX_DEPTH = 31;  // loop nesting depth the chain handles
// bound on loop re-runs per chunk walk: each loop of a reducible CFG needs
// at most one re-run per entry, so 8 per position is far beyond any valid
// walk; hitting it reports OMPDART_E_NOCONVERGE instead of spinning
__host__ __device__ inline int rerun_cap(int len) { return 8 * len + 64; }

enum PhaseKind { K_ANT = 0, K_HP = 1, K_D = 2, K_H = 3 };
// summary walk (liveness); its complement problem for eager `to'
// placement (not anticipated by a device read: ~AntDm); loop-restricted
// anticipation (the loop masks)
enum ModeKind { M_SUM = 0, M_NA = 1, M_LANT = 2 };

struct PosMeta {  // one per position, 80 B
  int32_t blk;
  int32_t fin_beg, out_beg, acc_beg, srcent_beg, bend_beg;  // acc_beg: in caller order
  int16_t nfin, nout, nacc, nsrcent, nbend, fslot, bslot;
  int16_t bend_depth;     // the first (outermost) loop ending here: its depth,
  int32_t head_loop;      // loop whose header is this position, else -1
  int32_t bend_ph;        // header position,
  int32_t exit_idx;       // index in exit_blocks, else -1
  int32_t pacc_beg;       // first access of the block in position order
  int32_t flags;          // PM_RECORDS: the block's summary records are given
  int32_t bend_pend;      // body end and header slot (the backward walks read
                          // them here instead of from bend_info)
  // a header position: its loop's body end, header slot and depth (kept
  // here so the walks need no loop record at a header)
  int32_t head_pend;
  int16_t head_hslot, head_depth;
  int32_t pad6;
  int16_t bend_hslot, pad5;
};
// a block with call pseudo-accesses: its entries in the position-ordered
// access stream are already summary records (folded on the host with the
// callees' rows), and its access flags come from the call-site pass
constexpr int32_t PM_RECORDS = 1;
constexpr int32_t LINK_RECORD = -2;
static_assert(sizeof(PosMeta) == 80, "PosMeta layout");

struct LoopMeta {
  int32_t ph, pend;   // body = positions [ph, pend)
  int16_t hslot, depth;
  int32_t lat_beg;    // latch slots (forward): their values close the loop
  int32_t lat_cnt;
  int32_t cfg;        // the CFG of a batch it belongs to
  int32_t xs_beg;     // forward slots read after the body ends (exit sources)
  int32_t xs_cnt;
};

struct ChunkMeta {
  int32_t s, e;             // positions [s, e)
  int32_t carry_beg, carry_cnt;
  int32_t loop_beg, loop_end;
  int32_t cfg;              // which CFG of a batch the chunk belongs to
  int32_t flags;            // CH_FIRST / CH_LAST: first / last chunk of its CFG
};
constexpr int32_t CH_FIRST = 1, CH_LAST = 2;

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
  const int2 *fin_pk;   // per forward in-edge {source slot or CARRY, loop-entry edge or -1}
  const int2 *out_pk;   // per backward out-edge {target slot or CARRY, target position}
  const uint32_t *acc_p;  // accesses in position order
  uint32_t *rec_p;        // summary records in position order
  uint32_t *emit_p;       // per access in position order: variable | flag table << 24 (flag_table)
  const int2 *acc_link;   // per access: {first access of its variable in the block, next one or -1};
                          // {LINK_RECORD, -1}: the entry is a given summary record
  long long n_acc_p;      // entries of the position-ordered access stream
  int sh_slots;           // slots per plane held in shared memory
  const int32_t *lat_slot;
  const int32_t *lat_ent;   // edge-constant entry of each latch's back edge, or -1
  const int32_t *exit_slot;  // per loop (xs_beg, xs_cnt): forward slots of its exit sources
  const int4 *bend_info;  // per loop ending at a position: {depth, header position, body end, header's backward slot}
  const int32_t *srcent;
  uint64_t *spill;     // per warp spill area
  int spill_stride;    // words per warp
  uint64_t *gsum, *psum;   // [planes][C][W] chunk maps
  uint64_t *carry;         // [planes][C][W] carry into each chunk
  uint64_t *seg_g, *seg_p;  // [S][W] maps of the scan's segments (one region per branch of a run)
  int seg_n;                // segments per word column of the chunk-carry scan
  uint64_t *d_src;  // [K][W] device validity at loop-entry sources
  // affine pairs the summary walks leave per position: value = G | (carry & P)
  // with the carry into the position's chunk (resolved by k_resolve_*)
  uint64_t *pair_g, *pair_p;    // [N][W] by block: Live_in, later H_out stale
  uint64_t *pair_gd, *pair_pd;  // [N][W] D_in stale (the device phase runs beside liveness)
  uint64_t *pair_g2, *pair_p2;  // [N][W] D_out stale (kept states only), else null
  // liveness walks an outermost loop once, with a third plane: the part of
  // a body position's value that comes from the header's own value A
  // (Live = G | (carry & P) | (A & PA)); at the header A's fixed point goes
  // to hdrl_* and the resolve folds it in
  uint64_t *pair_a;             // [N][W] PA of positions inside a loop
  uint64_t *hdrl_g, *hdrl_p;    // [L][W] liveness at an outermost loop's header (pair of the carry)
  // a loop one level down is closed the same way with a fourth plane, the
  // coefficient of its own header value A2: at its header A2 (a triple of
  // the carry and A) goes to hdrl2_*; deeper loops are walked again until
  // their header values stop changing
  uint64_t *pair_a2;                     // [N][W] PA2 of positions inside a second-level loop
  uint64_t *hdrl2_g, *hdrl2_p, *hdrl2_a;  // [L][W] A2 = G | (carry & P) | (A & PA) at its header
  const int32_t *loop_d2;       // [L] second-level loop holding loop l (itself at that level), or -1
  uint64_t *src_g, *src_p;      // [K][W] out value at each loop-entry edge's source
  const int32_t *pos_chunk;     // [M] chunk of each position
  // forward walks take each loop body once, relative to the header's value;
  // at the loop's end the header's fixed point (relative to the enclosing
  // level) goes to hdr_*, and the resolve composes up the loop tree
  uint64_t *hdr_g, *hdr_p;      // [L][W] header value, plane at 0 / at top of the enclosing level
  uint64_t *hdr_ag, *hdr_ap;    // [L][W] the same composed up the loop tree: a pair of the chunk's carry
  const int32_t *pos_loop;      // [M] innermost loop holding each position, or -1
  const int32_t *loop_up;       // [L] enclosing loop, or -1
  const int32_t *loop_root;     // [L] outermost loop holding it
  const int32_t *src_pos;       // [K] position of each loop-entry edge's source
  const int2 *emit_rng;         // [n_emit] position ranges of the emission items (within one chunk)
  int n_emit;
  int32_t *rec_cnt;    // [streams]
  const int32_t *rec_base, *rec_cap;  // [streams]
  EdgeXfer *stream;    // record streams
  int n_streams;
  int keep_states;
  const int32_t *work;  // [C] chunks by decreasing cost: the order warps take them in
  const int32_t *lant_work;  // [L] loops by decreasing body length (loop-mask walks)
  int n_loops;
  int32_t *queue;       // [Q_SLOTS] work-queue heads, one per chain launch of a run
  int32_t *cfg_err;     // [n_cfg] set to 1 for a CFG whose walk hit the re-run cap, or null
};
constexpr int Q_SLOTS = 16;

// ---- host side: per-chunk metadata and slot colouring -------------------------------

struct Interval {
  int a, b, id;
};

// Host arrays that are written in full by parallel passes: resize leaves
// them uninitialised, so their pages are first touched by the threads
// that fill them.
template <class T>
struct DefaultInit : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = DefaultInit<U>;
  };
  DefaultInit() = default;
  template <class U>
  DefaultInit(const DefaultInit<U> &) {}
  template <class U>
  void construct(U *p) {
    ::new (static_cast<void *>(p)) U;
  }
  template <class U, class... A>
  void construct(U *p, A &&...a) {
    ::new (static_cast<void *>(p)) U(std::forward<A>(a)...);
  }
};
template <class T>
using HostVec = std::vector<T, DefaultInit<T>>;

// Interval colouring: intervals sharing no position may share a slot
// (lowest free slot first).  The heaps are the caller's scratch.
struct Colouring {
  std::vector<std::pair<int, int>> active;  // min-heap of (end, slot)
  std::vector<int> freeq;                   // min-heap of free slots
  int run(std::vector<Interval> &iv, std::vector<int32_t> &slot_of) {
    std::sort(iv.begin(), iv.end(), [](const Interval &x, const Interval &y) { return x.a < y.a; });
    active.clear();
    freeq.clear();
    const std::greater<> gt;
    int n = 0;
    for (const Interval &x : iv) {
      while (!active.empty() && active.front().first < x.a) {
        freeq.push_back(active.front().second);
        std::push_heap(freeq.begin(), freeq.end(), gt);
        std::pop_heap(active.begin(), active.end(), gt);
        active.pop_back();
      }
      int s;
      if (freeq.empty()) {
        s = n++;
      } else {
        s = freeq.front();
        std::pop_heap(freeq.begin(), freeq.end(), gt);
        freeq.pop_back();
      }
      slot_of[x.id] = s;
      active.push_back({x.b, s});
      std::push_heap(active.begin(), active.end(), gt);
    }
    return n;
  }
};


}  // namespace

// launch shape of one persistent chain kernel
struct ChainShape {
  int grid = 1, wpc = 4, sh_slots = 0;
  size_t smem = 0;
};
enum ChainKind { CK_BSUM, CK_BLANT, CK_FSUM, CK_BNA, CK_COUNT };

struct ScanState {
  int C = 0, G = 0, fslots = 0, bslots = 0, n_streams = 0;
  ChainShape shape[CK_COUNT];
  long long total_cap = 0;
  long long h2d = 0;
  std::vector<void *> allocs;
  ScanDev sd{};
  std::vector<int32_t> h_rec_cap;  // host copy of capacities
  int32_t *d_rec_cap = nullptr, *d_rec_base = nullptr;
  int32_t *offs = nullptr;         // stream offsets in the gathered result
  int32_t *part = nullptr;         // per-CTA sums of the stream prefix
  std::vector<int32_t> chunk_item0;  // [C+1] first emission item of each chunk
  uint64_t *init = nullptr;        // [W] stale set entering the first chunk
  EdgeXfer *stream_buf = nullptr;
  long long bytes = 0;  // device bytes held
  // a run forks: loop masks and liveness on two side streams beside the
  // plain-host / device / host pipeline on the caller's stream (their walks'
  // tails overlap); each branch has its own spill region and chunk maps
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  size_t spill_region = 0;  // words per branch
  // eager `to' placement: the not-anticipated walk (~AntDm) keeps its own
  // pairs, header values and chunk maps (it runs beside liveness)
  bool eager = false;
  uint64_t *na_pg = nullptr, *na_pp = nullptr, *na_pa = nullptr, *na_pa2 = nullptr;
  uint64_t *na_hg = nullptr, *na_hp = nullptr, *na_h2g = nullptr, *na_h2p = nullptr, *na_h2a = nullptr;
  ~ScanState() {
    for (cudaStream_t x : side)
      if (x) cudaStreamDestroy(x);
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    for (void *p : allocs) dev_free(p);
  }
  template <class T>
  T *alloc(size_t n) {
    const size_t b = std::max<size_t>(n, 1) * sizeof(T);
    void *p = dev_malloc(b);
    if (!p) return nullptr;
    allocs.push_back(p);
    bytes += (long long)b;
    return (T *)p;
  }
  template <class T, class A>
  T *up(const std::vector<T, A> &v) {
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

// host threads of the plan builder's parallel passes (each pass takes no
// more than the machine has, and one per a few thousand items).  Batches
// build their arenas on parallel threads already: 16 here made the
// 2,000-function program 35% slower end to end and the single large CFG
// no faster beyond the host's noise
#ifndef OMPDART_HOST_THREADS
#define OMPDART_HOST_THREADS 8
#endif
constexpr int kHostThreads = OMPDART_HOST_THREADS;

bool build_meta(const Ingest &g, int target, ScanState *st, HostVec<PosMeta> &meta, std::vector<LoopMeta> &loops,
                std::vector<ChunkMeta> &chunks, std::vector<CarrySrc> &csrc, HostVec<int32_t> &fin_slot,
                HostVec<int32_t> &out_slot, HostVec<int32_t> &out_pos, std::vector<int32_t> &lat_slot,
                std::vector<int32_t> &lat_ent, std::vector<int32_t> &bend_loop, std::vector<int32_t> &srcent,
                std::vector<int32_t> &exit_slot, std::string *err) {
  Ingest &gm = const_cast<Ingest &>(g);
  make_chunks(&gm, target);
  const int M = g.M, C = (int)g.chunk_off.size() - 1, L = g.L;
  meta.resize(M);  // every record is written by the per-position pass
  loops.assign(L, LoopMeta{});
  chunks.assign(C, ChunkMeta{});
  std::vector<int32_t> head_loop_of_pos(M, -1);
  for (int l = 0; l < L; ++l) head_loop_of_pos[g.pos[g.loop_head[l]]] = l;
  std::vector<int32_t> exit_idx(g.N, -1);
  for (size_t x = 0; x < g.exit_blocks.size(); ++x) exit_idx[g.exit_blocks[x]] = (int32_t)x;
  // loop-entry edges by source block, loops ending at each position (outer
  // first): both as offset lists
  std::vector<int32_t> ebs_off(g.N + 1, 0), ebs(g.K), end_off(M + 1, 0), end_l(L);
  for (int k = 0; k < g.K; ++k) ebs_off[g.ent_src[k] + 1]++;
  for (int b = 0; b < g.N; ++b) ebs_off[b + 1] += ebs_off[b];
  {
    std::vector<int32_t> f(ebs_off.begin(), ebs_off.end() - 1);
    for (int k = 0; k < g.K; ++k) ebs[f[g.ent_src[k]]++] = k;
  }
  for (int l = 0; l < L; ++l) end_off[g.loop_end[l]]++;
  for (int i = 0; i < M; ++i) end_off[i + 1] += end_off[i];
  {
    std::vector<int32_t> f(end_off.begin(), end_off.end() - 1);
    for (int l = 0; l < L; ++l) end_l[f[g.loop_end[l] - 1]++] = l;
    for (int i = 0; i < M; ++i)
      if (end_off[i + 1] - end_off[i] > 1)
        std::sort(end_l.begin() + end_off[i], end_l.begin() + end_off[i + 1],
                  [&](int a, int b) { return g.loop_depth[a] < g.loop_depth[b]; });
  }
  bend_loop.assign(end_l.begin(), end_l.end());

  // positions the backward walks may jump to (a loop body walked again):
  // the last body position.  Only at other positions is "the position
  // walked just before" the neighbouring one.  The forward walks take every
  // position once, in order.
  std::vector<uint8_t> bwd_target(M, 0);
  for (int l = 0; l < L; ++l) bwd_target[g.loop_end[l] - 1] = 1;
  // every entry of these is written by the per-chunk passes below
  fin_slot.resize(g.fin_src.size());
  out_slot.resize(g.out_dst.size());
  out_pos.resize(g.out_dst.size());
  HostVec<int32_t> fslot(M), bslot(M), hslot(L);
  // loop containing a block but not another: outermost such
  auto contains = [&](int l, int p) { return p >= g.pos[g.loop_head[l]] && p < g.loop_end[l]; };
  auto outermost = [&](int l) {
    while (g.loop_parent[l] >= 0) l = g.loop_parent[l];
    return l;
  };
  // ---- per chunk: slots by interval colouring (chunks are independent)
  struct alignas(128) ChunkScratch {  // one per thread, on cache lines of its own
    std::vector<Interval> iv;
    std::vector<int32_t> loc_loops, so, sb;
    Colouring col;
    int max_f = 0, max_b = 0;
    bool bad = false;
  };
  auto colour_chunk = [&](int c, ChunkScratch &x) {
    const int s = g.chunk_off[c], e = g.chunk_off[c + 1];
    ChunkMeta &cm = chunks[c];
    cm.s = s;
    cm.e = e;
    cm.cfg = (int32_t)(std::upper_bound(g.cfg_pos_off.begin(), g.cfg_pos_off.end(), s) - g.cfg_pos_off.begin()) - 1;
    cm.flags = (s == g.cfg_pos_off[cm.cfg] ? CH_FIRST : 0) | (e == g.cfg_pos_off[cm.cfg + 1] ? CH_LAST : 0);
    // ---- forward values
    std::vector<Interval> &iv = x.iv;
    iv.clear();
    const int nval = e - s;  // ids: [0, nval) positions, [nval, nval + nloops) header in-values
    int lb = L, le = -1;
    for (int i = s; i < e; ++i) {
      const int b = g.order[i];
      int a = i, z = -1;
      for (int k = g.out_off[i]; k < g.out_off[i + 1]; ++k) {
        const int pt = g.pos[g.out_dst[k]];
        if (pt == i + 1 && pt < e) continue;  // read from registers
        if (pt >= e) {
          z = std::max(z, e);
        } else if (pt > i) {
          z = std::max(z, pt);
        } else {  // a latch: read when its loop closes, at the body's last position
          const int l = head_loop_of_pos[pt];
          if (l < 0) {
            x.bad = true;
            return;
          }
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
    std::vector<int32_t> &loc_loops = x.loc_loops;
    loc_loops.clear();
    if (le >= 0)
      for (int l = lb; l <= le; ++l) {
        loc_loops.push_back(l);
        iv.push_back({g.pos[g.loop_head[l]], g.loop_end[l] - 1, nval + (int)loc_loops.size() - 1});
      }
    cm.loop_beg = le >= 0 ? lb : 0;
    cm.loop_end = le >= 0 ? le + 1 : 0;
    std::vector<int32_t> &so = x.so;
    so.assign(nval + loc_loops.size(), -1);
    x.max_f = std::max(x.max_f, x.col.run(iv, so));
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
        if (pp == i - 1 && i < e && !bwd_target[pp]) continue;  // read from registers
        if (pp < i) {
          int lo = pp;
          for (int x = g.inner_loop[p]; x >= 0; x = g.loop_parent[x]) {
            if (contains(x, i)) break;
            lo = std::min(lo, g.pos[g.loop_head[x]]);
          }
          a = std::min(a, lo);
          z = std::max(z, i);
        } else {
          // the header's value, read by its latches, survives re-entries
          const int lo = outermost(head_loop_of_pos[i]);
          a = std::min(a, g.pos[g.loop_head[lo]]);
          z = std::max(z, g.loop_end[lo] - 1);
        }
      }
      (void)b;
      if (z >= 0) iv.push_back({a, z, i - s});
    }
    std::vector<int32_t> &sb = x.sb;
    sb.assign(nval, -1);
    x.max_b = std::max(x.max_b, x.col.run(iv, sb));
    for (int i = s; i < e; ++i) bslot[i] = sb[i - s];
  };
  int max_f = 0, max_b = 0;
  {
    std::vector<ChunkScratch> xs(kHostThreads);  // one per thread of the pass below
    parallel_ranges(C, 256, kHostThreads, [&](int t, int lo, int hi) {
      for (int c = lo; c < hi && !xs[t].bad; ++c) colour_chunk(c, xs[t]);
    });
    for (const ChunkScratch &x : xs) {
      if (x.bad) {
        if (err) *err = "retreating edge into a non-header";
        return false;
      }
      max_f = std::max(max_f, x.max_f);
      max_b = std::max(max_b, x.max_b);
    }
  }
  // ---- per position records (positions independent: loop-entry sources
  // by block in position order via an offset list)
  std::vector<int32_t> src_off(M + 1, 0);
  for (int i = 0; i < M; ++i) src_off[i + 1] = src_off[i] + ebs_off[g.order[i] + 1] - ebs_off[g.order[i]];
  srcent.resize(src_off[M]);
  parallel_ranges(M, 1 << 14, kHostThreads, [&](int, int lo, int hi) {
    for (int i = lo; i < hi; ++i) {
      const int b = g.order[i];
      PosMeta &m = meta[i];
      m = PosMeta{};
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
      m.srcent_beg = src_off[i];
      std::copy(ebs.begin() + ebs_off[b], ebs.begin() + ebs_off[b + 1], srcent.begin() + src_off[i]);
      m.nsrcent = (int16_t)(src_off[i + 1] - src_off[i]);
      m.bend_beg = end_off[i];
      m.nbend = (int16_t)(end_off[i + 1] - end_off[i]);
      if (m.nbend) {
        const int l = end_l[end_off[i]], ph = g.pos[g.loop_head[l]];
        m.bend_depth = (int16_t)g.loop_depth[l];
        m.bend_ph = ph;
        m.bend_pend = g.loop_end[l];
        m.bend_hslot = (int16_t)bslot[ph];
      }
    }
  });
  // ---- edge entries per chunk, then the carry sources (edges into the
  // next chunk's first position from this chunk), counted first
  std::vector<int32_t> cs_off(C + 1, 0);
  parallel_ranges(C, 256, kHostThreads, [&](int, int lo, int hi) {
    for (int c = lo; c < hi; ++c) {
      const int s = chunks[c].s, e = chunks[c].e;
      for (int i = s; i < e; ++i) {
        for (int k = g.fin_off[i]; k < g.fin_off[i + 1]; ++k) {
          const int pp = g.pos[g.fin_src[k]];
          fin_slot[k] = pp < s ? CARRY : pp >= i ? BACK : pp == i - 1 ? PREV : fslot[pp];
        }
        for (int k = g.out_off[i]; k < g.out_off[i + 1]; ++k) {
          const int pt = g.pos[g.out_dst[k]];
          out_pos[k] = pt;
          out_slot[k] = pt >= e ? CARRY : (pt == i + 1 && !bwd_target[i]) ? PREV : bslot[pt];
        }
      }
      int n = 0;
      if (e < M)
        for (int k = g.fin_off[e]; k < g.fin_off[e + 1]; ++k) n += g.pos[g.fin_src[k]] < e;
      cs_off[c + 1] = n;
    }
  });
  for (int c = 0; c < C; ++c) cs_off[c + 1] += cs_off[c];
  csrc.resize(cs_off[C]);
  for (int c = 0; c < C; ++c) {
    const int e = chunks[c].e;
    chunks[c].carry_beg = cs_off[c];
    chunks[c].carry_cnt = cs_off[c + 1] - cs_off[c];
    int q = cs_off[c];
    if (e < M)
      for (int k = g.fin_off[e]; k < g.fin_off[e + 1]; ++k) {
        const int pp = g.pos[g.fin_src[k]];
        if (pp < e) csrc[q++] = CarrySrc{fslot[pp], g.fin_ent[k], k, 0};
      }
  }
  // ---- per loop: its record, latch slots and exit sources (loops
  // independent: counted, then written at their offsets, in parallel)
  auto loop_lists = [&](int l, std::vector<int32_t> &lat, std::vector<int32_t> &lent, std::vector<int32_t> &xs) {
    const int ph = g.pos[g.loop_head[l]], pend = g.loop_end[l];
    lat.clear();
    lent.clear();
    xs.clear();
    for (int k = g.fin_off[ph]; k < g.fin_off[ph + 1]; ++k) {
      const int pp = g.pos[g.fin_src[k]];
      if (pp >= ph && std::find(lat.begin(), lat.end(), fslot[pp]) == lat.end()) {
        lat.push_back(fslot[pp]);
        lent.push_back(g.fin_ent[k]);  // the back edge's constant entry (eager placement), else -1
      }
    }
    // exit sources: body positions whose value is read from their slot
    // outside the body: after it (or as the next chunk's carry), or at an
    // enclosing loop's end (a back edge to an enclosing header)
    const int ce = chunks[std::upper_bound(g.chunk_off.begin(), g.chunk_off.end(), ph) - g.chunk_off.begin() - 1].e;
    for (int q = ph; q < pend; ++q) {
      if (fslot[q] < 0) continue;
      bool read_after = false;
      for (int k = g.out_off[q]; k < g.out_off[q + 1] && !read_after; ++k) {
        const int pt = g.pos[g.out_dst[k]];
        read_after = (pt >= pend || pt < ph) && (pt >= ce || pt != q + 1);
      }
      if (read_after) xs.push_back(fslot[q]);
    }
  };
  {
    std::vector<int32_t> lat_off(L + 1, 0), xs_off(L + 1, 0);
    parallel_ranges(L, 1024, kHostThreads, [&](int, int lo, int hi) {
      std::vector<int32_t> lat, lent, xs;
      for (int l = lo; l < hi; ++l) {
        loop_lists(l, lat, lent, xs);
        lat_off[l + 1] = (int32_t)lat.size();
        xs_off[l + 1] = (int32_t)xs.size();
      }
    });
    for (int l = 0; l < L; ++l) {
      lat_off[l + 1] += lat_off[l];
      xs_off[l + 1] += xs_off[l];
    }
    lat_slot.resize(lat_off[L]);
    lat_ent.resize(lat_off[L]);
    exit_slot.resize(xs_off[L]);
    parallel_ranges(L, 1024, kHostThreads, [&](int, int lo, int hi) {
      std::vector<int32_t> lat, lent, xs;
      for (int l = lo; l < hi; ++l) {
        loop_lists(l, lat, lent, xs);
        std::copy(lat.begin(), lat.end(), lat_slot.begin() + lat_off[l]);
        std::copy(lent.begin(), lent.end(), lat_ent.begin() + lat_off[l]);
        std::copy(xs.begin(), xs.end(), exit_slot.begin() + xs_off[l]);
        LoopMeta &lm = loops[l];
        lm.cfg = (int32_t)(std::upper_bound(g.cfg_pos_off.begin(), g.cfg_pos_off.end(), g.pos[g.loop_head[l]]) -
                           g.cfg_pos_off.begin()) - 1;
        lm.ph = g.pos[g.loop_head[l]];
        lm.pend = g.loop_end[l];
        lm.hslot = (int16_t)hslot[l];
        lm.depth = (int16_t)g.loop_depth[l];
        lm.lat_beg = lat_off[l];
        lm.lat_cnt = lat_off[l + 1] - lat_off[l];
        lm.xs_beg = xs_off[l];
        lm.xs_cnt = xs_off[l + 1] - xs_off[l];
        PosMeta &hm = meta[lm.ph];
        hm.head_pend = lm.pend;
        hm.head_hslot = lm.hslot;
        hm.head_depth = lm.depth;
      }
    });
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

#ifndef OMPDART_WIN
#define OMPDART_WIN 16
#endif
constexpr int WIN = OMPDART_WIN;       // positions per metadata window
constexpr int EDGE_CAP = 8 * WIN;      // edge entries a window holds
constexpr int REC_CAP = 16 * WIN;      // access records a window holds

// Per-warp cache of a run of positions: their metadata, their edge entries
// and their access records (all stored in position order in HBM, so each
// window is a few coalesced loads instead of dependent loads per position).
struct Win {
  PosMeta meta[WIN];
  int2 edge[EDGE_CAP];    // forward: {slot, loop-entry edge}; backward: {slot, target position}
  uint32_t rec[REC_CAP];  // summary records
  int mbase, ws, we, e0, r0, big;
};

struct WinRegs {  // warp-uniform copy of the window bounds
  int mbase = 0, ws = 0, we = 0, e0 = 0, r0 = 0;
  bool big = false;
};

// Load the window containing position i: forward [i, i+WIN) clipped to hi,
// backward (i-WIN, i] clipped to lo; shrunk so its edges and records fit.
// A single position too large for the buffers is read from HBM directly.
// A walk reads each window once: evict-first loads, like the dense rows.
template <bool FWD>
__device__ void load_window(Win &w, WinRegs &r, const ScanDev &sd, int i, int lo, int hi, int lane) {
  const unsigned FULL = 0xffffffffu;
  const int mbase = FWD ? i : max(i - WIN + 1, lo);
  const int n = FWD ? min(WIN, hi - i) : (i + 1 - mbase);
  int eb = 0, ee = 0, rb = 0, re = 0;
  if (lane < n) {
    PosMeta pm;
    {
      const ulonglong2 *src = reinterpret_cast<const ulonglong2 *>(sd.meta + mbase + lane);
      ulonglong2 *dst = reinterpret_cast<ulonglong2 *>(&pm);
#pragma unroll
      for (int u = 0; u < 5; ++u) dst[u] = __ldcs(src + u);
    }
    w.meta[lane] = pm;
    eb = FWD ? pm.fin_beg : pm.out_beg;
    ee = eb + (FWD ? pm.nfin : pm.nout);
    rb = pm.pacc_beg;
    re = rb + pm.nacc;
  }
  const int kcur = FWD ? 0 : n - 1;
  const int ea = __shfl_sync(FULL, FWD ? eb : ee, kcur);
  const int ra = __shfl_sync(FULL, FWD ? rb : re, kcur);
  const bool fits = lane < n && (FWD ? (ee - ea <= EDGE_CAP && re - ra <= REC_CAP)
                                     : (ea - eb <= EDGE_CAP && ra - rb <= REC_CAP));
  const unsigned fm = __ballot_sync(FULL, fits);
  int ws, we;
  if (FWD) {
    const int keep = (~fm == 0u) ? 32 : (__ffs(~fm) - 1);
    ws = i;
    we = i + keep;
  } else {
    const unsigned x = (n == 32) ? fm : (fm << (32 - n));
    const int keep = (~x == 0u) ? 32 : __clz(~x);
    ws = i + 1 - keep;
    we = i + 1;
  }
  const bool big = we == ws;
  if (big) { ws = i; we = i + 1; }
  const int k0 = ws - mbase, k1 = we - 1 - mbase;
  const int e0 = __shfl_sync(FULL, eb, k0), e1 = __shfl_sync(FULL, ee, k1);
  const int r0 = __shfl_sync(FULL, rb, k0), r1 = __shfl_sync(FULL, re, k1);
  if (!big) {
    const int2 *src = FWD ? sd.fin_pk : sd.out_pk;
    for (int j = lane; j < e1 - e0; j += 32) w.edge[j] = __ldcs(src + e0 + j);
    for (int j = lane; j < r1 - r0; j += 32) w.rec[j] = __ldcs(sd.rec_p + r0 + j);
  }
  __syncwarp();
  r.mbase = mbase; r.ws = ws; r.we = we; r.e0 = e0; r.r0 = r0; r.big = big;
}

__device__ __forceinline__ int2 win_edge(const Win &w, const WinRegs &r, const int2 *g, int k) {
  return r.big ? g[k] : w.edge[k - r.e0];
}
__device__ __forceinline__ uint32_t win_rec(const Win &w, const WinRegs &r, const ScanDev &sd, int k) {
  return r.big ? sd.rec_p[k] : w.rec[k - r.r0];
}
struct Lane {
  int lane, wg, w0;     // w0: first of the lane's two words (global word index)
  uint64_t top0, top1;  // valid-variable masks of the two words
};

template <int NP>
struct Slots {
  uint64_t *sh;     // [nsh][NP][64]
  uint64_t *spill;  // [extra][NP][64]
  int nsh;
  __device__ ulonglong2 *at(int slot, int plane, int lane) const {
    if (slot < nsh) return reinterpret_cast<ulonglong2 *>(sh + ((size_t)(slot * NP + plane) * 64) + 2 * lane);
    return reinterpret_cast<ulonglong2 *>(spill + ((size_t)((slot - nsh) * NP + plane) * 64) + 2 * lane);
  }
  // Spilled slots are read back a few positions after they are written:
  // their lines are kept in L1 ahead of the streams (evict-last).
  __device__ ulonglong2 ld(int slot, int plane, int lane) const {
    if (slot < nsh) return *at(slot, plane, lane);
    const size_t g = __cvta_generic_to_global(at(slot, plane, lane));
    ulonglong2 v;
    asm volatile("ld.global.L1::evict_last.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(g) : "memory");
    return v;
  }
  __device__ void st(int slot, int plane, int lane, ulonglong2 v) const {
    if (slot < nsh) {
      *at(slot, plane, lane) = v;
      return;
    }
    const size_t g = __cvta_generic_to_global(at(slot, plane, lane));
    asm volatile("st.global.L1::evict_last.v2.u64 [%0], {%1, %2};" ::"l"(g), "l"(v.x), "l"(v.y) : "memory");
  }
};

__device__ __forceinline__ uint64_t ld_word(const uint64_t *plane, size_t row, int W, int w) {
  return w < W ? plane[row * W + w] : 0ull;
}
__device__ __forceinline__ void st_word(uint64_t *plane, size_t row, int W, int w, uint64_t v) {
  if (w < W) plane[row * W + w] = v;
}
// a lane's two words w, w + 1 (w even) of a row: one 16-byte access when
// both exist and rows are an even number of words (16-byte aligned)
__device__ __forceinline__ ulonglong2 ld_pair(const uint64_t *plane, size_t row, int W, int w) {
  if (!(W & 1) && w + 1 < W) return *reinterpret_cast<const ulonglong2 *>(plane + row * W + w);
  return make_ulonglong2(ld_word(plane, row, W, w), ld_word(plane, row, W, w + 1));
}
__device__ __forceinline__ void st_pair(uint64_t *plane, size_t row, int W, int w, uint64_t a, uint64_t b) {
  if (!(W & 1) && w + 1 < W) {
    *reinterpret_cast<ulonglong2 *>(plane + row * W + w) = make_ulonglong2(a, b);
  } else {
    st_word(plane, row, W, w, a);
    st_word(plane, row, W, w + 1, b);
  }
}
// The same for rows a walk touches once (the dense rows it reads, the pairs
// it writes) and for the emission's rows (Live, D_in and H_in of its
// positions, H_out of their sources, read by a few items at different
// times, so not worth keeping either): evict-first cache hints,
// so that L1 and L2 keep the walks' spilled slots, which are read back a
// few positions later, rather than the streams.  (The resolves, pure
// streams themselves, ran 12% slower with these hints, so they have none.)
#ifndef OMPDART_STREAM_HINTS
#define OMPDART_STREAM_HINTS 1
#endif
__device__ __forceinline__ ulonglong2 ld_stream(const ulonglong2 *a) {
#if OMPDART_STREAM_HINTS
  return __ldcs(a);
#else
  return *a;
#endif
}
__device__ __forceinline__ void st_stream(ulonglong2 *a, ulonglong2 v) {
#if OMPDART_STREAM_HINTS
  __stcs(a, v);
#else
  *a = v;
#endif
}
__device__ __forceinline__ ulonglong2 ld_pair_s(const uint64_t *plane, size_t row, int W, int w) {
  if (!(W & 1) && w + 1 < W) return ld_stream(reinterpret_cast<const ulonglong2 *>(plane + row * W + w));
  return make_ulonglong2(ld_word(plane, row, W, w), ld_word(plane, row, W, w + 1));
}
__device__ __forceinline__ void st_pair_s(uint64_t *plane, size_t row, int W, int w, uint64_t a, uint64_t b) {
  if (!(W & 1) && w + 1 < W) {
    st_stream(reinterpret_cast<ulonglong2 *>(plane + row * W + w), make_ulonglong2(a, b));
  } else {
    st_word(plane, row, W, w, a);
    st_word(plane, row, W, w + 1, b);
  }
}

// Rows of one mask table (64 words each): the affine walks keep [set,
// clear] of the local plane and one `clear' row shared by the coefficient
// planes; the loop-mask walk keeps [set, clear] of H and of D and the
// `clear' rows of their header-value coefficients.
__host__ __device__ constexpr int mask_rows(int np, bool lant) { return lant ? 6 : 3; }

// shared memory per warp (words):
//   slots [nsh][np][64] | mask tables [2][rows][64] | window | kill sets 128 (loop masks only)
// each part a multiple of 16 words (128 B): slots and masks are read and
// written as 16-byte ulonglong2 and must stay 16-byte aligned
constexpr size_t WIN_WORDS = ((sizeof(Win) + 127) / 128) * 16;
__host__ __device__ inline size_t warp_smem_words(int nsh, int np, bool lant) {
  return (size_t)nsh * np * 64 + (size_t)2 * mask_rows(np, lant) * 64 + WIN_WORDS + (lant ? 128 : 0);
}
static_assert(WIN_WORDS % 16 == 0 && WIN_WORDS * 8 >= sizeof(Win), "window layout");
static_assert(alignof(Win) <= 16, "window alignment");

struct WarpMem {
  uint64_t *slots, *tbl, *kill;
  Win *win;
};
template <int NP, bool KILL>
__device__ __forceinline__ WarpMem carve(uint64_t *smem, int warp_in_cta, int nsh) {
  uint64_t *b = smem + (size_t)warp_in_cta * warp_smem_words(nsh, NP, KILL);
  WarpMem m;
  m.slots = b;
  m.tbl = b + (size_t)nsh * NP * 64;
  m.win = reinterpret_cast<Win *>(m.tbl + 2 * mask_rows(NP, KILL) * 64);
  m.kill = KILL ? m.tbl + 2 * mask_rows(NP, KILL) * 64 + WIN_WORDS : nullptr;
  return m;
}

// A block's summary records as set/clear masks: lane r takes record r and
// ORs its bit into the mask table (mask 2*pl = bits the block sets in plane
// pl, 2*pl+1 = bits it clears); the lanes owning the words then apply
// z = (z & ~clear) | set.  Records of one block are for distinct variables,
// so the order of the ORs does not matter.  Building the masks needs
// nothing of the value flowing in, so the walk builds the next position's
// masks while the current value is still being computed.
//   liveness (AntH | AntD share the kill "any write", so their union is one
//   problem): local: read in either space first -> set, else write -> clear;
//   coefficients: both -> clear.  LANT: separate H and D planes, and the
//   block's kills ORed into `kill` ([H|D][64]).
//   forward planes (stale sets): local: GEN -> clear (valid), KILL -> set
//   (stale); coefficient: both -> clear.
// Rows: [set, clear, coefficient clear], LANT [H set, H clear, D set, D
// clear, H coefficient clear, D coefficient clear].
template <int PH, int MODE>
__device__ __forceinline__ void prep_masks(const ScanDev &sd, const Win &w, const WinRegs &wr, const PosMeta &m,
                                           const Lane &L, uint64_t *tb, uint64_t *kill) {
  for (int r = L.lane; r < m.nacc; r += 32) {
    const uint32_t rc = win_rec(w, wr, sd, m.pacc_beg + r);
    if (rc == REC_NONE) continue;
    const int lw = (int)((rc & 0xFFFFFFu) >> 6) - L.wg * 64;
    if ((unsigned)lw >= 64u) continue;
    unsigned long long *t = reinterpret_cast<unsigned long long *>(tb) + lw;
    const unsigned long long bit = 1ull << (rc & 63u);
    if (PH == K_ANT) {
      const bool uh = rc & R_UH, ud = rc & R_UD, df = rc & R_DF;
      if (MODE == M_LANT) {
        if (uh) atomicOr(t, bit); else if (df) atomicOr(t + 64, bit);
        if (ud) atomicOr(t + 128, bit); else if (df) atomicOr(t + 192, bit);
        if (uh || df) atomicOr(t + 256, bit);  // coefficients of the open loop's header value
        if (ud || df) atomicOr(t + 320, bit);
        if (rc & R_KH) atomicOr(reinterpret_cast<unsigned long long *>(kill) + lw, bit);
        if (rc & R_KD) atomicOr(reinterpret_cast<unsigned long long *>(kill) + 64 + lw, bit);
      } else {
        if (MODE == M_NA) {  // not anticipated: a write before any device read sets, a device read clears
          if (!ud && df) atomicOr(t, bit); else if (ud) atomicOr(t + 64, bit);
          if (ud || df) atomicOr(t + 128, bit);
        } else {
          const bool ue = uh || ud;
          if (ue) atomicOr(t, bit); else if (df) atomicOr(t + 64, bit);
          if (MODE == M_SUM && (ue || df)) atomicOr(t + 128, bit);
        }
      }
    } else {
      const uint32_t GEN = PH == K_D ? R_GD : R_GH, KILL = PH == K_D ? R_KD : R_KH;
      if (rc & GEN) atomicOr(t + 64, bit); else if (rc & KILL) atomicOr(t, bit);
      if (MODE == M_SUM && (rc & (GEN | KILL))) atomicOr(t + 128, bit);
    }
  }
}

// apply the lane's words of the prepared masks and clear them
template <int NP, bool LANT>
__device__ __forceinline__ void take_masks(uint64_t *tb, int lane, uint64_t (&z)[NP][2]) {
  ulonglong2 *row = reinterpret_cast<ulonglong2 *>(tb) + lane;  // row r at row[32 * r]
#pragma unroll
  for (int pl = 0; pl < NP; ++pl) {
    // LANT planes: H, D, then their header-value coefficients
    const int rs = LANT ? (pl < 2 ? 2 * pl : -1) : (pl ? -1 : 0);
    const int rc = LANT ? (pl < 2 ? 2 * pl + 1 : 2 + pl) : (pl ? 2 : 1);
    const ulonglong2 a = rs >= 0 ? row[32 * rs] : make_ulonglong2(0ull, 0ull), b = row[32 * rc];
    z[pl][0] = (z[pl][0] & ~b.x) | a.x;
    z[pl][1] = (z[pl][1] & ~b.y) | a.y;
  }
#pragma unroll
  for (int r = 0; r < mask_rows(NP, LANT); ++r) row[32 * r] = make_ulonglong2(0ull, 0ull);
}

// clear the lane's words of a prepared table that will not be used
template <int NP, bool LANT>
__device__ __forceinline__ void drop_masks(uint64_t *tb, int lane) {
#pragma unroll
  for (int r = 0; r < mask_rows(NP, LANT); ++r)
    *reinterpret_cast<ulonglong2 *>(tb + r * 64 + 2 * lane) = make_ulonglong2(0ull, 0ull);
}

// Append the nonzero words of one edge's transfers to the warp's record
// stream (lanes hold words w0, w0 + 1; warp-uniform call).
__device__ __forceinline__ void push_edge_records(const ScanDev &sd, int stream, int &rec_count, int eid, int w0,
                                                  uint64_t to0, uint64_t fr0, uint64_t to1, uint64_t fr1,
                                                  int lane) {
  const bool n0 = (to0 | fr0) != 0, n1 = (to1 | fr1) != 0;
  const unsigned b0 = __ballot_sync(0xffffffffu, n0), b1 = __ballot_sync(0xffffffffu, n1);
  if (!(b0 | b1)) return;
  const unsigned below = (1u << lane) - 1u;
  const int base = rec_count;
  const int cap = sd.rec_cap[stream];
  EdgeXfer *out = sd.stream + sd.rec_base[stream];
  int idx = base + __popc(b0 & below) + __popc(b1 & below);
  if (n0) { if (idx < cap) out[idx] = EdgeXfer{eid, w0, to0, fr0}; ++idx; }
  if (n1) { if (idx < cap) out[idx] = EdgeXfer{eid, w0 + 1, to1, fr1}; }
  rec_count = base + __popc(b0) + __popc(b1);
}

// --------------------------------------------------------------------------------------
// forward chain (Hp, D, H): positions ascending
// --------------------------------------------------------------------------------------
// v relative to a header value h (v = v0 | (h & v1)), h relative to the
// enclosing level: v relative to the enclosing level
template <class T>  // uint64_t or the members of ulonglong2
__device__ __forceinline__ void compose_pair(T &v0, T &v1, uint64_t h0, uint64_t h1) {
  const T a = v0 | (h0 & v1), b = v0 | (h1 & v1);
  v0 = a;
  v1 = b;
}

// End of loop l's body in a forward walk (stale sets grow along paths, so
// the header's value is the least fixed point of h = e | L(h), with e the
// meet of its entry edges and L the latches' values; the latches are
// affine in h, L(h) = A | (h & B), hence h = e | A: Kam-Ullman rapidity
// in closed form).  The body was walked relative to h; the header's value
// is stored for the resolve, and the values still to be read after the
// body (exit sources, the previous position) are re-expressed in the
// enclosing level.
// With eager `to' placement a back edge can carry an edge constant: the
// latch's value enters the header less it (ec, or null).
__device__ __forceinline__ void close_loop(const ScanDev &sd, const Slots<2> &sl, const Lane &L, int W, int l,
                                           int hs, uint64_t (&pv)[2][2], const uint64_t *ec) {
  const LoopMeta lm = sd.loops[l];
  uint64_t a0 = 0, a1 = 0;
  for (int q = 0; q < lm.lat_cnt; ++q) {
    const ulonglong2 v = sl.ld(sd.lat_slot[lm.lat_beg + q], 0, L.lane);
    const int ent = ec ? sd.lat_ent[lm.lat_beg + q] : -1;
    if (ent >= 0) {
      a0 |= v.x & ~ld_word(ec, ent, W, L.w0);
      a1 |= v.y & ~ld_word(ec, ent, W, L.w0 + 1);
    } else {
      a0 |= v.x;
      a1 |= v.y;
    }
  }
  const ulonglong2 e0 = sl.ld(hs, 0, L.lane), e1 = sl.ld(hs, 1, L.lane);
  const uint64_t h00 = e0.x | a0, h01 = e0.y | a1, h10 = e1.x | a0, h11 = e1.y | a1;
  st_pair(sd.hdr_g, l, W, L.w0, h00, h01);
  st_pair(sd.hdr_p, l, W, L.w0, h10, h11);
  for (int q = 0; q < lm.xs_cnt; ++q) {
    const int x = sd.exit_slot[lm.xs_beg + q];
    ulonglong2 v0 = sl.ld(x, 0, L.lane), v1 = sl.ld(x, 1, L.lane);
    compose_pair(v0.x, v1.x, h00, h10);
    compose_pair(v0.y, v1.y, h01, h11);
    sl.st(x, 0, L.lane, v0);
    sl.st(x, 1, L.lane, v1);
  }
  compose_pair(pv[0][0], pv[1][0], h00, h10);
  compose_pair(pv[0][1], pv[1][1], h01, h11);
  __syncwarp();
}

// One warp walks chunk c for the 64-word group wg.
template <int PH>
__device__ __forceinline__ void fwd_walk(const DevPlan &p, const ScanDev &sd, const WarpMem &wm, uint64_t *spill,
                                         int c, int wg) {
  constexpr int NP = 2;  // the chunk's affine map: local plane (carry 0), coefficient plane (carry all)
  constexpr int MODE = M_SUM;
  const int W = p.W;
  Lane L;
  L.lane = threadIdx.x & 31;
  L.wg = wg;
  L.w0 = wg * 64 + 2 * L.lane;
  const uint64_t *tp = p.top + (size_t)sd.chunks[c].cfg * W;  // this CFG's valid-variable mask
  L.top0 = L.w0 < W ? tp[L.w0] : 0;
  L.top1 = L.w0 + 1 < W ? tp[L.w0 + 1] : 0;
  Slots<NP> sl{wm.slots, spill, sd.sh_slots};
  Win &w = *wm.win;
  WinRegs wr;
  wr.ws = wr.we = 0;
  const ChunkMeta cm = sd.chunks[c];
  const uint64_t *ec = PH == K_D ? p.ec_d : p.ec_h;
  // the identity map enters the chunk: (local 0, coefficient all)
  uint64_t cin[NP][2];
  cin[0][0] = cin[0][1] = 0;
  cin[1][0] = L.top0;
  cin[1][1] = L.top1;
  // open loops, innermost last: loop, body end, header slot
  int st_l[MAX_DEPTH + 1], st_pend[MAX_DEPTH + 1], st_hs[MAX_DEPTH + 1];
  int depth = 0;
  uint64_t z[NP][2], zo[NP][2], pv[NP][2] = {};
  int top_pend = -1;  // end of the innermost open loop (warp-uniform)
  constexpr int TBW = mask_rows(NP, false) * 64;  // words of one mask table
  int pbuf = 0, prep_pos = -1;      // table holding the built masks of prep_pos
  drop_masks<NP, false>(wm.tbl, L.lane);   // shared memory starts undefined: the
  drop_masks<NP, false>(wm.tbl + TBW, L.lane);  // masks are built by ORing into zeros
  __syncwarp();
  uint64_t din[2] = {0, 0}, lv[2] = {0, 0};
  uint64_t pdin[2] = {0, 0}, plv[2] = {0, 0};
  int ppos = -1;  // position whose dense rows are prefetched in pdin/plv
  for (int i = cm.s; i < cm.e; ++i) {
    if (i < wr.ws || i >= wr.we) load_window<true>(w, wr, sd, i, cm.s, cm.e, L.lane);
    const PosMeta m = w.meta[i - wr.mbase];
    if (prep_pos != i) {  // masks of this position not built yet (start, window edge)
      if (prep_pos >= 0) {
        drop_masks<NP, false>(wm.tbl + pbuf * TBW, L.lane);
        __syncwarp();
      }
      prep_masks<PH, MODE>(sd, w, wr, m, L, wm.tbl + pbuf * TBW, wm.kill);
      prep_pos = i;
    }
    if (PH == K_H) {
      // dense rows of this position (prefetched one position ahead)
      if (ppos == i) {
        lv[0] = plv[0]; lv[1] = plv[1]; din[0] = pdin[0]; din[1] = pdin[1];
      } else {
        { const ulonglong2 t = ld_pair_s(p.live, m.blk, W, L.w0); lv[0] = t.x; lv[1] = t.y; }
        { const ulonglong2 t = ld_pair_s(p.d_in, m.blk, W, L.w0); din[0] = t.x; din[1] = t.y; }
      }
      ppos = -1;
      if (i + 1 < wr.we) {
        const int nb = w.meta[i + 1 - wr.mbase].blk;
        { const ulonglong2 t = ld_pair_s(p.live, nb, W, L.w0); plv[0] = t.x; plv[1] = t.y; }
        { const ulonglong2 t = ld_pair_s(p.d_in, nb, W, L.w0); pdin[0] = t.x; pdin[1] = t.y; }
        ppos = i + 1;
      }
    }
    if (m.head_loop >= 0) {  // a loop opens: its body is walked once
      st_l[depth] = m.head_loop;
      st_pend[depth] = m.head_pend;
      st_hs[depth] = m.head_hslot;
      ++depth;
      top_pend = m.head_pend;
    }
    // ---- value entering the block
#pragma unroll
    for (int pl = 0; pl < NP; ++pl) z[pl][0] = z[pl][1] = 0;
    if (i == cm.s) {
#pragma unroll
      for (int pl = 0; pl < NP; ++pl) { z[pl][0] = cin[pl][0]; z[pl][1] = cin[pl][1]; }
    }
    for (int q = 0; q < m.nfin; ++q) {
      const int2 fe = win_edge(w, wr, sd.fin_pk, m.fin_beg + q);
      const int slot = fe.x;
      if (slot == CARRY || slot == BACK) continue;  // in z via cin / closed at the loop's end
      // a loop-entry edge leaves out what is hoisted to it (Sec. IV-D)
      uint64_t m0 = ~0ull, m1 = ~0ull;
      if (PH != K_HP && fe.y >= 0) { m0 = ~ld_word(ec, fe.y, W, L.w0); m1 = ~ld_word(ec, fe.y, W, L.w0 + 1); }
      if (slot == PREV) {  // the position walked just before
#pragma unroll
        for (int pl = 0; pl < NP; ++pl) { z[pl][0] |= pv[pl][0] & m0; z[pl][1] |= pv[pl][1] & m1; }
        continue;
      }
#pragma unroll
      for (int pl = 0; pl < NP; ++pl) {
        const ulonglong2 v = sl.ld(slot, pl, L.lane);
        z[pl][0] |= v.x & m0;
        z[pl][1] |= v.y & m1;
      }
    }
    // a header keeps the meet of its entry edges (enclosing level) for the
    // loop's end; the body is walked relative to the header's value
    if (m.head_loop >= 0) {
      const int hs = m.head_hslot;
#pragma unroll
      for (int pl = 0; pl < NP; ++pl) sl.st(hs, pl, L.lane, make_ulonglong2(z[pl][0], z[pl][1]));
      z[0][0] = z[0][1] = 0;
      z[1][0] = L.top0;
      z[1][1] = L.top1;
    }
    if (PH == K_H) {  // live and stale on the device -> resolved toward the host
      const uint64_t b0 = ~(lv[0] & ~din[0]), b1 = ~(lv[1] & ~din[1]);
#pragma unroll
      for (int pl = 0; pl < NP; ++pl) { z[pl][0] &= b0; z[pl][1] &= b1; }
    }
#pragma unroll
    for (int pl = 0; pl < NP; ++pl) { zo[pl][0] = z[pl][0]; zo[pl][1] = z[pl][1]; }
    __syncwarp();
    take_masks<NP, false>(wm.tbl + pbuf * TBW, L.lane, zo);
    // build the next position's masks while this value is finished
    if (i + 1 < wr.we) {
      pbuf ^= 1;
      prep_masks<PH, MODE>(sd, w, wr, w.meta[i + 1 - wr.mbase], L, wm.tbl + pbuf * TBW, wm.kill);
      prep_pos = i + 1;
    } else {
      prep_pos = -1;
    }
    if (m.fslot >= 0) {
#pragma unroll
      for (int pl = 0; pl < NP; ++pl) sl.st(m.fslot, pl, L.lane, make_ulonglong2(zo[pl][0], zo[pl][1]));
    }
#pragma unroll
    for (int pl = 0; pl < NP; ++pl) {
      pv[pl][0] = zo[pl][0];
      pv[pl][1] = zo[pl][1];
    }
    // ---- outputs: each position's affine pairs
    {
      const size_t row = (size_t)m.blk;
      if (PH == K_D) {  // device validity at the block entry (and exit, kept states)
        st_pair_s(sd.pair_gd, row, W, L.w0, z[0][0], z[0][1]);
        st_pair_s(sd.pair_pd, row, W, L.w0, z[1][0], z[1][1]);
        if (sd.pair_g2) {
          st_pair_s(sd.pair_g2, row, W, L.w0, zo[0][0], zo[0][1]);
          st_pair_s(sd.pair_p2, row, W, L.w0, zo[1][0], zo[1][1]);
        }
      }
      if (PH == K_H) {  // host validity at the block exit
        st_pair_s(sd.pair_g, row, W, L.w0, zo[0][0], zo[0][1]);
        st_pair_s(sd.pair_p, row, W, L.w0, zo[1][0], zo[1][1]);
      }
      if ((PH == K_HP || PH == K_D) && m.nsrcent) {  // at loop-entry sources
        for (int q = 0; q < m.nsrcent; ++q) {
          const int k = sd.srcent[m.srcent_beg + q];
          st_pair(sd.src_g, k, W, L.w0, zo[0][0], zo[0][1]);
          st_pair(sd.src_p, k, W, L.w0, zo[1][0], zo[1][1]);
        }
      }
    }
    __syncwarp();
    // ---- close the loops ending here
    while (depth > 0 && top_pend - 1 == i) {
      --depth;
      close_loop(sd, sl, L, W, st_l[depth], st_hs[depth], pv, PH == K_D && p.ant_dm ? p.ec_d : nullptr);
      top_pend = depth > 0 ? st_pend[depth - 1] : -1;
    }
  }
  // ---- what leaves the chunk: its map of the carry into the next chunk
  uint64_t co[NP][2];
#pragma unroll
  for (int pl = 0; pl < NP; ++pl) co[pl][0] = co[pl][1] = 0;
  for (int q = 0; q < cm.carry_cnt; ++q) {
    const CarrySrc cs = sd.csrc[cm.carry_beg + q];
    uint64_t m0 = ~0ull, m1 = ~0ull;
    if (PH != K_HP && cs.ent >= 0) { m0 = ~ld_word(ec, cs.ent, W, L.w0); m1 = ~ld_word(ec, cs.ent, W, L.w0 + 1); }
#pragma unroll
    for (int pl = 0; pl < NP; ++pl) {
      const ulonglong2 v = sl.ld(cs.slot, pl, L.lane);
      co[pl][0] |= v.x & m0;
      co[pl][1] |= v.y & m1;
    }
  }
  if (cm.carry_cnt) {
    st_pair(sd.gsum, c, W, L.w0, co[0][0], co[0][1]);
    st_pair(sd.psum, c, W, L.w0, co[1][0], co[1][1]);
  }
}

// Take the next (chunk, word group) item of a launch's work queue: lane 0
// bumps the queue head, the warp shares the value.
__device__ __forceinline__ int next_item(const ScanDev &sd, int qslot) {
  int item = 0;
  if ((threadIdx.x & 31) == 0) item = atomicAdd(&sd.queue[qslot], 1);
  return __shfl_sync(0xffffffffu, item, 0);
}

// Persistent forward chain: each warp takes items (longest chunks first)
// from the launch's work queue until none is left.
template <int PH>
__global__ void __launch_bounds__(32 * OMPDART_MAX_WPC, OMPDART_FWD_MIN_CTAS)
    k_fwd_chain(DevPlan p, ScanDev sd, int qslot) {
  extern __shared__ __align__(16) uint64_t smem[];
  const int warp_in_cta = threadIdx.x >> 5;
  const int gw = blockIdx.x * (blockDim.x >> 5) + warp_in_cta;
  const WarpMem wm = carve<2, false>(smem, warp_in_cta, sd.sh_slots);
  uint64_t *spill = sd.spill + (size_t)gw * sd.spill_stride;
  const int n_items = sd.C * sd.G;
  for (int item = next_item(sd, qslot); item < n_items; item = next_item(sd, qslot)) {
    fwd_walk<PH>(p, sd, wm, spill, sd.work[item / sd.G], item % sd.G);
    __syncwarp();
  }
}

// --------------------------------------------------------------------------------------
// backward chain (anticipation; loop-restricted anticipation for the masks)
// --------------------------------------------------------------------------------------
template <int MODE>
struct BwdPlanes {  // SUM: [Live local, carry coefficient, A coefficient, A2 coefficient];
                    // LANT: [H, D, H header coefficient, D header coefficient]
  static constexpr int NP = 4;
};

template <int MODE>
__device__ void bwd_range(const DevPlan &p, const ScanDev &sd, const Lane &L, const WarpMem &wm,
                          const Slots<BwdPlanes<MODE>::NP> &sl, int s, int e, int base_depth, int lo_pos,
                          bool use_carry, const uint64_t (&cin)[BwdPlanes<MODE>::NP][2],
                          uint64_t (&zlast)[BwdPlanes<MODE>::NP][2], int cfg) {
  Win &w = *wm.win;
  constexpr int NP = BwdPlanes<MODE>::NP;
  const int W = p.W;
  const uint64_t *xlr = p.exit_live + (size_t)cfg * W;
  const uint64_t xl0 = L.w0 < W ? xlr[L.w0] : 0, xl1 = L.w0 + 1 < W ? xlr[L.w0 + 1] : 0;
  int st_ph[MAX_DEPTH + 1], st_pend[MAX_DEPTH + 1];  // open loops: header position, body end
  int depth = base_depth;
  uint32_t dirty = 0;
  int reruns = 0;
  uint64_t z[NP][2];
  WinRegs wr;
  wr.ws = wr.we = 0;
  int lwm = e;  // lowest position walked so far
  int top_ph = -1;  // header of the innermost open loop (warp-uniform)
  uint64_t pv[NP][2] = {};
  constexpr bool LANT = MODE == M_LANT;
  constexpr int TBW = mask_rows(NP, LANT) * 64;  // words of one mask table
  int pbuf = 0, prep_pos = -1;      // table holding the built masks of prep_pos
  drop_masks<NP, LANT>(wm.tbl, L.lane);   // shared memory starts undefined: the
  drop_masks<NP, LANT>(wm.tbl + TBW, L.lane);  // masks are built by ORing into zeros
  __syncwarp();
  int i = e - 1;
  while (i >= s) {
    if (i < wr.ws || i >= wr.we) load_window<false>(w, wr, sd, i, s, e, L.lane);
    const PosMeta m = w.meta[i - wr.mbase];
    if (prep_pos != i) {
      if (prep_pos >= 0) {
        drop_masks<NP, LANT>(wm.tbl + pbuf * TBW, L.lane);
        __syncwarp();
      }
      prep_masks<K_ANT, MODE>(sd, w, wr, m, L, wm.tbl + pbuf * TBW, wm.kill);
      prep_pos = i;
    }
    // enter loops whose range ends here (outer first)
    for (int q = 0; q < m.nbend; ++q) {
      // {depth, header position, body end, header slot}
      const int4 bi = q ? sd.bend_info[m.bend_beg + q] : make_int4(m.bend_depth, m.bend_ph, m.bend_pend, m.bend_hslot);
      if (bi.x <= depth) continue;
      st_ph[bi.x - 1] = bi.y;
      st_pend[bi.x - 1] = bi.z;
      dirty &= ~(1u << (bi.x - 1));
      depth = bi.x;
      top_ph = bi.y;
      // first visit: the header's value, read by the latches, starts from
      // nothing (outermost open loop: the latches read A itself, the
      // header coefficient planes all ones; liveness, one level down: A2
      // itself, plane 3 all ones); a re-entry keeps the previous visit's
      // value
      if (i < lwm) {
        const int hs = bi.w, rel = bi.x - base_depth;
        if (hs >= 0)
          for (int pl = 0; pl < NP; ++pl) {
            const bool one = LANT ? rel == 1 && pl >= 2 : (rel == 1 && pl == 2) || (rel == 2 && pl == 3);
            sl.st(hs, pl, L.lane, one ? make_ulonglong2(L.top0, L.top1) : make_ulonglong2(0ull, 0ull));
          }
        __syncwarp();
      }
    }
#pragma unroll
    for (int pl = 0; pl < NP; ++pl) z[pl][0] = z[pl][1] = 0;
    if (MODE != M_LANT && m.exit_idx >= 0) {  // region exit: the host may read what is live
      z[0][0] = MODE == M_NA ? L.top0 : xl0;    // (not anticipated: nothing is read after it)
      z[0][1] = MODE == M_NA ? L.top1 : xl1;
    }
    for (int q = 0; q < m.nout; ++q) {
      const int2 oe = win_edge(w, wr, sd.out_pk, m.out_beg + q);
      const int slot = oe.x;
      if (MODE == M_LANT) {
        if (oe.y <= lo_pos || oe.y >= e) continue;  // back to the loop header or out of the body
      }
      if (slot == PREV) {  // the position walked just before
#pragma unroll
        for (int pl = 0; pl < NP; ++pl) { z[pl][0] |= pv[pl][0]; z[pl][1] |= pv[pl][1]; }
        continue;
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
        const ulonglong2 v = sl.ld(slot, pl, L.lane);
        z[pl][0] |= v.x;
        z[pl][1] |= v.y;
      }
    }
    __syncwarp();
    take_masks<NP, LANT>(wm.tbl + pbuf * TBW, L.lane, z);
    if (i - 1 >= wr.ws && i - 1 >= s) {
      pbuf ^= 1;
      prep_masks<K_ANT, MODE>(sd, w, wr, w.meta[i - 1 - wr.mbase], L, wm.tbl + pbuf * TBW, wm.kill);
      prep_pos = i - 1;
    } else {
      prep_pos = -1;
    }
    const bool is_top_header = depth > base_depth && top_ph == i;
    // at the header of an outermost open loop: A = G | (carry & P) | (A & PA)
    // has the least solution A = G | (carry & P) (so no second walk); the
    // value leaves the loop without the header planes.  Liveness keeps A
    // for the resolve; the loop masks need values at their own header only.
    const bool sym_close = is_top_header && depth == base_depth + 1;
    // liveness, one level down: A2 = X | (A2 & PA2) likewise has the least
    // solution X, a triple of the carry and A kept for the resolve
    const bool sym2_close = MODE != M_LANT && is_top_header && depth == base_depth + 2;
    if (sym_close) {
      if (MODE != M_LANT) {
        st_pair(sd.hdrl_g, m.head_loop, W, L.w0, z[0][0], z[0][1]);
        st_pair(sd.hdrl_p, m.head_loop, W, L.w0, z[1][0], z[1][1]);
      }
#pragma unroll
      for (int pl = 2; pl < NP; ++pl) z[pl][0] = z[pl][1] = 0;
    }
    if (sym2_close) {
      st_pair(sd.hdrl2_g, m.head_loop, W, L.w0, z[0][0], z[0][1]);
      st_pair(sd.hdrl2_p, m.head_loop, W, L.w0, z[1][0], z[1][1]);
      st_pair(sd.hdrl2_a, m.head_loop, W, L.w0, z[2][0], z[2][1]);
      z[3][0] = z[3][1] = 0;
    }
    const bool rewalk = is_top_header && !sym_close && !sym2_close;
    if (m.bslot >= 0) {
      bool changed = false;
#pragma unroll
      for (int pl = 0; pl < NP; ++pl) {
        if (rewalk) {
          const ulonglong2 old = sl.ld(m.bslot, pl, L.lane);
          changed |= (old.x != z[pl][0]) || (old.y != z[pl][1]);
        }
        sl.st(m.bslot, pl, L.lane, make_ulonglong2(z[pl][0], z[pl][1]));
      }
      if (rewalk && __any_sync(0xffffffffu, changed)) dirty |= 1u << (depth - 1);
    }
    if (MODE != M_LANT) {  // the value at entry as an affine pair of the chunk's carry (and A, A2 inside loops)
      st_pair_s(sd.pair_g, m.blk, W, L.w0, z[0][0], z[0][1]);
      st_pair_s(sd.pair_p, m.blk, W, L.w0, z[1][0], z[1][1]);
      if (depth > base_depth) st_pair_s(sd.pair_a, m.blk, W, L.w0, z[2][0], z[2][1]);
      if (depth > base_depth + 1) st_pair_s(sd.pair_a2, m.blk, W, L.w0, z[3][0], z[3][1]);
    }
    __syncwarp();
#pragma unroll
    for (int pl = 0; pl < NP; ++pl) {
      zlast[pl][0] = pv[pl][0] = z[pl][0];
      zlast[pl][1] = pv[pl][1] = z[pl][1];
    }
    bool jumped = false;
    while (depth > base_depth && top_ph == i) {
      if (dirty & (1u << (depth - 1))) {
        dirty &= ~(1u << (depth - 1));
        i = st_pend[depth - 1] - 1;
        jumped = true;
        break;
      }
      --depth;
      top_ph = depth > base_depth ? st_ph[depth - 1] : -1;
    }
    lwm = min(lwm, i);
    if (jumped) {
      if (++reruns > rerun_cap(e - s)) {
        if (L.lane == 0) {
          atomicExch(&p.status[ST_ERROR], ERR_NOCONVERGE);
          if (sd.cfg_err) atomicExch(&sd.cfg_err[cfg], 1);
        }
        return;
      }
    } else {
      --i;
    }
  }
  if (L.lane == 0 && reruns) atomicAdd(&p.status[ST_SWEEPS], reruns);
}

template <int MODE>
__device__ __forceinline__ void bwd_walk(const DevPlan &p, const ScanDev &sd, const WarpMem &wm, uint64_t *spill,
                                         int c, int wg) {
  constexpr int NP = BwdPlanes<MODE>::NP;
  const int W = p.W;
  Lane L;
  L.lane = threadIdx.x & 31;
  L.wg = wg;
  L.w0 = wg * 64 + 2 * L.lane;
  const uint64_t *tp = p.top + (size_t)sd.chunks[c].cfg * W;  // this CFG's valid-variable mask
  L.top0 = L.w0 < W ? tp[L.w0] : 0;
  L.top1 = L.w0 + 1 < W ? tp[L.w0 + 1] : 0;
  Slots<NP> sl{wm.slots, spill, sd.sh_slots};
  const ChunkMeta cm = sd.chunks[c];
  uint64_t cin[NP][2] = {}, zl[NP][2];
  // the identity map of the liveness entering from the next chunk
  cin[1][0] = L.top0;
  cin[1][1] = L.top1;
  bwd_range<MODE>(p, sd, L, wm, sl, cm.s, cm.e, 0, -1, true, cin, zl, cm.cfg);
  st_pair(sd.gsum, c, W, L.w0, zl[0][0], zl[0][1]);
  st_pair(sd.psum, c, W, L.w0, zl[1][0], zl[1][1]);
}

// The loop masks of loop l for the 64-word group wg: anticipation
// restricted to its body (one iteration from the header) and the kills
// anywhere in the body, by one walk of the body (Sec. IV-D loop rule).
__device__ __forceinline__ void lant_walk(const DevPlan &p, const ScanDev &sd, const WarpMem &wm, uint64_t *spill,
                                          int l, int wg) {
  constexpr int NP = BwdPlanes<M_LANT>::NP;
  const int W = p.W;
  const LoopMeta lm = sd.loops[l];
  Lane L;
  L.lane = threadIdx.x & 31;
  L.wg = wg;
  L.w0 = wg * 64 + 2 * L.lane;
  const uint64_t *tp = p.top + (size_t)lm.cfg * W;
  L.top0 = L.w0 < W ? tp[L.w0] : 0;
  L.top1 = L.w0 + 1 < W ? tp[L.w0 + 1] : 0;
  Slots<NP> sl{wm.slots, spill, sd.sh_slots};
  uint64_t cin[NP][2] = {}, zl[NP][2];
  *reinterpret_cast<ulonglong2 *>(wm.kill + 2 * L.lane) = make_ulonglong2(0ull, 0ull);
  *reinterpret_cast<ulonglong2 *>(wm.kill + 64 + 2 * L.lane) = make_ulonglong2(0ull, 0ull);
  __syncwarp();
  bwd_range<M_LANT>(p, sd, L, wm, sl, lm.ph, lm.pend, lm.depth, lm.ph, false, cin, zl, lm.cfg);
  const ulonglong2 kh = *reinterpret_cast<const ulonglong2 *>(wm.kill + 2 * L.lane);
  const ulonglong2 kd = *reinterpret_cast<const ulonglong2 *>(wm.kill + 64 + 2 * L.lane);
  st_pair(p.mask_h, l, W, L.w0, zl[0][0] & ~kh.x & L.top0, zl[0][1] & ~kh.y & L.top1);
  st_pair(p.mask_d, l, W, L.w0, zl[1][0] & ~kd.x & L.top0, zl[1][1] & ~kd.y & L.top1);
}

// persistent backward chain (same work queue scheme as the forward one);
// the loop-mask walks take one loop per item
template <int MODE>
__global__ void __launch_bounds__(32 * OMPDART_MAX_WPC, OMPDART_BWD_MIN_CTAS)
    k_bwd_chain(DevPlan p, ScanDev sd, int qslot) {
  constexpr int NP = BwdPlanes<MODE>::NP;
  extern __shared__ __align__(16) uint64_t smem[];
  const int warp_in_cta = threadIdx.x >> 5;
  const int gw = blockIdx.x * (blockDim.x >> 5) + warp_in_cta;
  const WarpMem wm = carve<NP, MODE == M_LANT>(smem, warp_in_cta, sd.sh_slots);
  uint64_t *spill = sd.spill + (size_t)gw * sd.spill_stride;
  const int n_items = (MODE == M_LANT ? sd.n_loops : sd.C) * sd.G;
  for (int item = next_item(sd, qslot); item < n_items; item = next_item(sd, qslot)) {
    if (MODE == M_LANT)
      lant_walk(p, sd, wm, spill, sd.lant_work[item / sd.G], item % sd.G);
    else
      bwd_walk<MODE>(p, sd, wm, spill, sd.work[item / sd.G], item % sd.G);
    __syncwarp();
  }
}

// Local summary records and flag tables, one thread per access of the
// position-ordered stream.  The host links every access to the first
// access of the same variable in its block and to the next one, so each
// thread visits only its variable's accesses:
//   record (at the variable's first access, REC_NONE elsewhere): the last
//     event on each copy decides Gen/Kill, a read before any write is
//     upward exposed, any write defines (Sec. IV-D local rule);
//   flag table: for each validity of the variable at the block entry,
//     k = host | device << 1, bits 2k..2k+1 hold the transfer right before
//     this access (0, 1 `to', 2 `from'): the earlier accesses replayed from
//     the four entry states at once, one bit each (a read makes its space
//     valid, a write its space valid and the other stale).
__global__ void __launch_bounds__(256) k_local_summary_pos(ScanDev sd) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= sd.n_acc_p) return;
  const int2 lk = sd.acc_link[j];
  const uint32_t aj = sd.acc_p[j];
  if (lk.x == LINK_RECORD) {  // a block with calls: records given
    sd.rec_p[j] = aj;
    return;
  }
  if (lk.x == j) {  // the variable's first access: fold its accesses
    int last_h = 0, last_d = 0, first_rh = 0, first_rd = 0, first_w = 0, t = 0;
    for (int q = (int)j; q >= 0; q = sd.acc_link[q].y) {
      const uint32_t a = sd.acc_p[q];
      const int kind = acc_kind(a), dev = acc_space(a);
      if (kind & 1) {
        ++t;
        if (dev) { last_d = 1; if (!first_rd) first_rd = t; }
        else     { last_h = 1; if (!first_rh) first_rh = t; }
      }
      if (kind & 2) {
        ++t;
        if (dev) { last_d = 1; last_h = 2; } else { last_h = 1; last_d = 2; }
        if (!first_w) first_w = t;
      }
    }
    uint32_t r = (uint32_t)acc_var(aj);
    if (last_h == 1) r |= R_GH;
    if (last_h == 2) r |= R_KH;
    if (last_d == 1) r |= R_GD;
    if (last_d == 2) r |= R_KD;
    if (first_rh && (!first_w || first_rh < first_w)) r |= R_UH;
    if (first_rd && (!first_w || first_rd < first_w)) r |= R_UD;
    if (first_w) r |= R_DF;
    sd.rec_p[j] = r;
  } else {
    sd.rec_p[j] = REC_NONE;
  }
  uint32_t h = 0xAu, d = 0xCu;  // entry state k: host bit k & 1, device bit k & 2
  for (int q = lk.x; q != (int)j; q = sd.acc_link[q].y) {
    const uint32_t x = sd.acc_p[q];
    const int kind = acc_kind(x), dev = acc_space(x);
    if (kind & 1) { if (dev) d = 0xFu; else h = 0xFu; }
    if (kind & 2) { if (dev) { d = 0xFu; h = 0u; } else { h = 0xFu; d = 0u; } }
  }
  uint32_t lut = 0;
  if (acc_kind(aj) & 1) {
    const int dev = acc_space(aj);
    const uint32_t miss = ~(dev ? d : h) & 0xFu;
    for (int k = 0; k < 4; ++k)
      if (miss >> k & 1u) lut |= (dev ? 1u : 2u) << (2 * k);
  }
  sd.emit_p[j] = (uint32_t)acc_var(aj) | (lut << 24);
}

// --------------------------------------------------------------------------------------
// resolve: every position's value from its pair and its chunk's carry
// --------------------------------------------------------------------------------------
// liveness as is; stale sets to valid sets; a liveness-shaped complement
// (not anticipated) to the anticipated set
enum ResolveKind { RV_LIVE = 0, RV_VALID = 1, RV_NA = 2 };

// Each loop's header value composed up the loop tree (maps compose
// associatively): a pair of the chunk's carry, one thread per (loop, word).
__global__ void k_loop_abs(DevPlan p, ScanDev sd) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int W = p.W;
  if (t >= (long long)p.L * W) return;
  const int l = (int)(t / W), w = (int)(t % W);
  uint64_t g = sd.hdr_g[t], q = sd.hdr_p[t];
  for (int a = sd.loop_up[l]; a >= 0; a = sd.loop_up[a])
    compose_pair(g, q, sd.hdr_g[(size_t)a * W + w], sd.hdr_p[(size_t)a * W + w]);
  sd.hdr_ag[t] = g;
  sd.hdr_ap[t] = q;
}

// out[b] = G[b] | (carry[chunk] & P[b]), converted for RV_VALID to ~x & top
// (the CFG's valid-variable mask).  A forward (RV_VALID) pair is relative
// to the header value of the innermost loop holding the position: it is
// first composed with that header's value as a pair of the carry
// (k_loop_abs).  A liveness pair inside a loop first takes in its
// outermost loop's header value A through PA (G |= A_G & PA,
// P |= A_P & PA).  A thread takes
// two consecutive words of a row (16-byte accesses when W is even); the
// grid strides over (position, word pair).
template <int KIND>
__global__ void __launch_bounds__(256) k_resolve(DevPlan p, ScanDev sd, const uint64_t *G, const uint64_t *P,
                                                 uint64_t *out) {
  const int W = p.W, W2 = (W + 1) >> 1;
  const long long n = (long long)p.M * W2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / W2), w = 2 * (int)(t % W2);
    const int b = p.order[i], c = sd.pos_chunk[i];
    const size_t o = (size_t)b * W + w, oc = (size_t)c * W + w;
    const uint64_t *tp = p.top + (size_t)sd.chunks[c].cfg * W + w;
    if ((W & 1) == 0) {
      ulonglong2 g = *reinterpret_cast<const ulonglong2 *>(G + o);
      ulonglong2 q = *reinterpret_cast<const ulonglong2 *>(P + o);
      const int pl = sd.pos_loop[i];
      if (KIND != RV_VALID && pl >= 0) {
        const int l = sd.loop_root[pl], l2 = sd.loop_d2[pl];
        ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(sd.pair_a + o);
        if (l2 >= 0) {  // first A2 (a triple of the carry and A) through PA2
          const size_t ol = (size_t)l2 * W + w;
          const ulonglong2 a2 = *reinterpret_cast<const ulonglong2 *>(sd.pair_a2 + o);
          const ulonglong2 x0 = *reinterpret_cast<const ulonglong2 *>(sd.hdrl2_g + ol);
          const ulonglong2 x1 = *reinterpret_cast<const ulonglong2 *>(sd.hdrl2_p + ol);
          const ulonglong2 x2 = *reinterpret_cast<const ulonglong2 *>(sd.hdrl2_a + ol);
          g = make_ulonglong2(g.x | (x0.x & a2.x), g.y | (x0.y & a2.y));
          q = make_ulonglong2(q.x | (x1.x & a2.x), q.y | (x1.y & a2.y));
          a = make_ulonglong2(a.x | (x2.x & a2.x), a.y | (x2.y & a2.y));
        }
        const ulonglong2 h0 = *reinterpret_cast<const ulonglong2 *>(sd.hdrl_g + (size_t)l * W + w);
        const ulonglong2 h1 = *reinterpret_cast<const ulonglong2 *>(sd.hdrl_p + (size_t)l * W + w);
        g = make_ulonglong2(g.x | (h0.x & a.x), g.y | (h0.y & a.y));
        q = make_ulonglong2(q.x | (h1.x & a.x), q.y | (h1.y & a.y));
      }
      if (KIND == RV_VALID && pl >= 0) {
        const ulonglong2 h0 = *reinterpret_cast<const ulonglong2 *>(sd.hdr_ag + (size_t)pl * W + w);
        const ulonglong2 h1 = *reinterpret_cast<const ulonglong2 *>(sd.hdr_ap + (size_t)pl * W + w);
        compose_pair(g.x, q.x, h0.x, h1.x);
        compose_pair(g.y, q.y, h0.y, h1.y);
      }
      const ulonglong2 k = *reinterpret_cast<const ulonglong2 *>(sd.carry + oc);
      ulonglong2 x = make_ulonglong2(g.x | (k.x & q.x), g.y | (k.y & q.y));
      if (KIND != RV_LIVE) x = make_ulonglong2(~x.x & tp[0], ~x.y & tp[1]);
      *reinterpret_cast<ulonglong2 *>(out + o) = x;
    } else {
      for (int u = 0; u < 2 && w + u < W; ++u) {
        uint64_t g = G[o + u], q = P[o + u];
        const int pl = sd.pos_loop[i];
        if (KIND != RV_VALID && pl >= 0) {
          const int l = sd.loop_root[pl], l2 = sd.loop_d2[pl];
          uint64_t a = sd.pair_a[o + u];
          if (l2 >= 0) {
            const size_t ol = (size_t)l2 * W + w + u;
            const uint64_t a2 = sd.pair_a2[o + u];
            g |= sd.hdrl2_g[ol] & a2;
            q |= sd.hdrl2_p[ol] & a2;
            a |= sd.hdrl2_a[ol] & a2;
          }
          g |= sd.hdrl_g[(size_t)l * W + w + u] & a;
          q |= sd.hdrl_p[(size_t)l * W + w + u] & a;
        }
        if (KIND == RV_VALID && pl >= 0)
          compose_pair(g, q, sd.hdr_ag[(size_t)pl * W + w + u], sd.hdr_ap[(size_t)pl * W + w + u]);
        const uint64_t x = g | (sd.carry[oc + u] & q);
        out[o + u] = KIND == RV_LIVE ? x : ~x & tp[u];
      }
    }
  }
}

// The same for the out values at the sources of the edges with constants
// ([K][W]), as valid sets, and the constants they decide (Sec. IV-D) in the
// same pass: which = 0, plain host validity: ec_d = mask_d & Hp on a
// loop-entry edge (the value itself is not kept); which = 1, device
// validity: d_src (the emission reads it) and ec_h = mask_h & D on a
// loop-entry edge, plus, on an edge leaving the data region, what is live
// at its target (made valid on the host there).
__global__ void k_resolve_src(DevPlan p, ScanDev sd, int which) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int W = p.W;
  if (t >= (long long)p.K * W) return;
  const int k = (int)(t / W), w = (int)(t % W);
  const int i = sd.src_pos[k], c = sd.pos_chunk[i];
  uint64_t g = sd.src_g[t], q = sd.src_p[t];
  const int l = sd.pos_loop[i];
  if (l >= 0) compose_pair(g, q, sd.hdr_ag[(size_t)l * W + w], sd.hdr_ap[(size_t)l * W + w]);
  const uint64_t x = ~(g | (sd.carry[(size_t)c * W + w] & q)) & p.top[(size_t)sd.chunks[c].cfg * W + w];
  const int le = p.ent_loop[k];
  if (which == 0) {
    uint64_t need = le >= 0 ? p.mask_d[(size_t)le * W + w] : 0ull;
    if (p.ant_dm) need |= p.ant_dm[(size_t)p.ent_dst[k] * W + w];  // eager: read on the device on every path on
    p.ec_d[t] = need & x;
  } else {
    sd.d_src[t] = x;
    uint64_t h = le >= 0 ? p.mask_h[(size_t)le * W + w] & x : 0ull;
    if (p.ent_rx && p.ent_rx[k]) h |= p.live[(size_t)p.ent_dst[k] * W + w];
    p.ec_h[t] = h;
  }
}

// --------------------------------------------------------------------------------------
// emission (Table II; Sec. IV-D), from the final states, one warp per
// (chunk, word group), positions in order (no dependency between them):
//   H_in = (OR over in-edges of the source's host-stale set, less the
//          hoisted `from' of a loop-entry edge) minus the conflicts (live,
//          valid on the device at no entry) resolved toward the host;
//          the CFG's entry starts from its entry row;
//   per in-edge p->b: `to' = hoisted device need not valid at p (loop
//          entries), `from' = hoisted host need stale at p (loop entries)
//          or a conflict the edge leaves stale on the host;
//   per access: its flag table at the variable's entry validity;
//   region exit: live after the exit and stale on the host.
// --------------------------------------------------------------------------------------
constexpr int EMIT_WARPS = 4;
#ifndef OMPDART_EMIT_SPAN
#define OMPDART_EMIT_SPAN 8
#endif
constexpr int EMIT_SPAN = OMPDART_EMIT_SPAN;  // positions per emission item (its own record stream)
// 10 CTAs of 4 warps per SM (48 registers): the emission waits on loads of
// state rows; 40 warps per SM ran it 20% faster than 28 (72 registers)
#ifndef OMPDART_EMIT_MIN_CTAS
#define OMPDART_EMIT_MIN_CTAS 10
#endif
// H_out (valid) of position i, block b, resolved from the host-validity
// walk's pairs: composed with the innermost loop's header, then the carry
// `car' of the position's chunk (G | (carry & P), as a stale set)
__device__ __forceinline__ ulonglong2 h_out_at(const ScanDev &sd, size_t b, int i, int W, int w0, uint64_t car0,
                                               uint64_t car1, uint64_t top0, uint64_t top1) {
  const ulonglong2 g = ld_pair_s(sd.pair_g, b, W, w0), q = ld_pair_s(sd.pair_p, b, W, w0);
  uint64_t g0 = g.x, g1 = g.y, q0 = q.x, q1 = q.y;
  const int lp = sd.pos_loop[i];
  if (lp >= 0) {
    const ulonglong2 h0 = ld_pair(sd.hdr_ag, lp, W, w0), h1 = ld_pair(sd.hdr_ap, lp, W, w0);
    compose_pair(g0, q0, h0.x, h1.x);
    compose_pair(g1, q1, h0.y, h1.y);
  }
  return make_ulonglong2(~(g0 | (car0 & q0)) & top0, ~(g1 | (car1 & q1)) & top1);
}

__global__ void __launch_bounds__(32 * EMIT_WARPS, OMPDART_EMIT_MIN_CTAS)
    k_emit(DevPlan p, ScanDev sd, const uint64_t *init) {
  __shared__ uint64_t hd_all[EMIT_WARPS][128];
  const int gw = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  if (gw >= sd.n_emit * sd.G) return;
  const int item = gw / sd.G, wg = gw % sd.G, lane = threadIdx.x & 31, W = p.W;
  uint64_t *hd = hd_all[threadIdx.x >> 5];
  const int2 rng = sd.emit_rng[item];
  const int ci = sd.pos_chunk[rng.x];
  const ChunkMeta cm = sd.chunks[ci];
  const int w0 = wg * 64 + 2 * lane;
  const uint64_t *tp = p.top + (size_t)cm.cfg * W;
  const uint64_t top0 = w0 < W ? tp[w0] : 0, top1 = w0 + 1 < W ? tp[w0 + 1] : 0;
  const uint64_t *xl = p.exit_live + (size_t)cm.cfg * W;
  const int stream = item * sd.G + wg;
  // H_out is resolved here, not in a pass of its own: each position's own
  // value (kept for the next position, whose in-edge from it is the usual
  // one), and a source elsewhere from its pairs and its chunk's carry
  ulonglong2 prev_ho = make_ulonglong2(0ull, 0ull);
  int rec_count = 0;
  for (int i = rng.x; i < rng.y; ++i) {
    const PosMeta m = sd.meta[i];
    const size_t b = (size_t)m.blk;
    ulonglong2 own_ho;
    {
      const ulonglong2 hcar = ld_pair(sd.carry, ci, W, w0);  // the same row all item long: cached
      own_ho = h_out_at(sd, b, i, W, w0, hcar.x, hcar.y, top0, top1);
    }
    const ulonglong2 lv = ld_pair_s(p.live, b, W, w0), di = ld_pair_s(p.d_in, b, W, w0);
    const uint64_t lv0 = lv.x, lv1 = lv.y, di0 = di.x, di1 = di.y;
    const uint64_t c0 = lv0 & ~di0, c1 = lv1 & ~di1;
    uint64_t z0 = 0, z1 = 0;
    if (m.nfin == 0) {  // the CFG's entry
      z0 = ld_word(init, cm.cfg, W, w0);
      z1 = ld_word(init, cm.cfg, W, w0 + 1);
    }
    for (int q = 0; q < m.nfin; ++q) {
      const int k = m.fin_beg + q;
      const int2 fk = sd.fin_pk[k];
      const int ent = fk.y;  // loop-entry edge or -1
      const size_t src = (size_t)p.fin_src[k];
      ulonglong2 ho;
      if (fk.x == PREV && i > rng.x) {
        ho = prev_ho;
      } else {
        const int sp = p.pos[src], sc = sd.pos_chunk[sp];
        const ulonglong2 car = ld_pair(sd.carry, sc, W, w0);
        ho = h_out_at(sd, src, sp, W, w0, car.x, car.y, top0, top1);
      }
      const uint64_t s0 = ~ho.x & top0, s1 = ~ho.y & top1;
      uint64_t m0 = 0, m1 = 0, to0 = 0, to1 = 0;
      if (ent >= 0) {
        const ulonglong2 eh = ld_pair(p.ec_h, ent, W, w0), ed = ld_pair(p.ec_d, ent, W, w0),
                         ds = ld_pair(sd.d_src, ent, W, w0);
        m0 = eh.x;
        m1 = eh.y;
        to0 = ed.x & ~ds.x;
        to1 = ed.y & ~ds.y;
      }
      const uint64_t e0 = s0 & ~m0, e1 = s1 & ~m1;
      z0 |= e0;
      z1 |= e1;
      const uint64_t fr0 = (m0 & s0) | (c0 & e0), fr1 = (m1 & s1) | (c1 & e1);
      if (p.fin_bnd) {  // an edge on the data region's boundary: its row for the map clauses
        const int bi = p.fin_bnd[k];
        if (bi >= 0) {
          st_pair(p.bnd_to, bi, W, w0, to0, to1);
          st_pair(p.bnd_from, bi, W, w0, fr0, fr1);
        }
      }
      push_edge_records(sd, stream, rec_count, p.fin_eid[k], w0, to0, fr0, to1, fr1, lane);
    }
    z0 &= ~c0;
    z1 &= ~c1;
    const uint64_t hi0 = ~z0 & top0, hi1 = ~z1 & top1;
    st_pair_s(p.h_in, b, W, w0, hi0, hi1);
    if (m.nacc && !(m.flags & PM_RECORDS)) {  // flag table at the entry validity
      hd[2 * lane] = hi0;
      hd[2 * lane + 1] = hi1;
      hd[64 + 2 * lane] = di0;
      hd[64 + 2 * lane + 1] = di1;
      __syncwarp();
      for (int j = lane; j < m.nacc; j += 32) {
        const uint32_t e = sd.emit_p[m.pacc_beg + j];
        const int v = (int)(e & 0xFFFFFFu), lw = (v >> 6) - wg * 64;
        if ((unsigned)lw >= 64u) continue;
        const uint64_t bit = 1ull << (v & 63);
        const int kk = ((hd[lw] & bit) ? 1 : 0) | ((hd[64 + lw] & bit) ? 2 : 0);
        p.acc_flag[m.acc_beg + j] = (uint8_t)((e >> (24 + 2 * kk)) & 3u);
      }
      __syncwarp();
    }
    if (m.exit_idx >= 0) {  // region exit: live after it and stale on the host
      if (w0 < W) st_word(p.from_exit, m.exit_idx, W, w0, xl[w0] & ~own_ho.x & top0);
      if (w0 + 1 < W) st_word(p.from_exit, m.exit_idx, W, w0 + 1, xl[w0 + 1] & ~own_ho.y & top1);
    }
    if (sd.keep_states) st_pair_s(p.h_out, b, W, w0, own_ho.x, own_ho.y);
    prev_ho = own_ho;
  }
  if (lane == 0) sd.rec_cnt[stream] = rec_count;
}

// --------------------------------------------------------------------------------------
// scan of the chunk maps: carry[c] for every chunk (one thread per word and plane)
// --------------------------------------------------------------------------------------
// The walk order of the chunks is cut into S segments.  A CTA of SCAN_T
// threads takes one segment for a block of WB word columns (WB a power of
// two up to 64, covering W where it can), so the WB threads of a run read
// a chunk's row of maps together: thread (run r, word w) composes the maps
// of its contiguous run of chunks (walk order), the CTA scans the runs'
// maps per word in shared memory, then every thread walks its run again
// to write each chunk's carry.  Map composition: first (g1, p1), then
// (g2, p2) gives (g2 | (g1 & p2), p1 & p2).  The first chunk (in walk
// order) of each CFG of a batch starts from that CFG's own boundary value
// -- the forward entry value, or nothing for the backward problem -- so in
// the run maps it acts as a constant map.
constexpr int SCAN_T = 1024;
__device__ __forceinline__ void compose_after(uint64_t &g, uint64_t &p, uint64_t g1, uint64_t p1) {
  // (g1, p1) first, then the current (g, p)
  g = g | (g1 & p);
  p = p1 & p;
}
// word columns per scan CTA: the least power of two >= W, at most 64
inline int scan_wb(int W) {
  int wb = 1;
  while (wb < W && wb < 64) wb <<= 1;
  return wb;
}

// Inclusive scan over the runs of a CTA, word by word: thread t holds run
// t / WB of word t % WB; afterwards (g, p) is the composition of runs
// 0..r and the shared arrays hold every run's inclusive value.
__device__ __forceinline__ void scan_runs(uint64_t *gs, uint64_t *ps, uint64_t &g, uint64_t &p, int t, int r,
                                          int R, int WB) {
  gs[t] = g;
  ps[t] = p;
  __syncthreads();
  for (int d = 1; d < R; d <<= 1) {
    uint64_t g1 = 0, p1 = ~0ull;
    const bool has = r >= d;
    if (has) {
      g1 = gs[t - d * WB];
      p1 = ps[t - d * WB];
    }
    __syncthreads();
    if (has) {
      compose_after(g, p, g1, p1);
      gs[t] = g;
      ps[t] = p;
    }
    __syncthreads();
  }
}

// Grid (ceil(W / WB), S): phase 0 leaves each segment's map in seg; phase 1
// composes the maps of the segments before its own into the carry entering
// it (the CTA's runs share that work), then scans its runs again and
// writes every chunk's carry.
template <int PHASE>
__global__ void __launch_bounds__(SCAN_T) k_scan_carry(ScanDev sd, int W, int WB, int backward, const uint64_t *init) {
  __shared__ uint64_t gs[SCAN_T], ps[SCAN_T];
  const int t = threadIdx.x, wl = t & (WB - 1), r = t / WB, R = SCAN_T / WB;
  const int w = blockIdx.x * WB + wl, sg = blockIdx.y, S = gridDim.y;
  const bool on = w < W;
  const int C = sd.C;
  const int s0 = (int)((long long)C * sg / S), s1 = (int)((long long)C * (sg + 1) / S);
  const int per = (s1 - s0 + R - 1) / R;
  const int b = min(s1, s0 + r * per), e = min(s1, b + per);
  const int32_t rflag = backward ? CH_LAST : CH_FIRST;
  auto chunk = [&](int k) { return backward ? C - 1 - k : k; };  // k-th chunk in walk order
  auto reset_val = [&](int c) -> uint64_t {
    return backward || !init ? 0ull : init[(size_t)sd.chunks[c].cfg * W + w];
  };
  // the run's chunk maps are read in batches of SCAN_B independent loads
  // (the composition is sequential, the loads are not)
  constexpr int SCAN_B = 6;
  uint64_t gb[SCAN_B], pb[SCAN_B];
  int32_t fb[SCAN_B];
  auto load_batch = [&](int k0) {
#pragma unroll
    for (int j = 0; j < SCAN_B; ++j) {
      const int k = k0 + j;
      if (k < e) {
        const int c = chunk(k);
        gb[j] = sd.gsum[(size_t)c * W + w];
        pb[j] = sd.psum[(size_t)c * W + w];
        fb[j] = sd.chunks[c].flags;
      }
    }
  };
  // 1. the run's map
  uint64_t g = 0, pp = ~0ull;
  if (on)
    for (int k0 = b; k0 < e; k0 += SCAN_B) {
      load_batch(k0);
#pragma unroll
      for (int j = 0; j < SCAN_B; ++j) {
        if (k0 + j >= e) break;
        if (fb[j] & rflag) {
          g = reset_val(chunk(k0 + j));
          pp = 0;
        }
        g = gb[j] | (g & pb[j]);
        pp &= pb[j];
      }
    }
  // 2. inclusive scan of the run maps over the CTA's runs
  scan_runs(gs, ps, g, pp, t, r, R, WB);
  if (PHASE == 0) {  // the segment's map
    if (r == R - 1 && on) {
      sd.seg_g[(size_t)sg * W + w] = g;
      sd.seg_p[(size_t)sg * W + w] = pp;
    }
    return;
  }
  // the runs before this one
  uint64_t xg = 0, xp = ~0ull;
  if (r > 0) {
    xg = gs[t - WB];
    xp = ps[t - WB];
  }
  __syncthreads();
  // 3. the value entering the segment: the maps of the segments before it
  // applied to nothing (every walk starts at a CFG's first chunk, which
  // resets); run r composes segments [q0, q1), then the runs' parts are
  // composed in order
  uint64_t cg = 0, cp = ~0ull;
  if (on)
    for (int q0 = (int)((long long)sg * r / R), q1 = (int)((long long)sg * (r + 1) / R); q0 < q1; q0 += SCAN_B) {
#pragma unroll
      for (int j = 0; j < SCAN_B; ++j)
        if (q0 + j < q1) {
          gb[j] = sd.seg_g[(size_t)(q0 + j) * W + w];
          pb[j] = sd.seg_p[(size_t)(q0 + j) * W + w];
        }
#pragma unroll
      for (int j = 0; j < SCAN_B; ++j)
        if (q0 + j < q1) {
          cg = gb[j] | (cg & pb[j]);
          cp &= pb[j];
        }
    }
  scan_runs(gs, ps, cg, cp, t, r, R, WB);
  const uint64_t cin = gs[(R - 1) * WB + wl];
  uint64_t x = xg | (cin & xp);
  // 4. every chunk's carry
  if (on)
    for (int k0 = b; k0 < e; k0 += SCAN_B) {
      load_batch(k0);
#pragma unroll
      for (int j = 0; j < SCAN_B; ++j) {
        if (k0 + j >= e) break;
        const int c = chunk(k0 + j);
        if (fb[j] & rflag) x = reset_val(c);
        sd.carry[(size_t)c * W + w] = x;
        x = gb[j] | (x & pb[j]);
      }
    }
}

// initial stale sets at the entry block of each CFG (forward problems): ~valid & top
__global__ void k_entry_stale(const uint64_t *valid, const uint64_t *top, uint64_t *out, int W, int n_cfg) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < (long long)W * n_cfg) out[t] = ~valid[t] & top[t];
}


// gather the record streams into the result array: per-CTA sums of the
// streams' counts, a scan of those sums, per-CTA offsets, then the copy
constexpr int PF_T = 1024, PF_PER = 4, PF_TILE = PF_T * PF_PER;  // streams per prefix CTA

__device__ __forceinline__ int block_exclusive_sum(int v, int *total) {
  __shared__ int ws[PF_T / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) ws[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int a = ws[lane];
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, a, d);
      if (lane >= d) a += y;
    }
    ws[lane] = a;
  }
  __syncthreads();
  const int before = (wid ? ws[wid - 1] : 0) + x - v;
  *total = ws[PF_T / 32 - 1];
  __syncthreads();
  return before;
}

__global__ void __launch_bounds__(PF_T) k_streams_sums(ScanDev sd, int32_t *part, int32_t *status) {
  const int base = blockIdx.x * PF_TILE + threadIdx.x * PF_PER;
  int sum = 0;
  bool over = false;
  for (int u = 0; u < PF_PER; ++u) {
    const int i = base + u;
    if (i >= sd.n_streams) break;
    const int cnt = sd.rec_cnt[i];
    over |= cnt > sd.rec_cap[i];
    sum += cnt;
  }
  if (over) atomicExch(&status[ST_OVERFLOW], 1);
  int total = 0;
  block_exclusive_sum(sum, &total);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// one CTA: exclusive scan of the per-CTA sums (in tiles of PF_T), total
__global__ void __launch_bounds__(PF_T) k_streams_top(int32_t *part, int n_parts, int32_t *status) {
  int run = 0;
  for (int base = 0; base < n_parts; base += PF_T) {
    const int i = base + threadIdx.x;
    const int v = i < n_parts ? part[i] : 0;
    int total = 0;
    const int before = block_exclusive_sum(v, &total);
    if (i < n_parts) part[i] = run + before;
    run += total;
  }
  if (threadIdx.x == 0) status[ST_NREC] = run;
}

__global__ void __launch_bounds__(PF_T) k_streams_offsets(ScanDev sd, const int32_t *part, int32_t *offs) {
  const int base = blockIdx.x * PF_TILE + threadIdx.x * PF_PER;
  int cnt[PF_PER], sum = 0;
  for (int u = 0; u < PF_PER; ++u) {
    const int i = base + u;
    cnt[u] = i < sd.n_streams ? sd.rec_cnt[i] : 0;
    sum += cnt[u];
  }
  int total = 0;
  int run = part[blockIdx.x] + block_exclusive_sum(sum, &total);
  for (int u = 0; u < PF_PER; ++u) {
    const int i = base + u;
    if (i < sd.n_streams) offs[i] = run;
    run += cnt[u];
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
  if (st->stream_buf) {  // the buffer's last user (a finished run) is done
    dev_free(st->stream_buf);
    st->bytes -= (long long)sizeof(EdgeXfer) * std::max<long long>(st->total_cap, 1);
    st->allocs.erase(std::find(st->allocs.begin(), st->allocs.end(), (void *)st->stream_buf));
  }
  st->stream_buf = st->alloc<EdgeXfer>((size_t)tot);
  if (!st->stream_buf || cudaStreamSynchronize(cudaStreamPerThread) != cudaSuccess) return false;
  st->total_cap = tot;
  st->sd.stream = st->stream_buf;
  if (cudaMemcpy(st->d_rec_cap, st->h_rec_cap.data(), sizeof(int32_t) * st->n_streams, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(st->d_rec_base, base.data(), sizeof(int32_t) * st->n_streams, cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  return true;
}

namespace {
// warps of one CTA of a chain kernel: 1..8, default 4
int clamp_wpc(int wpc) { return wpc <= 0 ? WPC : std::min(OMPDART_MAX_WPC, std::max(1, wpc)); }

// Shape of a persistent chain launch: as many CTAs as can be resident at
// once (never more than the items need), slots in shared memory up to
// sh_words words per warp.
template <class K>
ChainShape chain_shape(K kern, int need, int np, bool kill, int sh_words, int wpc, int n_items, int n_sm) {
  ChainShape c;
  c.wpc = wpc;
  c.sh_slots = std::min(need, sh_words / (64 * np));
  c.smem = (size_t)wpc * warp_smem_words(c.sh_slots, np, kill) * 8;
  // the attribute belongs to the kernel, not to this plan: always the
  // largest size any plan launches with (most warps, every slot in shared
  // memory), so plans alive at the same time never shrink it for each other
  // both depend only on the device, the kernel and the launch shape: done
  // once per process and shape (a serving loop builds plans all the time)
  static std::mutex mu;
  static std::map<std::tuple<int, const void *, int, size_t>, int> known;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(dev, (const void *)kern, wpc, c.smem);
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = known.find(key);
    if (it != known.end()) per_sm = it->second;
  }
  if (!per_sm) {
    set_smem(kern, (size_t)OMPDART_MAX_WPC * warp_smem_words(sh_words / (64 * np), np, kill) * 8);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * wpc, c.smem) != cudaSuccess || per_sm < 1)
      per_sm = 1;
    std::lock_guard<std::mutex> lk(mu);
    known[key] = per_sm;
  }
  const long long need_ctas = ((long long)n_items + wpc - 1) / wpc;
  c.grid = (int)std::max<long long>(1, std::min<long long>(need_ctas, (long long)per_sm * n_sm));
  return c;
}
}  // namespace

// Summary records of a block with call pseudo-accesses, folded on the host
// by the local rule (Sec. IV-D) with each call contributing its callee's
// reads first, then its net effect (Sec. IV-C): one record per variable the
// block touches, in the device record format.  `idx` is scratch of size V
// filled with -1 (restored on return).
static void fold_call_block(const uint32_t *acc, int a0, int a1, const CallHost &calls, int row_base, int W,
                            std::vector<int32_t> &idx, std::vector<uint32_t> *out) {
  struct St { int32_t v; uint8_t last[2], ue[2], def; };
  std::vector<St> st;
  auto at = [&](int v) -> St & {
    if (idx[v] < 0) {
      idx[v] = (int32_t)st.size();
      st.push_back(St{v, {0, 0}, {0, 0}, 0});
    }
    return st[idx[v]];
  };
  auto read = [](St &x, int S) {
    x.last[S] = 1;
    if (!x.ue[S]) x.ue[S] = 1;
  };
  auto wrote = [](St &x) {
    if (!x.ue[0]) x.ue[0] = 2;
    if (!x.ue[1]) x.ue[1] = 2;
    x.def = 1;
  };
  for (int i = a0; i < a1; ++i) {
    const uint32_t a = acc[i];
    if (a >> 31) {
      const uint64_t *row = calls.planes + (size_t)(row_base + (int)(a & 0x7FFFFFFFu)) * 7 * W;
      for (int w = 0; w < W; ++w) {
        uint64_t any = 0;
        for (int k = 0; k < 7; ++k) any |= row[(size_t)k * W + w];
        while (any) {
          const int bit = __builtin_ctzll(any);
          any &= any - 1;
          const uint64_t m = 1ull << bit;
          St &x = at(w * 64 + bit);
          if (row[0 * W + w] & m) read(x, 0);
          if (row[1 * W + w] & m) read(x, 1);
          if (row[2 * W + w] & m) x.last[0] = 1; else if (row[3 * W + w] & m) x.last[0] = 2;
          if (row[4 * W + w] & m) x.last[1] = 1; else if (row[5 * W + w] & m) x.last[1] = 2;
          if (row[6 * W + w] & m) wrote(x);
        }
      }
      continue;
    }
    St &x = at((int)(a & 0xFFFFFFu));
    const int kind = (int)((a >> 24) & 3u), S = (int)((a >> 26) & 1u);
    if (kind & 1) read(x, S);
    if (kind & 2) {
      x.last[S] = 1;
      x.last[1 - S] = 2;
      wrote(x);
    }
  }
  for (const St &x : st) {
    uint32_t r = (uint32_t)x.v;
    if (x.last[0] == 1) r |= R_GH;
    if (x.last[0] == 2) r |= R_KH;
    if (x.last[1] == 1) r |= R_GD;
    if (x.last[1] == 2) r |= R_KD;
    if (x.ue[0] == 1) r |= R_UH;
    if (x.ue[1] == 1) r |= R_UD;
    if (x.def) r |= R_DF;
    out->push_back(r);
    idx[x.v] = -1;
  }
}

ScanState *scan_create(const Ingest &g, const int32_t *acc_off, const uint32_t *acc, const CallHost &calls,
                       int32_t *cfg_err, DevPlan &p, int chunk_target, int keep_states, std::string *err, int wpc) {
  ScanState *st = new ScanState();
  HostVec<PosMeta> meta;
  std::vector<LoopMeta> loops;
  std::vector<ChunkMeta> chunks;
  std::vector<CarrySrc> csrc;
  HostVec<int32_t> fin_slot, out_slot, out_pos;
  std::vector<int32_t> lat_slot, lat_ent, bend_loop, srcent, exit_slot;
  // short chunks give more independent walks (one warp each) and shorter
  // longest walks; 32 positions measured fastest on the 2^20-block CFG
  if (chunk_target <= 0) chunk_target = 32;
  // The accesses in position order need only the order, so on a large CFG
  // they are laid out on a second host thread while build_meta runs.
  struct AccPos {
    int32_t pacc_beg;
    int16_t nacc;
    int16_t flags;
  };
  HostVec<uint32_t> acc_p;
  HostVec<int2> acc_link;
  std::vector<AccPos> apos;
  std::string acc_err;
  auto access_pass = [&]() {
    // accesses in position order: a block's own accesses with same-variable
    // links inside the block (a short list for the usual handful of accesses,
    // a hash map for long blocks), or, for a block with calls, its folded
    // summary records.  Positions are independent once their offsets are
    // known: a first parallel pass sizes them (folding the call blocks into
    // per-thread buffers), a second fills them, over the same ranges.
    constexpr int kThreads = kHostThreads, kMinPos = 4096;
    struct Folded {
      std::vector<uint32_t> recs;
      std::vector<std::pair<int32_t, int32_t>> at;  // (position, first record), in position order
      std::vector<int32_t> var_idx;
    };
    std::vector<Folded> fold(kThreads);
    std::vector<int32_t> cnt(g.M + 1, 0);
    std::atomic<bool> too_big{false};
    // a call block of a CFG given with the same arrays and table as an earlier
    // one takes that CFG's folded records (the same position in its order)
    auto twin = [&](int i) -> int {
      if (calls.same_as.empty()) return -1;
      const int cfg = (int)(std::upper_bound(g.cfg_pos_off.begin(), g.cfg_pos_off.end(), i) - g.cfg_pos_off.begin()) - 1;
      const int f = calls.same_as[cfg];
      return f == cfg ? -1 : i - g.cfg_pos_off[cfg] + g.cfg_pos_off[f];
    };
    std::vector<int32_t> twin_pos;  // call positions that copy a twin's records
    std::mutex twin_mu;
    const int T = parallel_ranges(g.M, kMinPos, kThreads, [&](int t, int lo, int hi) {
      Folded &fd = fold[t];
      std::vector<int32_t> mine;
      for (int i = lo; i < hi; ++i) {
        const int b = g.order[i], a0 = acc_off[b], a1 = acc_off[b + 1];
        bool has_call = false;
        for (int k = a0; k < a1 && calls.rows; ++k) has_call |= (acc[k] >> 31) != 0;
        int n = a1 - a0;
        if (has_call) {
          if (twin(i) >= 0) {
            mine.push_back(i);
            continue;
          }
          if (fd.var_idx.empty()) fd.var_idx.assign((size_t)p.W * 64, -1);
          const int cfg =
              (int)(std::upper_bound(g.cfg_pos_off.begin(), g.cfg_pos_off.end(), i) - g.cfg_pos_off.begin()) - 1;
          const size_t r0 = fd.recs.size();
          fold_call_block(acc, a0, a1, calls, calls.row_base.empty() ? 0 : calls.row_base[cfg], p.W, fd.var_idx,
                          &fd.recs);
          fd.at.push_back({i, (int32_t)r0});
          n = (int)(fd.recs.size() - r0);
        }
        if (n > 32767) too_big = true;
        cnt[i + 1] = n;
      }
      std::lock_guard<std::mutex> lk(twin_mu);
      twin_pos.insert(twin_pos.end(), mine.begin(), mine.end());
    });
    // where each folded position's records are: (thread, first record)
    std::unordered_map<int32_t, std::pair<int, int32_t>> folded_at;
    std::vector<uint8_t> is_twin;
    if (!twin_pos.empty()) {
      for (int t = 0; t < T; ++t)
        for (const auto &x : fold[t].at) folded_at.emplace(x.first, std::make_pair(t, x.second));
      is_twin.assign(g.M, 0);
      for (int i : twin_pos) is_twin[i] = 1;
    }
    for (int i : twin_pos) cnt[i + 1] = cnt[twin(i) + 1];
    if (too_big) {
      acc_err = "a block with more than 32767 accesses (or variables touched by its calls)";
      return;
    }
    for (int i = 0; i < g.M; ++i) cnt[i + 1] += cnt[i];
    acc_p.resize(cnt[g.M]);  // filled in full by the second pass
    acc_link.resize(cnt[g.M]);
    apos.resize(g.M);
    parallel_ranges(g.M, kMinPos, kThreads, [&](int t, int lo, int hi) {
      const Folded &fd = fold[t];
      size_t next_fold = 0;
      std::vector<std::pair<int32_t, int32_t>> seen;  // (variable, its latest access) within the block
      std::unordered_map<int32_t, int32_t> latest;
      for (int i = lo; i < hi; ++i) {
        const int b = g.order[i], a0 = acc_off[b], a1 = acc_off[b + 1], base = cnt[i];
        AccPos &m = apos[i];
        m.pacc_beg = base;
        m.nacc = (int16_t)(cnt[i + 1] - base);
        m.flags = 0;
        if (next_fold < fd.at.size() && fd.at[next_fold].first == i) {
          const int r0 = fd.at[next_fold++].second;
          std::copy(fd.recs.begin() + r0, fd.recs.begin() + r0 + m.nacc, acc_p.begin() + base);
          std::fill(acc_link.begin() + base, acc_link.begin() + base + m.nacc, make_int2(LINK_RECORD, -1));
          m.flags = PM_RECORDS;
          continue;
        }
        if (!is_twin.empty() && is_twin[i]) {
          const auto it = folded_at.find(twin(i));
          if (it != folded_at.end()) {  // a call block folded for its twin
            const std::vector<uint32_t> &recs = fold[it->second.first].recs;
            std::copy(recs.begin() + it->second.second, recs.begin() + it->second.second + m.nacc,
                      acc_p.begin() + base);
            std::fill(acc_link.begin() + base, acc_link.begin() + base + m.nacc, make_int2(LINK_RECORD, -1));
            m.flags = PM_RECORDS;
            continue;
          }
        }
        std::copy(acc + a0, acc + a1, acc_p.begin() + base);
        if (a1 - a0 <= 64) {
          seen.clear();
          for (int k = a0; k < a1; ++k) {
            const int v = (int)(acc[k] & 0xFFFFFFu), idx = base + (k - a0);
            int first = idx;
            for (auto &sv : seen)
              if (sv.first == v) {
                first = acc_link[sv.second].x;
                acc_link[sv.second].y = idx;
                sv.second = idx;
                break;
              }
            if (first == idx) seen.push_back({v, idx});
            acc_link[idx] = make_int2(first, -1);
          }
        } else {
          latest.clear();
          for (int k = a0; k < a1; ++k) {
            const int v = (int)(acc[k] & 0xFFFFFFu), idx = base + (k - a0);
            auto it = latest.find(v);
            int first = idx;
            if (it != latest.end()) {
              first = acc_link[it->second].x;
              acc_link[it->second].y = idx;
              it->second = idx;
            } else {
              latest.emplace(v, idx);
            }
            acc_link[idx] = make_int2(first, -1);
          }
        }
      }
    });
  };
  TraceScope trace_bm("scan build_meta + accesses", g.M);
  bool meta_ok;
  if (g.M >= (1 << 14)) {  // (a thread start costs tens of microseconds)
    std::thread th(access_pass);
    meta_ok = build_meta(g, chunk_target, st, meta, loops, chunks, csrc, fin_slot, out_slot, out_pos, lat_slot,
                         lat_ent, bend_loop, srcent, exit_slot, err);
    th.join();
  } else {
    meta_ok = build_meta(g, chunk_target, st, meta, loops, chunks, csrc, fin_slot, out_slot, out_pos, lat_slot,
                         lat_ent, bend_loop, srcent, exit_slot, err);
    if (meta_ok) access_pass();
  }
  if (meta_ok && !acc_err.empty()) {
    if (err) *err = acc_err;
    meta_ok = false;
  }
  if (!meta_ok) {
    delete st;
    return nullptr;
  }
  parallel_ranges(g.M, 1 << 15, kHostThreads, [&](int, int lo, int hi) {
    for (int i = lo; i < hi; ++i) {
      PosMeta &m = meta[i];
      m.acc_beg = acc_off[m.blk];
      m.pacc_beg = apos[i].pacc_beg;
      m.nacc = apos[i].nacc;
      m.flags = apos[i].flags;
    }
  });
  trace_bm.next("scan uploads: edge entries", g.M);
  std::vector<int2> fin_pk(fin_slot.size()), out_pk(out_slot.size());
  // in-edge entries: {source slot, loop-entry edge or -1}
  parallel_ranges((int)fin_pk.size(), 1 << 17, kHostThreads, [&](int, int lo, int hi) {
    for (int k = lo; k < hi; ++k) fin_pk[k] = make_int2(fin_slot[k], g.fin_ent[k]);
  });
  parallel_ranges((int)out_pk.size(), 1 << 17, kHostThreads, [&](int, int lo, int hi) {
    for (int k = lo; k < hi; ++k) out_pk[k] = make_int2(out_slot[k], out_pos[k]);
  });
  const int W = p.W, C = st->C, G = (W + 63) / 64;
  st->G = G;
  ScanDev &sd = st->sd;
  sd.C = C;
  sd.G = G;
  sd.fslots = st->fslots;
  sd.bslots = st->bslots;
  sd.keep_states = keep_states;
  sd.cfg_err = cfg_err;
  // work order: costliest chunks first (their walks bound the launch); a
  // position inside d nested loops may be walked up to about 2^d times
  std::vector<int32_t> work(C);
  std::vector<long long> cost(C, 0);
  parallel_ranges(C, 2048, kHostThreads, [&](int, int lo, int hi) {
    for (int c = lo; c < hi; ++c) {
      work[c] = c;
      for (int i = chunks[c].s; i < chunks[c].e; ++i) {
        const int l = g.inner_loop[g.order[i]];
        cost[c] += 1ll << std::min(l >= 0 ? g.loop_depth[l] : 0, 4);
      }
    }
  });
  trace_bm.next("scan work order", C);
  std::stable_sort(work.begin(), work.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<int32_t> lant_work(g.L);
  for (int l = 0; l < g.L; ++l) lant_work[l] = l;
  std::stable_sort(lant_work.begin(), lant_work.end(), [&](int a, int b) {
    return loops[a].pend - loops[a].ph > loops[b].pend - loops[b].ph;
  });
  sd.n_loops = g.L;
  bool ok = true;
  auto chk = [&](const void *x) { ok = ok && x; };
  trace_bm.next("scan uploads: copies", g.M);
  chk(sd.meta = st->up(meta));
  chk(sd.loops = st->up(loops));
  chk(sd.chunks = st->up(chunks));
  chk(sd.csrc = st->up(csrc));
  chk(sd.fin_pk = st->up(fin_pk));
  chk(sd.out_pk = st->up(out_pk));
  chk(sd.acc_p = st->up(acc_p));
  chk(sd.rec_p = st->alloc<uint32_t>(acc_p.size()));
  chk(sd.emit_p = st->alloc<uint32_t>(acc_p.size()));
  chk(sd.acc_link = st->up(acc_link));
  sd.n_acc_p = (long long)acc_p.size();
  chk(sd.lat_slot = st->up(lat_slot));
  chk(sd.lat_ent = st->up(lat_ent));
  chk(sd.exit_slot = st->up(exit_slot));
  {
    std::vector<int4> bend_info(bend_loop.size());
    for (size_t q = 0; q < bend_loop.size(); ++q) {
      const LoopMeta &lm = loops[bend_loop[q]];
      bend_info[q] = make_int4(lm.depth, lm.ph, lm.pend, meta[lm.ph].bslot);
    }
    chk(sd.bend_info = st->up(bend_info));
  }
  chk(sd.srcent = st->up(srcent));
  chk(sd.work = st->up(work));
  chk(sd.lant_work = st->up(lant_work));
  chk(sd.queue = st->alloc<int32_t>(Q_SLOTS));
  trace_bm.next("scan shapes", g.M);
  // launch shapes (persistent: the grid is what fits on the GPU at once)
  {
    wpc = clamp_wpc(wpc);
    int dev = 0, n_sm = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int items = C * G;
    const int NPS = BwdPlanes<M_SUM>::NP;
    st->shape[CK_BSUM] = chain_shape(k_bwd_chain<M_SUM>, st->bslots, NPS, false, BWD_SH_WORDS, wpc, items, n_sm);
    st->shape[CK_BLANT] = chain_shape(k_bwd_chain<M_LANT>, st->bslots, BwdPlanes<M_LANT>::NP, true,
                                      OMPDART_LANT_SH_WORDS, wpc, std::max(1, g.L) * G, n_sm);
    st->shape[CK_FSUM] = chain_shape(k_fwd_chain<K_HP>, st->fslots, 2, false, FWD_SH_WORDS, wpc, items, n_sm);
    st->shape[CK_BNA] = p.ant_dm ? chain_shape(k_bwd_chain<M_NA>, st->bslots, BwdPlanes<M_NA>::NP, false, BWD_SH_WORDS,
                                               wpc, items, n_sm)
                                 : ChainShape{};
    chain_shape(k_fwd_chain<K_D>, st->fslots, 2, false, FWD_SH_WORDS, wpc, items, n_sm);
    chain_shape(k_fwd_chain<K_H>, st->fslots, 2, false, FWD_SH_WORDS, wpc, items, n_sm);
  }
  int max_warps = 1;
  for (const ChainShape &c : st->shape) max_warps = std::max(max_warps, c.grid * c.wpc);
  // slots beyond those a kernel keeps in shared memory spill to a per-warp area
  {
    const int fwd = std::max(0, st->fslots - st->shape[CK_FSUM].sh_slots) * 2 * 64;
    const int lant = std::max(0, st->bslots - st->shape[CK_BLANT].sh_slots) * BwdPlanes<M_LANT>::NP * 64;
    const int NPS = BwdPlanes<M_SUM>::NP;
    const int live = std::max(0, st->bslots - st->shape[CK_BSUM].sh_slots) * NPS * 64;
    sd.spill_stride = std::max({64, fwd, lant, live});
  }
  st->spill_region = (size_t)std::max(1, sd.spill_stride) * max_warps;
  chk(sd.spill = st->alloc<uint64_t>(st->spill_region * 3));  // one region per branch of a run
  st->eager = p.ant_dm != nullptr;
  const size_t n_maps = st->eager ? 3 : 2;  // chunk maps: liveness, forward problems (, not anticipated)
  chk(sd.gsum = st->alloc<uint64_t>(n_maps * C * W));
  chk(sd.psum = st->alloc<uint64_t>(n_maps * C * W));
  if (ok) {  // chunks that end a CFG never write their map: keep it defined
    cudaMemset(sd.gsum, 0, sizeof(uint64_t) * n_maps * C * W);
    cudaMemset(sd.psum, 0, sizeof(uint64_t) * n_maps * C * W);
  }
  chk(sd.carry = st->alloc<uint64_t>(n_maps * C * W));
  {
    // chunk-carry scan: about two CTAs per SM over the word columns' segments
    int dev = 0, n_sm = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    // about two CTAs per SM over the column blocks' segments, a few chunks per run
    const int wb = scan_wb(W), gx = (W + wb - 1) / wb, runs = SCAN_T / wb;
    sd.seg_n = std::max(1, std::min({2 * n_sm / gx, (C + 4 * runs - 1) / (4 * runs), 1024}));
    chk(sd.seg_g = st->alloc<uint64_t>(n_maps * sd.seg_n * W));  // one region per branch
    chk(sd.seg_p = st->alloc<uint64_t>(n_maps * sd.seg_n * W));
  }
  chk(sd.d_src = st->alloc<uint64_t>((size_t)std::max(1, g.K) * W));
  trace_bm.next("scan emission items", g.M);
  // emission items: runs of at most EMIT_SPAN positions inside one chunk,
  // each with a record stream per word group, in position order, so each
  // chunk's (and each CFG's) records are contiguous
  std::vector<int2> emit_rng;
  st->chunk_item0.assign(C + 1, 0);
  for (int c = 0; c < C; ++c) {
    st->chunk_item0[c] = (int32_t)emit_rng.size();
    for (int i = chunks[c].s; i < chunks[c].e; i += EMIT_SPAN)
      emit_rng.push_back(make_int2(i, std::min(chunks[c].e, i + EMIT_SPAN)));
  }
  st->chunk_item0[C] = (int32_t)emit_rng.size();
  sd.n_emit = (int)emit_rng.size();
  chk(sd.emit_rng = st->up(emit_rng));
  st->n_streams = sd.n_emit * G;
  sd.n_streams = st->n_streams;
  st->h_rec_cap.assign(st->n_streams, 0);
  for (int k = 0; k < sd.n_emit; ++k)
    for (int wg = 0; wg < G; ++wg) st->h_rec_cap[k * G + wg] = 32 + 2 * (emit_rng[k].y - emit_rng[k].x);
  // affine pairs of the summary walks and where each position's carry comes from
  {
    std::vector<int32_t> pos_chunk(g.M), src_pos(std::max(1, g.K), 0);
    parallel_ranges(C, 2048, kHostThreads, [&](int, int lo, int hi) {
      for (int c = lo; c < hi; ++c)
        for (int i = chunks[c].s; i < chunks[c].e; ++i) pos_chunk[i] = c;
    });
    for (int k = 0; k < g.K; ++k) src_pos[k] = g.pos[g.ent_src[k]];
    chk(sd.pos_chunk = st->up(pos_chunk));
    chk(sd.src_pos = st->up(src_pos));
    std::vector<int32_t> pos_loop(g.M);
    parallel_ranges(g.M, 1 << 16, kHostThreads, [&](int, int lo, int hi) {
      for (int i = lo; i < hi; ++i) pos_loop[i] = g.inner_loop[g.order[i]];
    });
    chk(sd.pos_loop = st->up(pos_loop));
    chk(sd.loop_up = st->up(g.loop_parent));
    std::vector<int32_t> loop_root(g.L);
    for (int l = 0; l < g.L; ++l) {  // parents come first (headers in walk order)
      const int up = g.loop_parent[l];
      loop_root[l] = up < 0 ? l : loop_root[up];
    }
    chk(sd.loop_root = st->up(loop_root));
    std::vector<int32_t> loop_d2(g.L);
    for (int l = 0; l < g.L; ++l) {
      const int up = g.loop_parent[l];
      loop_d2[l] = up < 0 ? -1 : g.loop_parent[up] < 0 ? l : loop_d2[up];
    }
    chk(sd.loop_d2 = st->up(loop_d2));
    trace_bm.next("scan state planes", g.M);
    chk(sd.hdr_g = st->alloc<uint64_t>((size_t)std::max(1, g.L) * W));
    chk(sd.hdr_p = st->alloc<uint64_t>((size_t)std::max(1, g.L) * W));
    chk(sd.hdr_ag = st->alloc<uint64_t>((size_t)std::max(1, g.L) * W));
    chk(sd.hdr_ap = st->alloc<uint64_t>((size_t)std::max(1, g.L) * W));
    chk(sd.hdrl_g = st->alloc<uint64_t>((size_t)std::max(1, g.L) * W));
    chk(sd.hdrl_p = st->alloc<uint64_t>((size_t)std::max(1, g.L) * W));
    chk(sd.hdrl2_g = st->alloc<uint64_t>((size_t)std::max(1, g.L) * W));
    chk(sd.hdrl2_p = st->alloc<uint64_t>((size_t)std::max(1, g.L) * W));
    chk(sd.hdrl2_a = st->alloc<uint64_t>((size_t)std::max(1, g.L) * W));
    const size_t NW = (size_t)g.N * W, KW = (size_t)std::max(1, g.K) * W;
    chk(sd.pair_a = st->alloc<uint64_t>(NW));
    chk(sd.pair_a2 = st->alloc<uint64_t>(NW));
    if (st->eager) {
      const size_t LW = (size_t)std::max(1, g.L) * W;
      chk(st->na_pg = st->alloc<uint64_t>(NW));
      chk(st->na_pp = st->alloc<uint64_t>(NW));
      chk(st->na_pa = st->alloc<uint64_t>(NW));
      chk(st->na_pa2 = st->alloc<uint64_t>(NW));
      chk(st->na_hg = st->alloc<uint64_t>(LW));
      chk(st->na_hp = st->alloc<uint64_t>(LW));
      chk(st->na_h2g = st->alloc<uint64_t>(LW));
      chk(st->na_h2p = st->alloc<uint64_t>(LW));
      chk(st->na_h2a = st->alloc<uint64_t>(LW));
    }
    chk(sd.pair_g = st->alloc<uint64_t>(NW));
    chk(sd.pair_p = st->alloc<uint64_t>(NW));
    chk(sd.pair_gd = st->alloc<uint64_t>(NW));
    chk(sd.pair_pd = st->alloc<uint64_t>(NW));
    sd.pair_g2 = sd.pair_p2 = nullptr;
    if (keep_states) {
      chk(sd.pair_g2 = st->alloc<uint64_t>(NW));
      chk(sd.pair_p2 = st->alloc<uint64_t>(NW));
    }
    chk(sd.src_g = st->alloc<uint64_t>(KW));
    chk(sd.src_p = st->alloc<uint64_t>(KW));
  }
  trace_bm.next("scan record streams", g.M);
  chk(st->d_rec_cap = st->alloc<int32_t>(st->n_streams));
  chk(st->d_rec_base = st->alloc<int32_t>(st->n_streams));
  chk(sd.rec_cnt = st->alloc<int32_t>(st->n_streams + 1));
  chk(st->offs = st->alloc<int32_t>(st->n_streams + 1));
  chk(st->part = st->alloc<int32_t>(st->n_streams / PF_TILE + 2));
  chk(st->init = st->alloc<uint64_t>((size_t)W * p.n_cfg));
  if (ok) ok = scan_set_streams(st);
  for (int k = 0; k < 2 && ok; ++k) ok = cudaStreamCreateWithFlags(&st->side[k], cudaStreamNonBlocking) == cudaSuccess;
  for (int k = 0; k < 3 && ok; ++k) ok = cudaEventCreateWithFlags(&st->ev[k], cudaEventDisableTiming) == cudaSuccess;
  sd.rec_cap = st->d_rec_cap;
  sd.rec_base = st->d_rec_base;
  if (!ok) {
    if (err) *err = "device allocation for the scan solver failed";
    delete st;
    return nullptr;
  }
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

// the emission pass and the gather of its record streams
static int run_emission(ScanState *st, const DevPlan &p, cudaStream_t s, Prof *pf) {
  ScanDev &sd = st->sd;
  int32_t *offs = st->offs;
  const long long nw = (long long)sd.n_emit * sd.G;
  ScanDev se = sd;  // the forward problems' chunk carries (host validity's, the last scanned)
  se.carry = sd.carry + (size_t)sd.C * p.W;
  PROF("emit");
  k_emit<<<grid_of(nw * 32, 32 * EMIT_WARPS), 32 * EMIT_WARPS, 0, s>>>(p, se, st->init);
  PROF("streams_prefix");
  const int n_parts = (sd.n_streams + PF_TILE - 1) / PF_TILE;
  k_streams_sums<<<std::max(1, n_parts), PF_T, 0, s>>>(sd, st->part, p.status);
  k_streams_top<<<1, PF_T, 0, s>>>(st->part, n_parts, p.status);
  k_streams_offsets<<<std::max(1, n_parts), PF_T, 0, s>>>(sd, st->part, offs);
  PROF("streams_copy");
  k_streams_copy<<<grid_of((long long)sd.n_streams * 32, 256), 256, 0, s>>>(sd, offs, p.xfer, p.xfer_cap);
  return 5;
}

// launch a persistent chain kernel with its shape; qslot: its work-queue head
template <class K>
void chain_launch(K kern, const ChainShape &cs, const DevPlan &p, const ScanDev &sd, int qslot, cudaStream_t s) {
  ScanDev sd2 = sd;
  sd2.sh_slots = cs.sh_slots;
  kern<<<cs.grid, 32 * cs.wpc, cs.smem, s>>>(p, sd2, qslot);
}

// The chunk-carry scan of one problem: segment maps, then the carries (one
// launch when a column is one segment).  Returns the launches.
static int scan_carries(const ScanDev &x, int W, int backward, const uint64_t *init, cudaStream_t s) {
  const int wb = scan_wb(W);
  const dim3 grid((W + wb - 1) / wb, x.seg_n);
  if (x.seg_n > 1) k_scan_carry<0><<<grid, SCAN_T, 0, s>>>(x, W, wb, backward, init);
  k_scan_carry<1><<<grid, SCAN_T, 0, s>>>(x, W, wb, backward, init);
  return x.seg_n > 1 ? 2 : 1;
}

// One run: local summaries; per phase a summary walk that leaves every
// position's affine pair, the scan of the chunk maps, and a parallel resolve
// of the pairs with the carries; then the emission from the final states.
// The phases that need nothing of each other run on separate streams so
// the tails of their walks overlap:
//   side 0: loop masks;   side 1: liveness;
//   caller's stream: plain host validity, device validity (after the masks),
//                    host validity and emission (after liveness).
// With per-kernel profiling on, everything runs on the caller's stream.
int enqueue_scan_solver(ScanState *st, const DevPlan &p, cudaStream_t s, Prof *pf) {
  ScanDev &sd = st->sd;
  const int W = p.W, C = sd.C;
  uint64_t *init = st->init;
  int n = 0;
  const long long nw = (long long)p.M * W, kw = (long long)p.K * W;
  const bool fork = pf == nullptr;
  cudaStream_t s_lant = fork ? st->side[0] : s, s_live = fork ? st->side[1] : s;
  // per-branch views: own spill region and chunk maps
  ScanDev sl = sd, sm = sd, sq = sd;  // liveness, masks, the main pipeline
  sl.spill = sd.spill + st->spill_region;
  sm.spill = sd.spill;
  sq.spill = sd.spill + 2 * st->spill_region;
  sq.gsum = sd.gsum + (size_t)C * W;
  sq.psum = sd.psum + (size_t)C * W;
  sq.carry = sd.carry + (size_t)C * W;
  sq.seg_g = sd.seg_g + (size_t)sd.seg_n * W;
  sq.seg_p = sd.seg_p + (size_t)sd.seg_n * W;
  cudaMemsetAsync(p.acc_flag, 0, (size_t)p.A, s);
  cudaMemsetAsync(sd.queue, 0, sizeof(int32_t) * Q_SLOTS, s);
  PROF("local_summary");
  k_local_summary_pos<<<grid_of(sd.n_acc_p, 256), 256, 0, s>>>(sd); ++n;
  if (fork) {
    cudaEventRecord(st->ev[0], s);
    cudaStreamWaitEvent(s_lant, st->ev[0], 0);
    cudaStreamWaitEvent(s_live, st->ev[0], 0);
  }
  // ---- loop masks: need within the loop body, kills anywhere in it
  if (p.L) {
    PROF("loop_masks");
    chain_launch(k_bwd_chain<M_LANT>, st->shape[CK_BLANT], p, sm, 2, s_lant); ++n;
  }
  // ---- eager `to' placement: AntDm, as the complement of "not anticipated"
  // (a backward may problem shaped like liveness), after the masks on
  // their stream and in their spill region; the edge constants wait for both
  if (st->eager) {
    ScanDev sn = sd;
    sn.spill = sd.spill;
    sn.pair_g = st->na_pg;
    sn.pair_p = st->na_pp;
    sn.pair_a = st->na_pa;
    sn.pair_a2 = st->na_pa2;
    sn.hdrl_g = st->na_hg;
    sn.hdrl_p = st->na_hp;
    sn.hdrl2_g = st->na_h2g;
    sn.hdrl2_p = st->na_h2p;
    sn.hdrl2_a = st->na_h2a;
    sn.gsum = sd.gsum + (size_t)2 * C * W;
    sn.psum = sd.psum + (size_t)2 * C * W;
    sn.carry = sd.carry + (size_t)2 * C * W;
    sn.seg_g = sd.seg_g + (size_t)2 * sd.seg_n * W;
    sn.seg_p = sd.seg_p + (size_t)2 * sd.seg_n * W;
    PROF("antdm_summary");
    chain_launch(k_bwd_chain<M_NA>, st->shape[CK_BNA], p, sn, 9, s_lant); ++n;
    PROF("antdm_scan");
    n += scan_carries(sn, W, 1, nullptr, s_lant);
    PROF("antdm_resolve");
    k_resolve<RV_NA><<<grid_of((nw + 1) / 2, 256), 256, 0, s_lant>>>(p, sn, sn.pair_g, sn.pair_p, p.ant_dm); ++n;
  }
  // ---- liveness (backward)
  PROF("live_summary");
  chain_launch(k_bwd_chain<M_SUM>, st->shape[CK_BSUM], p, sl, 0, s_live); ++n;
  PROF("live_scan");
  n += scan_carries(sl, W, 1, nullptr, s_live);
  PROF("live_resolve");
  k_resolve<RV_LIVE><<<grid_of((nw + 1) / 2, 256), 256, 0, s_live>>>(p, sl, sl.pair_g, sl.pair_p, p.live); ++n;
  if (fork) {
    cudaEventRecord(st->ev[1], s_lant);
    cudaEventRecord(st->ev[2], s_live);
  }
  // ---- plain host validity (needed at loop-entry sources only)
  PROF("entry_stale");
  k_entry_stale<<<grid_of((long long)W * p.n_cfg, 128), 128, 0, s>>>(p.entry_h, p.top, init, W, p.n_cfg); ++n;
  PROF("hp_summary");
  chain_launch(k_fwd_chain<K_HP>, st->shape[CK_FSUM], p, sq, 3, s); ++n;
  PROF("fwd_scan");
  n += scan_carries(sq, W, 0, init, s);
  if (p.L) {
    PROF("loop_abs");
    k_loop_abs<<<grid_of((long long)p.L * W, 256), 256, 0, s>>>(p, sq); ++n;
  }
  if (fork) cudaStreamWaitEvent(s, st->ev[1], 0);  // the masks
  if (p.K) {
    PROF("src_resolve");
    k_resolve_src<<<grid_of(kw, 256), 256, 0, s>>>(p, sq, 0); ++n;
  }
  // ---- device validity
  PROF("entry_stale");
  k_entry_stale<<<grid_of((long long)W * p.n_cfg, 128), 128, 0, s>>>(p.entry_d, p.top, init, W, p.n_cfg); ++n;
  PROF("d_summary");
  chain_launch(k_fwd_chain<K_D>, st->shape[CK_FSUM], p, sq, 5, s); ++n;
  PROF("fwd_scan");
  n += scan_carries(sq, W, 0, init, s);
  if (p.L) {
    PROF("loop_abs");
    k_loop_abs<<<grid_of((long long)p.L * W, 256), 256, 0, s>>>(p, sq); ++n;
  }
  PROF("d_resolve");
  k_resolve<RV_VALID><<<grid_of((nw + 1) / 2, 256), 256, 0, s>>>(p, sq, sq.pair_gd, sq.pair_pd, p.d_in); ++n;
  if (sq.pair_g2) {
    k_resolve<RV_VALID><<<grid_of((nw + 1) / 2, 256), 256, 0, s>>>(p, sq, sq.pair_g2, sq.pair_p2, p.d_out); ++n;
  }
  // ---- host validity (its exit states), then the emission
  if (fork) cudaStreamWaitEvent(s, st->ev[2], 0);  // liveness (also in the constants of region exits)
  if (p.K) {
    PROF("src_resolve");
    k_resolve_src<<<grid_of(kw, 256), 256, 0, s>>>(p, sq, 1); ++n;
  }
  PROF("entry_stale");
  k_entry_stale<<<grid_of((long long)W * p.n_cfg, 128), 128, 0, s>>>(p.entry_h, p.top, init, W, p.n_cfg); ++n;
  PROF("h_summary");
  chain_launch(k_fwd_chain<K_H>, st->shape[CK_FSUM], p, sq, 7, s); ++n;
  PROF("fwd_scan");
  n += scan_carries(sq, W, 0, init, s);
  if (p.L) {
    PROF("loop_abs");
    k_loop_abs<<<grid_of((long long)p.L * W, 256), 256, 0, s>>>(p, sq); ++n;
  }
  // (H_out is resolved by the emission)
  n += run_emission(st, p, s, pf);
  return n;
}

int enqueue_scan_edges(ScanState *st, const DevPlan &p, cudaStream_t s, Prof *pf) {
  // after the record buffers grew: redo the emission and the gather (the
  // entry rows in `init' are still the host-validity ones)
  return run_emission(st, p, s, pf);
}


// first gathered record of each chunk (and the total at index C), after a
// completed run: the offsets of the chunk's first stream
bool scan_chunk_record_offsets(const ScanState *st, cudaStream_t s, std::vector<int32_t> *out, int32_t total) {
  std::vector<int32_t> offs(st->n_streams);
  if (st->n_streams &&
      (cudaMemcpyAsync(offs.data(), st->offs, sizeof(int32_t) * st->n_streams, cudaMemcpyDeviceToHost, s) !=
           cudaSuccess ||
       cudaStreamSynchronize(s) != cudaSuccess))
    return false;
  out->assign(st->C + 1, total);
  for (int c = 0; c < st->C; ++c) (*out)[c] = offs[(size_t)st->chunk_item0[c] * st->G];
  return true;
}

void scan_destroy(ScanState *st) { delete st; }

long long scan_h2d_bytes(const ScanState *st) { return st ? st->h2d : 0; }

long long scan_device_bytes(const ScanState *st) { return st ? st->bytes : 0; }

}  // namespace ompdart
