// summary.cu -- callee side-effect summaries (Sec. IV-C) on the device:
// ompdart_summarize_batch / ompdart_summarize_callee.
//
// A summary is seven planes over the callee's variables:
//   ReqH, ReqD   anticipation at the entry with nothing live after the exit
//                (read in that space before any write, on some path);
//   GenS, KillS  net effect of plain validity (the local rule along paths,
//                no transfers): GenS = valid at every reachable exit from an
//                all-stale entry, KillS = stale at some reachable exit from an
//                all-valid entry;
//   MustDef      written on every path from the entry to a reachable exit.
// A callee without a reachable exit gets all-zero Gen/Kill/MustDef.
//
// Device layout: the callees of one run laid end to end by position
// (loop-ordered reverse post-order of each, reachable blocks only); one
// warp per (callee, 32-word group), lane = word.  Per lane:
//   1. each block's local functions for the lane's word, folded over its
//      accesses (a call: the callee row's reads, then its net effect);
//   2. anticipation AntH / AntD: reverse sweeps to the least fixed point;
//   3. plain validity as stale-domain affine pairs (G, P), entry (0, all):
//      forward sweeps (OR over predecessors) to the least fixed point; the
//      exit pair gives Kill = G and Gen = ~(G | P);
//   4. must-written: forward sweeps (AND over predecessors) from all-ones
//      to the greatest fixed point, entry 0.
// Every sweep loop is bounded by max_sweeps (OMPDART_E_NOCONVERGE).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ompdart.h"
#include "solver.h"

using namespace ompdart;

namespace {

enum SumPlane { S_GH, S_KH, S_GD, S_KD, S_UH, S_UD, S_DF, S_AH, S_AD, S_HG, S_HP, S_DG, S_DP, S_MW, S_COUNT };

struct SumDev {
  int n_items;
  const int32_t *item_cfg, *item_grp;  // [n_items] warp work items
  const int32_t *pos_off;              // [n+1] positions of each callee
  const int32_t *W;                    // [n]
  const long long *scr_off;            // [n] scratch (words)
  const long long *out_off;            // [n] output rows (words)
  const long long *row_off;            // [n] first word of each callee's call table
  const long long *top_off;            // [n] its valid-variable mask
  const int32_t *fin_off, *fin_pos;    // in-edges by position (global source positions)
  const int32_t *sout_off, *sout_pos;  // out-edges by position (global target positions)
  const int32_t *acc_off;              // [P+1] accesses of each position
  const uint32_t *acc;
  const uint64_t *calls, *top;
  uint64_t *scr, *out;
  int32_t *status;                     // [n] per callee
  int max_sweeps;
};

__global__ void k_summarize(SumDev d) {
  const int item = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  if (item >= d.n_items) return;
  const int k = d.item_cfg[item], lane = threadIdx.x & 31;
  const int W = d.W[k], w = d.item_grp[item] * 32 + lane;
  const bool on = w < W;
  const int p0 = d.pos_off[k], M = d.pos_off[k + 1] - p0;
  const uint64_t top = on ? d.top[d.top_off[k] + w] : 0;
  uint64_t *scr = d.scr + d.scr_off[k];
  auto at = [&](int plane, int pos) -> uint64_t & { return scr[((size_t)plane * M + (pos - p0)) * W + w]; };
  // ---- 1. local functions of every block for this word
  for (int q = p0; q < p0 + M; ++q) {
    uint64_t gh = 0, kh = 0, gd = 0, kd = 0, uh = 0, ud = 0, df = 0;
    for (int i = d.acc_off[q]; i < d.acc_off[q + 1]; ++i) {
      const uint32_t a = d.acc[i];
      if (a >> 31) {
        if (!on) continue;
        const uint64_t *row = d.calls + d.row_off[k] + (size_t)(a & 0x7FFFFFFFu) * 7 * W;
        const uint64_t rh = row[w], rd = row[W + w], cgh = row[2 * W + w], ckh = row[3 * W + w] & ~cgh;
        const uint64_t cgd = row[4 * W + w], ckd = row[5 * W + w] & ~cgd, md = row[6 * W + w];
        uh |= rh & ~df;  // the callee's reads come first
        ud |= rd & ~df;
        gh = (gh | rh | cgh) & ~ckh;
        kh = (kh & ~(rh | cgh)) | ckh;
        gd = (gd | rd | cgd) & ~ckd;
        kd = (kd & ~(rd | cgd)) | ckd;
        df |= md;
        continue;
      }
      const int v = (int)(a & 0xFFFFFFu);
      if (!on || (v >> 6) != w) continue;
      const uint64_t bit = 1ull << (v & 63);
      const int kind = (int)((a >> 24) & 3u), dev = (int)((a >> 26) & 1u);
      if (kind & 1) {  // read: its space valid
        if (dev) { ud |= bit & ~df; gd |= bit; kd &= ~bit; }
        else     { uh |= bit & ~df; gh |= bit; kh &= ~bit; }
      }
      if (kind & 2) {  // write: its space valid, the other stale
        if (dev) { gd |= bit; kd &= ~bit; gh &= ~bit; kh |= bit; }
        else     { gh |= bit; kh &= ~bit; gd &= ~bit; kd |= bit; }
        df |= bit;
      }
    }
    if (on) {
      at(S_GH, q) = gh; at(S_KH, q) = kh; at(S_GD, q) = gd; at(S_KD, q) = kd;
      at(S_UH, q) = uh; at(S_UD, q) = ud; at(S_DF, q) = df;
      at(S_AH, q) = 0; at(S_AD, q) = 0;
      at(S_HG, q) = 0; at(S_HP, q) = 0; at(S_DG, q) = 0; at(S_DP, q) = 0;
      at(S_MW, q) = top;
    }
  }
  __syncwarp();
  bool ok = true;
  // ---- 2. anticipation (backward, least fixed point)
  for (int sweep = 0;; ++sweep) {
    if (sweep >= d.max_sweeps) { ok = false; break; }
    bool changed = false;
    for (int q = p0 + M - 1; q >= p0 && on; --q) {
      uint64_t oh = 0, od = 0;
      for (int e = d.sout_off[q]; e < d.sout_off[q + 1]; ++e) {
        oh |= at(S_AH, d.sout_pos[e]);
        od |= at(S_AD, d.sout_pos[e]);
      }
      const uint64_t dfq = at(S_DF, q);
      const uint64_t nh = at(S_UH, q) | (oh & ~dfq), nd = at(S_UD, q) | (od & ~dfq);
      if (nh != at(S_AH, q) || nd != at(S_AD, q)) {
        at(S_AH, q) = nh;
        at(S_AD, q) = nd;
        changed = true;
      }
    }
    if (!__any_sync(0xffffffffu, changed)) break;
  }
  // ---- 3. plain validity as stale-domain pairs, 4. must-written (forward)
  for (int sweep = 0; ok; ++sweep) {
    if (sweep >= d.max_sweeps) { ok = false; break; }
    bool changed = false;
    for (int q = p0; q < p0 + M && on; ++q) {
      uint64_t hg = 0, hp = 0, dg = 0, dp = 0, mw = ~0ull;
      if (q == p0) {  // the entry: nothing stale for G, everything for P; nothing written
        hp = dp = top;
        mw = 0;
      } else {
        for (int e = d.fin_off[q]; e < d.fin_off[q + 1]; ++e) {
          const int s = d.fin_pos[e];
          hg |= at(S_HG, s); hp |= at(S_HP, s);
          dg |= at(S_DG, s); dp |= at(S_DP, s);
          mw &= at(S_MW, s);
        }
      }
      const uint64_t th = at(S_GH, q) | at(S_KH, q), td = at(S_GD, q) | at(S_KD, q);
      const uint64_t nhg = at(S_KH, q) | (hg & ~th), nhp = hp & ~th;
      const uint64_t ndg = at(S_KD, q) | (dg & ~td), ndp = dp & ~td;
      const uint64_t nmw = (mw | at(S_DF, q)) & top;
      if (nhg != at(S_HG, q) || nhp != at(S_HP, q) || ndg != at(S_DG, q) || ndp != at(S_DP, q) ||
          nmw != at(S_MW, q)) {
        at(S_HG, q) = nhg; at(S_HP, q) = nhp; at(S_DG, q) = ndg; at(S_DP, q) = ndp; at(S_MW, q) = nmw;
        changed = true;
      }
    }
    if (!__any_sync(0xffffffffu, changed)) break;
  }
  if (!ok) {
    if (lane == 0) atomicExch(&d.status[k], OMPDART_E_NOCONVERGE);
    return;
  }
  if (!on) return;
  // ---- met over the reachable exits
  uint64_t eg_h = 0, ep_h = 0, eg_d = 0, ep_d = 0, mw = top;
  bool any_exit = false;
  for (int q = p0; q < p0 + M; ++q) {
    if (d.sout_off[q] != d.sout_off[q + 1]) continue;
    any_exit = true;
    eg_h |= at(S_HG, q); ep_h |= at(S_HP, q);
    eg_d |= at(S_DG, q); ep_d |= at(S_DP, q);
    mw &= at(S_MW, q);
  }
  uint64_t *o = d.out + d.out_off[k];
  o[w] = at(S_AH, p0);
  o[W + w] = at(S_AD, p0);
  o[2 * W + w] = any_exit ? ~(eg_h | ep_h) & top : 0;
  o[3 * W + w] = any_exit ? eg_h & top : 0;
  o[4 * W + w] = any_exit ? ~(eg_d | ep_d) & top : 0;
  o[5 * W + w] = any_exit ? eg_d & top : 0;
  o[6 * W + w] = any_exit ? mw : 0;
}

// Device memory of one summary run (stream-ordered pool; freed on scope exit).
struct SumMem {
  std::vector<void *> ptrs;
  ~SumMem() {
    for (void *p : ptrs) dev_free(p);
  }
  template <class T>
  T *up(const std::vector<T> &v) {
    void *p = dev_malloc(std::max<size_t>(v.size(), 1) * sizeof(T));
    if (!p) return nullptr;
    ptrs.push_back(p);
    if (!v.empty() && cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
      return nullptr;
    return static_cast<T *>(p);
  }
  template <class T>
  T *zeros(size_t n) {
    void *p = dev_malloc(std::max<size_t>(n, 1) * sizeof(T));
    if (!p) return nullptr;
    ptrs.push_back(p);
    return static_cast<T *>(p);
  }
};

}  // namespace

namespace ompdart {

// Summaries of n callees in one device run, in each callee's own numbering:
// rows[i] receives 7 * W_i words.  status[i] per callee.
int summarize_run(const ompdart_cfg *cfgs, int n, const ompdart_opts &o, uint64_t *const *rows, int32_t *status) {
  TraceScope trace("summaries", n);
  std::vector<Ingest> ing(n);
  std::vector<int32_t> st(n, OMPDART_OK);
  {  // host ingestion, one callee per task
    std::atomic<int> next{0};
    auto work = [&]() {
      for (int i = next++; i < n; i = next++) {
        std::string e;
        st[i] = ingest(&cfgs[i], &ing[i], &e);
      }
    };
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int T = (int)std::min<long long>({(long long)hw, 32ll, (long long)n / 8 + 1});
    std::vector<std::thread> pool;
    for (int t = 1; t < T; ++t) pool.emplace_back(work);
    work();
    for (auto &t : pool) t.join();
  }
  std::vector<int32_t> pos_off{0}, Wv, fin_off{0}, fin_pos, sout_off{0}, sout_pos, acc_off{0}, item_cfg, item_grp;
  std::vector<long long> scr_off, out_off, row_off, top_off;
  std::vector<uint32_t> acc;
  std::vector<uint64_t> calls, top;
  long long scr = 0, outw = 0;
  std::vector<int> idx;  // callee of each laid-out slot
  for (int i = 0; i < n; ++i) {
    if (st[i]) continue;
    const Ingest &g = ing[i];
    const ompdart_cfg &c = cfgs[i];
    const int k = (int)idx.size(), base = pos_off.back(), W = g.W;
    idx.push_back(i);
    Wv.push_back(W);
    scr_off.push_back(scr);
    out_off.push_back(outw);
    row_off.push_back((long long)calls.size());
    top_off.push_back((long long)top.size());
    scr += (long long)S_COUNT * g.M * W;
    outw += 7ll * W;
    if (c.call_planes && c.n_calls > 0) calls.insert(calls.end(), c.call_planes, c.call_planes + (size_t)c.n_calls * 7 * W);
    for (int w = 0; w < W; ++w) top.push_back((w == W - 1 && c.n_vars % 64) ? (1ull << (c.n_vars % 64)) - 1 : ~0ull);
    for (int q = 0; q < g.M; ++q) {
      const int b = g.order[q];
      for (int e = g.fin_off[q]; e < g.fin_off[q + 1]; ++e) fin_pos.push_back(base + g.pos[g.fin_src[e]]);
      fin_off.push_back((int32_t)fin_pos.size());
      for (int e = g.out_off[q]; e < g.out_off[q + 1]; ++e) sout_pos.push_back(base + g.pos[g.out_dst[e]]);
      sout_off.push_back((int32_t)sout_pos.size());
      acc.insert(acc.end(), c.acc + c.acc_off[b], c.acc + c.acc_off[b + 1]);
      acc_off.push_back((int32_t)acc.size());
    }
    pos_off.push_back(base + g.M);
    for (int grp = 0; grp * 32 < W; ++grp) {
      item_cfg.push_back(k);
      item_grp.push_back(grp);
    }
  }
  const int m = (int)idx.size();
  if (m) {
    SumMem mem;
    SumDev d{};
    d.n_items = (int)item_cfg.size();
    d.max_sweeps = o.max_sweeps > 0 ? o.max_sweeps : (1 << 20);
    bool ok = (d.item_cfg = mem.up(item_cfg)) && (d.item_grp = mem.up(item_grp)) && (d.pos_off = mem.up(pos_off)) &&
              (d.W = mem.up(Wv)) && (d.scr_off = mem.up(scr_off)) && (d.out_off = mem.up(out_off)) &&
              (d.row_off = mem.up(row_off)) && (d.top_off = mem.up(top_off)) && (d.fin_off = mem.up(fin_off)) &&
              (d.fin_pos = mem.up(fin_pos)) && (d.sout_off = mem.up(sout_off)) && (d.sout_pos = mem.up(sout_pos)) &&
              (d.acc_off = mem.up(acc_off)) && (d.acc = mem.up(acc)) && (d.calls = mem.up(calls)) &&
              (d.top = mem.up(top)) && (d.scr = mem.zeros<uint64_t>((size_t)scr)) &&
              (d.out = mem.zeros<uint64_t>((size_t)outw)) && (d.status = mem.zeros<int32_t>((size_t)m));
    if (!ok) return set_error(OMPDART_E_NOMEM, "device allocation for summaries failed");
    if (cudaStreamSynchronize(cudaStreamPerThread) != cudaSuccess)
      return set_error(OMPDART_E_CUDA, "device allocation for summaries failed");
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
      return set_error(OMPDART_E_CUDA, "stream creation failed");
    cudaMemsetAsync(d.status, 0, sizeof(int32_t) * m, s);
    const long long threads = (long long)d.n_items * 32;
    (void)cudaGetLastError();
    k_summarize<<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(d);
    std::vector<uint64_t> out((size_t)outw);
    std::vector<int32_t> dst(m);
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(out.data(), d.out, sizeof(uint64_t) * outw, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(dst.data(), d.status, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (ce != cudaSuccess) return set_error(OMPDART_E_CUDA, std::string("summary run: ") + cudaGetErrorString(ce));
    for (int k = 0; k < m; ++k) {
      const int i = idx[k];
      st[i] = dst[k];
      if (!st[i] && rows && rows[i]) memcpy(rows[i], out.data() + out_off[k], sizeof(uint64_t) * 7 * Wv[k]);
    }
  }
  if (status) std::copy(st.begin(), st.end(), status);
  return OMPDART_OK;
}

// A callee summary (callee numbering, 7 * Wc words) mapped into a caller's
// variable numbering (7 * Wr words): var_map[v] = caller variable or -1.
// Callee variables sharing one caller variable combine pessimistically:
// Req, Kill and MustDef by OR, Gen by AND.
void map_summary(const uint64_t *sum, int callee_vars, const int32_t *var_map, int caller_vars, uint64_t *row) {
  // Aliases (callee variables denoting one caller variable) combine into
  // the tightest row sound for every callee with these per-variable
  // summaries: Req, Kill, MustDef and Gen of any alias carry over, and a
  // kill of one alias overrides a gen of another (Sec. IV-C, applied
  // pessimistically at the call site).
  const int Wc = (callee_vars + 63) / 64, Wr = (caller_vars + 63) / 64;
  memset(row, 0, sizeof(uint64_t) * 7 * Wr);
  for (int v = 0; v < callee_vars; ++v) {
    const int t = var_map ? var_map[v] : v;
    if (t < 0 || t >= caller_vars) continue;
    const uint64_t mb = 1ull << (v & 63), tb = 1ull << (t & 63);
    for (int k = 0; k < 7; ++k)
      if (sum[(size_t)k * Wc + (v >> 6)] & mb) row[(size_t)k * Wr + (t >> 6)] |= tb;
  }
  for (int w = 0; w < Wr; ++w) {  // a kill overrides a gen of an alias
    row[2 * Wr + w] &= ~row[3 * Wr + w];
    row[4 * Wr + w] &= ~row[5 * Wr + w];
  }
}

}  // namespace ompdart

extern "C" {

int ompdart_summarize_batch(const ompdart_cfg *callees, int32_t n, const ompdart_opts *opts, uint64_t *const *rows,
                            int32_t *status) {
  set_last_error_text("");
  if (n < 0 || (n > 0 && (!callees || !rows))) return set_error(OMPDART_E_INVALID, "bad arguments");
  ompdart_opts o{};
  if (opts) o = *opts;
  if (cudaSetDevice(o.device) != cudaSuccess) return set_error(OMPDART_E_CUDA, "cudaSetDevice failed");
  StagedCfgs staged;  // callees given in device memory: copied for ingestion, a failure fails alone
  std::string serr;
  const int src = stage_cfgs(callees, n, &staged, &callees, &serr, true);
  if (src) return set_error(src, serr);
  const int rc = summarize_run(callees, n, o, rows, status);
  if (status)
    for (int i = 0; i < (int)staged.rc.size(); ++i)
      if (staged.rc[i]) status[i] = staged.rc[i];
  return rc;
}

int ompdart_summarize_callee(const ompdart_cfg *callee, const int32_t *var_map, int32_t caller_n_vars,
                             uint64_t *caller_row, const ompdart_opts *opts) {
  set_last_error_text("");
  if (!callee || !caller_row || caller_n_vars < 1) return set_error(OMPDART_E_INVALID, "bad arguments");
  StagedCfgs staged;
  std::string serr;
  const int src = stage_cfgs(callee, 1, &staged, &callee, &serr);
  if (src) return set_error(src, serr);
  std::vector<uint64_t> sum((size_t)7 * ((callee->n_vars + 63) / 64));
  uint64_t *rows[1] = {sum.data()};
  int32_t st = 0;
  int rc = ompdart_summarize_batch(callee, 1, opts, rows, &st);
  if (rc) return rc;
  if (st) return set_error(st, st == OMPDART_E_INVALID ? "invalid callee CFG" : "summary sweeps did not converge");
  map_summary(sum.data(), callee->n_vars, var_map, caller_n_vars, caller_row);
  return OMPDART_OK;
}

}  // extern "C"
