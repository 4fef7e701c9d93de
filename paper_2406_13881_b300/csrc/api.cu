// api.cu -- the C ABI of libompdart.so (see include/ompdart.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/ompdart.h"
#include "parallel.h"
#include "solver.h"

using namespace ompdart;

namespace {
thread_local std::string g_err;
}  // namespace

namespace ompdart {
void set_last_error_text(const std::string &msg) { g_err = msg; }
}  // namespace ompdart

namespace {

int set_err(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

int cuda_err(cudaError_t e, const char *what) {
  return set_err(OMPDART_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

// ==================================================================================
// the device plan core (one CFG, or a batch of CFGs of equal word count)
// ==================================================================================
namespace ompdart {

bool trace_on() {
  static const bool on = [] {
    const char *e = std::getenv("OMPDART_TRACE");
    return e && *e && *e != '0';
  }();
  return on;
}

void pool_setup() {
  static std::once_flag once;
  std::call_once(once, [] {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) return;
    for (int d = 0; d < n; ++d) {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, d) != cudaSuccess) continue;
      uint64_t keep = ~0ull;  // this process's pool keeps freed memory for reuse
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
  });
}

PlanCore::~PlanCore() {
  if (scan) scan_destroy(scan);
  for (void *p : allocs) dev_free(p);
}

long long estimate_device_bytes(const ompdart_cfg &c, int keep_states) {
  const long long N = c.n_blocks, W = (c.n_vars + 63) / 64;
  const long long E = c.succ_off ? c.succ_off[N] : 0, A = c.acc_off ? c.acc_off[N] : 0;
  // state planes (h_in, d_in, h_out, live), the walks' pairs (two per
  // phase and liveness's header plane), kept states (d_out and its pair);
  // loop header rows for at most one loop per 8 blocks
  const long long planes = (9 + (keep_states ? 3 : 0)) * N * W * 8 + 4 * (N / 8 + 1) * W * 8;
  const long long meta = N * (64 + 6 * 4) + E * (2 * 8 + 5 * 4) + A * (4 * 3 + 1);
  const long long chunks = (N / 16 + 1) * W * 8 * 6;  // chunk maps and carries
  const long long xfer = (N / 4 + 64) * 2 * 24 + (N / 8 + 8) * W * 8 * 4;
  return planes + meta + chunks + xfer + (1 << 16);
}

void boundary_rows(const ompdart_cfg *cfg, int W, std::vector<uint64_t> *top, std::vector<uint64_t> *eh,
                   std::vector<uint64_t> *ed, std::vector<uint64_t> *xl) {
  for (int w = 0; w < W; ++w) {
    const uint64_t t = (w == W - 1 && cfg->n_vars % 64) ? (1ull << (cfg->n_vars % 64)) - 1 : ~0ull;
    top->push_back(t);
    eh->push_back((cfg->entry_host_valid ? cfg->entry_host_valid[w] : ~0ull) & t);
    ed->push_back((cfg->entry_dev_valid ? cfg->entry_dev_valid[w] : 0ull) & t);
    xl->push_back((cfg->exit_host_live ? cfg->exit_host_live[w] : ~0ull) & t);
  }
}

// Device arrays of the data-region mode (Ingest::region_mode): the
// classification inputs, the boundary rows the emission fills and every
// output of the directives (see classify.cu).
int region_build(PlanCore *P, const int32_t *acc_off, int n_cfg, const std::vector<uint64_t> &fp, std::string *err) {
  const Ingest &g = P->g;
  DevPlan &d = P->dp;
  const int W = g.W, N = g.N, A = g.A, nk = g.kern_off.back();
  P->region = true;
  std::vector<int32_t> blk_cfg(N), kern(N, -1), acc_blk(A), acc_base(n_cfg);
  std::vector<uint8_t> has_r(n_cfg, 0);
  for (int c = 0; c < n_cfg; ++c) {
    acc_base[c] = acc_off[g.cfg_blk_off[c]];
    for (int b = g.cfg_blk_off[c]; b < g.cfg_blk_off[c + 1]; ++b) {
      blk_cfg[b] = c;
      if (g.kernel[b] >= 0) kern[b] = g.kern_off[c] + g.kernel[b];
      has_r[c] |= g.in_region[b];
    }
  }
  parallel_ranges(N, 1 << 16, 8, [&](int, int lo, int hi) {
    for (int b = lo; b < hi; ++b)
      for (int i = acc_off[b]; i < acc_off[b + 1]; ++i) acc_blk[i] = b;
  });
  // boundary rows: entry edges, then exit edges; the in-edge (fin index) of each
  const int n_rin = (int)g.rin_eid.size(), n_rout = (int)g.rout_eid.size();
  std::vector<int32_t> fin_bnd(std::max(1, P->n_fin), -1);
  for (int c = 0; c < n_cfg; ++c) {
    std::vector<std::pair<int32_t, int32_t>> rows;  // (local edge id, row)
    for (int r = g.rin_off[c]; r < g.rin_off[c + 1]; ++r) rows.push_back({g.rin_eid[r], r});
    for (int r = g.rout_off[c]; r < g.rout_off[c + 1]; ++r) rows.push_back({g.rout_eid[r], n_rin + r});
    if (rows.empty()) continue;
    for (int i = g.cfg_pos_off[c]; i < g.cfg_pos_off[c + 1]; ++i)
      for (int k = g.fin_off[i]; k < g.fin_off[i + 1]; ++k)
        for (const auto &x : rows)
          if (x.first == g.fin_eid[k]) fin_bnd[k] = x.second;
  }
  std::vector<int32_t> xin, xin_off(n_cfg + 1, 0), start_k(n_cfg, -1);
  for (size_t x = 0; x < g.exit_blocks.size(); ++x) {
    const int b = g.exit_blocks[x];
    if (g.in_region[b]) {
      xin.push_back((int32_t)x);
      xin_off[blk_cfg[b] + 1]++;
    }
  }
  for (int c = 0; c < n_cfg; ++c) {
    xin_off[c + 1] += xin_off[c];
    if (g.start_kernel[c] >= 0) start_k[c] = g.kern_off[c] + g.start_kernel[c];
  }
  std::vector<uint64_t> fp_rows = fp;
  fp_rows.resize((size_t)nk * W, 0);
  bool ok = true;
  auto chk = [&](const void *q) { ok = ok && q != nullptr; };
  ClsDev &c = P->cls;
  c.A = A; c.W = W; c.n_cfg = n_cfg; c.n_k = nk; c.n_rin = n_rin;
  c.acc = d.acc; c.acc_off = d.acc_off; c.pos = d.pos; c.acc_flag = d.acc_flag; c.from_exit = d.from_exit;
  chk(c.acc_blk = P->upload(acc_blk));
  chk(c.kern = P->upload(kern));
  chk(c.blk_cfg = P->upload(blk_cfg));
  chk(c.acc_base = P->upload(acc_base));
  chk(c.kw_h = P->dalloc<uint64_t>((size_t)nk * W));
  chk(c.kw_d = P->dalloc<uint64_t>((size_t)nk * W));
  chk(c.kernel_to = P->dalloc<uint64_t>((size_t)nk * W));
  chk(c.kernel_from = P->dalloc<uint64_t>((size_t)nk * W));
  chk(c.dev_touched = P->dalloc<uint64_t>((size_t)n_cfg * W));
  chk(c.acc_point = P->dalloc<int32_t>(A));
  chk(c.rin_off = P->upload(g.rin_off));
  chk(c.rout_off = P->upload(g.rout_off));
  chk(c.xin_off = P->upload(xin_off));
  chk(c.xin = P->upload(xin));
  chk(c.has_r = P->upload(has_r));
  chk(c.entry_in_r = P->upload(g.entry_in_region));
  chk(c.start_k = P->upload(start_k));
  uint64_t *bt = P->dalloc<uint64_t>((size_t)(n_rin + n_rout) * W), *bf = P->dalloc<uint64_t>((size_t)(n_rin + n_rout) * W);
  chk(bt);
  chk(bf);
  c.bnd_to = d.bnd_to = bt;
  c.bnd_from = d.bnd_from = bf;
  chk(c.map_to = P->dalloc<uint64_t>((size_t)n_cfg * W));
  chk(c.map_from = P->dalloc<uint64_t>((size_t)n_cfg * W));
  chk(c.map_alloc = P->dalloc<uint64_t>((size_t)n_cfg * W));
  chk(d.fin_bnd = P->upload(fin_bnd));
  chk(d.ent_rx = P->upload(g.ent_rx));
  chk(d.ent_dst = P->upload(g.ent_dst));
  chk(P->d_in_region = P->upload(g.in_region));
  chk(P->d_rin = P->upload(g.rin_eid));
  chk(P->d_rout = P->upload(g.rout_eid));
  chk(P->d_fp = P->upload(fp_rows));
  if (!ok) {
    *err = "device allocation failed";
    return OMPDART_E_NOMEM;
  }
  P->h_kern_off = g.kern_off;
  P->h_rin_off = g.rin_off;
  P->h_rout_off = g.rout_off;
  P->h_acc_base = acc_base;
  return OMPDART_OK;
}

int core_build(PlanCore *P, const int32_t *acc_off, const uint32_t *acc, const CallHost &calls,
               const std::vector<uint64_t> &top, const std::vector<uint64_t> &eh, const std::vector<uint64_t> &ed,
               const std::vector<uint64_t> &xl, int n_cfg, const std::vector<int32_t> &unreach_cfg,
               const ompdart_opts &o, std::string *err, const std::vector<uint64_t> &fp) {
  TraceScope trace("core_build", P->g.M);
  const Ingest &g = P->g;
  P->keep_states = o.keep_states;
  const int W = g.W;
  std::vector<int32_t> fin_dst(g.fin_src.size());
  parallel_ranges(g.M, 1 << 16, 8, [&](int, int lo, int hi) {
    for (int i = lo; i < hi; ++i)
      for (int k = g.fin_off[i]; k < g.fin_off[i + 1]; ++k) fin_dst[k] = g.order[i];
  });
  P->n_fin = (int)g.fin_src.size();

  DevPlan &d = P->dp;
  d.N = g.N; d.M = g.M; d.E = g.E; d.A = g.A; d.W = W; d.V = g.V; d.L = g.L; d.K = g.K;
  d.X = (int)g.exit_blocks.size();
  d.entry = g.entry;
  d.n_cfg = n_cfg;
  d.max_sweeps = o.max_sweeps > 0 ? o.max_sweeps : (1 << 20);
  const size_t NW = (size_t)g.N * W;
  bool ok = true;
  auto chk = [&](const void *p) { ok = ok && p != nullptr; };
  chk(d.order = P->upload(g.order));
  chk(d.pos = P->upload(g.pos));
  chk(d.fin_off = P->upload(g.fin_off));
  chk(d.fin_src = P->upload(g.fin_src));
  chk(d.fin_eid = P->upload(g.fin_eid));
  chk(d.fin_ent = P->upload(g.fin_ent));
  chk(d.fin_dst = P->upload(fin_dst));
  chk(d.out_off = P->upload(g.out_off));
  chk(d.out_dst = P->upload(g.out_dst));
  chk(d.is_exit = P->upload(g.is_exit));
  chk(d.exit_blocks = P->upload(g.exit_blocks));
  {
    std::vector<int32_t> un;
    for (int b = 0; b < g.N; ++b)
      if (g.pos[b] < 0) un.push_back(b);
    d.n_unreach = (int)un.size();
    chk(d.unreach = P->upload(un));
    d.unreach_cfg = nullptr;
    if (!unreach_cfg.empty()) chk(d.unreach_cfg = P->upload(unreach_cfg));
  }
  chk(d.acc_off = P->upload(acc_off, (size_t)g.N + 1));
  chk(d.acc = P->upload(acc, (size_t)g.A));
  chk(d.rec = P->dalloc<uint32_t>(g.A));
  chk(d.loop_head = P->upload(g.loop_head));
  chk(d.body_off = P->upload(g.body_off));
  chk(d.body_blk = P->upload(g.body_blk));
  chk(d.ent_loop = P->upload(g.ent_loop));
  chk(d.ent_src = P->upload(g.ent_src));
  chk(d.entry_h = P->upload(eh));
  chk(d.entry_d = P->upload(ed));
  chk(d.exit_live = P->upload(xl));
  chk(d.top = P->upload(top));
  chk(d.h_in = P->dalloc<uint64_t>(NW));
  chk(d.d_in = P->dalloc<uint64_t>(NW));
  // host validity at block exits: the scan solver's emission reads it
  chk(d.h_out = P->dalloc<uint64_t>(NW));
  if (o.keep_states) chk(d.d_out = P->dalloc<uint64_t>(NW));
  chk(d.live = P->dalloc<uint64_t>(NW));
  chk(d.mask_h = P->dalloc<uint64_t>((size_t)g.L * W));
  chk(d.mask_d = P->dalloc<uint64_t>((size_t)g.L * W));
  chk(d.ec_h = P->dalloc<uint64_t>((size_t)g.K * W));
  chk(d.ec_d = P->dalloc<uint64_t>((size_t)g.K * W));
  chk(d.acc_flag = P->dalloc<uint8_t>(g.A));
  chk(d.from_exit = P->dalloc<uint64_t>((size_t)d.X * W));
  chk(d.status = P->dalloc<int32_t>(ST_COUNT));
  if (!ok) {
    *err = "device allocation failed";
    return OMPDART_E_NOMEM;
  }
  // ---- the data region and the directives
  if (g.region_mode) {
    const int rc = region_build(P, acc_off, n_cfg, fp, err);
    if (rc) return rc;
  }
  // ---- call sites (Sec. IV-C): every call access; the reachable blocks holding them
  {
    std::vector<int32_t> site_acc, cblk, cblk_site0, cblk_rowbase, cblk_cfg;
    // without a call table no access is a call (the format check rejects one)
    for (int b = 0; b < g.N && calls.planes; ++b) {
      int first = -1;
      for (int i = acc_off[b]; i < acc_off[b + 1]; ++i)
        if (acc[i] >> 31) {
          if (first < 0) first = (int)site_acc.size();
          site_acc.push_back(i);
        }
      if (first < 0 || g.pos[b] < 0) continue;
      const int cfg = (int)(std::upper_bound(g.cfg_pos_off.begin(), g.cfg_pos_off.end(), g.pos[b]) -
                            g.cfg_pos_off.begin()) - 1;
      cblk.push_back(b);
      cblk_site0.push_back(first);
      cblk_rowbase.push_back(calls.row_base.empty() ? 0 : calls.row_base[cfg]);
      cblk_cfg.push_back(cfg);
    }
    d.n_sites = (int)site_acc.size();
    d.n_cblk = (int)cblk.size();
    if (d.n_sites) {
      if (!scan_supported(g) || o.path == 1 || o.eager_to) {
        *err = "CFGs with call pseudo-accesses need the chunked scan solver (a reducible CFG whose loop bodies "
               "are contiguous in loop order, lazy `to' placement)";
        return OMPDART_E_INVALID;
      }
      const size_t SW = (size_t)d.n_sites * W;
      chk(d.calls = P->upload(calls.planes, (size_t)calls.rows * 7 * W));
      chk(d.site_acc = P->upload(site_acc));
      chk(d.cblk = P->upload(cblk));
      chk(d.cblk_site0 = P->upload(cblk_site0));
      chk(d.cblk_rowbase = P->upload(cblk_rowbase));
      chk(d.cblk_cfg = P->upload(cblk_cfg));
      chk(d.call_to = P->dalloc<uint64_t>(SW));
      chk(d.call_from = P->dalloc<uint64_t>(SW));
      chk(d.call_entry_h = P->dalloc<uint64_t>(SW));
      chk(d.call_entry_d = P->dalloc<uint64_t>(SW));
      chk(d.call_exit_live = P->dalloc<uint64_t>(SW));
      if (!ok) {
        *err = "device allocation failed";
        return OMPDART_E_NOMEM;
      }
    }
    P->site_acc = std::move(site_acc);
  }
  int want = o.path;
  if (want == 0) want = scan_supported(g) ? 2 : 1;
  if (want == 2 && o.eager_to && g.K < (int)g.fin_src.size()) {
    *err = "eager `to' placement on the scan solver needs the CFG ingested with every edge's constant entry";
    return OMPDART_E_INVALID;
  }
  if (want == 2 && !scan_supported(g)) {
    *err = "the chunked scan solver needs a reducible CFG whose loop bodies are contiguous in loop order";
    return OMPDART_E_INVALID;
  }
  if (n_cfg > 1 && want != 2) {
    *err = "a batch plan needs the scan solver";
    return OMPDART_E_INVALID;
  }
  P->path = want;
  if (want == 1) {
    if (!o.keep_states) chk(d.d_out = P->dalloc<uint64_t>(NW));  // the sweep solver reads the exit states
    chk(d.hp_out = P->dalloc<uint64_t>(NW));
    chk(d.ant_h = P->dalloc<uint64_t>(NW));
    chk(d.ant_d = P->dalloc<uint64_t>(NW));
    if (o.eager_to) chk(d.ant_dm = P->dalloc<uint64_t>(NW));
    chk(d.lant = P->dalloc<uint64_t>(g.body_blk.size() * (size_t)W * 2));
  } else {
    chk(P->cfg_err = P->dalloc<int32_t>(n_cfg));
    if (o.eager_to) {  // AntDm and the edge constants' targets (eager `to' placement)
      chk(d.ant_dm = P->dalloc<uint64_t>(NW));
      if (!d.ent_dst) chk(d.ent_dst = P->upload(g.ent_dst));
    }
    if (!ok) {
      *err = "device allocation failed";
      return OMPDART_E_NOMEM;
    }
    P->scan = scan_create(g, acc_off, acc, calls, P->cfg_err, d, o.chunk_target, o.keep_states, err,
                          o.warps_per_cta);
    if (!P->scan) return OMPDART_E_NOMEM;
  }
  // transfer records: start with room for a few per loop-entry edge and
  // join; grown after a run that overflowed
  const size_t cap0 = std::min<size_t>((size_t)P->n_fin * W + 1, std::max<size_t>(4096, ((size_t)g.K + g.M / 8) * 2));
  chk(d.xfer = P->dalloc<EdgeXfer>(cap0));
  d.xfer_cap = (int)cap0;
  if (!ok) {
    *err = "device allocation failed";
    return OMPDART_E_NOMEM;
  }
  // the pool allocations are ordered on this thread's default stream: let
  // them complete before any other stream uses them
  if (cudaStreamSynchronize(cudaStreamPerThread) != cudaSuccess) {
    *err = "device allocation failed";
    return OMPDART_E_NOMEM;
  }
  if (P->scan) P->dev_bytes += scan_device_bytes(P->scan);
  return OMPDART_OK;
}

int core_enqueue(PlanCore *P, cudaStream_t s, Prof *pf) {
  cudaMemsetAsync(P->dp.status, 0, ST_COUNT * sizeof(int32_t), s);
  if (P->cfg_err) cudaMemsetAsync(P->cfg_err, 0, sizeof(int32_t) * P->dp.n_cfg, s);
  int n = 0;
  if (P->path == 1)
    n += enqueue_local_summary(P->dp, s, pf) + enqueue_sweep_solver(P->dp, s, P->n_fin, pf);
  else
    n += enqueue_scan_solver(P->scan, P->dp, s, pf) + enqueue_call_sites(P->dp, s, pf);
  n += enqueue_fill_unreachable(P->dp, s, P->keep_states, pf);
  if (P->region) n += enqueue_classify(P->cls, s, pf);
  return n;
}

int core_finish(PlanCore *P, cudaStream_t s, int32_t *h_status, bool *rerun) {
  cudaError_t ce;
  if (P->path == 2 && h_status[ST_OVERFLOW]) {
    // a per-warp record stream overflowed: size the streams and redo the
    // host-validity pass (it is the one that emits)
    if (!scan_grow_streams(P->scan)) return set_err(OMPDART_E_NOMEM, "growing transfer record streams failed");
    *rerun = true;
    cudaMemsetAsync(P->dp.status + ST_NREC, 0, 2 * sizeof(int32_t), s);
    enqueue_scan_edges(P->scan, P->dp, s, nullptr);
    ce = cudaMemcpyAsync(h_status, P->dp.status, ST_COUNT * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_err(ce, "device run");
  }
  const int nrec = h_status[ST_NREC];
  if (nrec > P->dp.xfer_cap) {
    // the record buffer overflowed: enlarge it and redo the edge emission
    const int need = nrec + nrec / 4 + 16;
    EdgeXfer *x = P->dalloc<EdgeXfer>((size_t)need);
    if (!x || cudaStreamSynchronize(cudaStreamPerThread) != cudaSuccess)
      return set_err(OMPDART_E_NOMEM, "device allocation of transfer records failed");
    P->dp.xfer = x;
    P->dp.xfer_cap = need;
    *rerun = true;
    cudaMemsetAsync(P->dp.status + ST_NREC, 0, sizeof(int32_t), s);
    if (P->path == 1)
      enqueue_sweep_edges(P->dp, s, P->n_fin);
    else
      enqueue_scan_edges(P->scan, P->dp, s, nullptr);
    ce = cudaMemcpyAsync(h_status, P->dp.status, ST_COUNT * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_err(ce, "device run");
  }
  return OMPDART_OK;
}

void core_view(const PlanCore &P, const int32_t *h_status, ompdart_result *v) {
  const Ingest &g = P.g;
  memset(v, 0, sizeof *v);
  v->n_blocks = g.N; v->n_vars = g.V; v->n_words = g.W; v->n_edges = g.E; v->n_acc = g.A;
  v->n_exits = P.dp.X;
  v->mem = OMPDART_MEM_DEVICE;
  v->h_in = P.dp.h_in; v->d_in = P.dp.d_in;
  v->h_out = P.keep_states ? P.dp.h_out : nullptr;
  v->d_out = P.keep_states ? P.dp.d_out : nullptr;
  v->acc_flag = P.dp.acc_flag;
  v->n_edge_xfers = std::min(h_status[ST_NREC], P.dp.xfer_cap);
  v->edge_xfers = reinterpret_cast<ompdart_edge_xfer *>(P.dp.xfer);
  v->exit_blocks = const_cast<int32_t *>(P.dp.exit_blocks);
  v->from_exit = P.dp.from_exit;
  v->path = P.path;
  v->sweeps = h_status[ST_SWEEPS];
  v->h2d_bytes = P.h2d + scan_h2d_bytes(P.scan);
  v->d2h_bytes = 0;
  v->live_in = P.keep_states ? P.dp.live : nullptr;
  v->n_call_sites = P.dp.n_sites;
  v->call_site_acc = const_cast<int32_t *>(P.dp.site_acc);
  v->call_to = P.dp.call_to;
  v->call_from = P.dp.call_from;
  v->call_entry_h = P.dp.call_entry_h;
  v->call_entry_d = P.dp.call_entry_d;
  v->call_exit_live = P.dp.call_exit_live;
  if (P.region) {  // CFG 0 of the plan (a batch arena's views offset these per CFG)
    v->in_region = P.d_in_region;
    v->map_to = P.cls.map_to;
    v->map_from = P.cls.map_from;
    v->map_alloc = P.cls.map_alloc;
    v->n_kernels = P.h_kern_off.size() > 1 ? P.h_kern_off[1] - P.h_kern_off[0] : 0;
    v->kernel_to = P.cls.kernel_to;
    v->kernel_from = P.cls.kernel_from;
    v->firstprivate = P.d_fp;
    v->acc_point = P.cls.acc_point;
    v->n_region_entries = P.h_rin_off.size() > 1 ? P.h_rin_off[1] : 0;
    v->n_region_exits = P.h_rout_off.size() > 1 ? P.h_rout_off[1] : 0;
    v->region_entry_edges = P.d_rin;
    v->region_exit_edges = P.d_rout;
  }
}

int result_copy(const ompdart_result &v, bool pin, cudaStream_t s, ompdart_result **out, HostStage *stage) {
  *out = nullptr;
  const size_t NW = (size_t)v.n_blocks * v.n_words, SW = (size_t)v.n_call_sites * v.n_words;
  // one host block: every array at a 64-byte aligned offset
  struct Part {
    void **dst;
    const void *src;
    size_t bytes;
  };
  ompdart_result r = v;
  r.mem = OMPDART_MEM_HOST;
  r.host_block = nullptr;
  Part parts[] = {
      {(void **)&r.h_in, v.h_in, NW * 8},
      {(void **)&r.d_in, v.d_in, NW * 8},
      {(void **)&r.h_out, v.h_out, v.h_out ? NW * 8 : 0},
      {(void **)&r.d_out, v.d_out, v.d_out ? NW * 8 : 0},
      {(void **)&r.live_in, v.live_in, v.live_in ? NW * 8 : 0},
      {(void **)&r.acc_flag, v.acc_flag, (size_t)v.n_acc},
      {(void **)&r.edge_xfers, v.edge_xfers, sizeof(ompdart_edge_xfer) * (size_t)v.n_edge_xfers},
      {(void **)&r.exit_blocks, v.exit_blocks, sizeof(int32_t) * (size_t)v.n_exits},
      {(void **)&r.from_exit, v.from_exit, 8 * (size_t)v.n_exits * v.n_words},
      {(void **)&r.call_site_acc, v.call_site_acc, sizeof(int32_t) * (size_t)v.n_call_sites},
      {(void **)&r.call_to, v.call_to, 8 * SW},
      {(void **)&r.call_from, v.call_from, 8 * SW},
      {(void **)&r.call_entry_h, v.call_entry_h, 8 * SW},
      {(void **)&r.call_entry_d, v.call_entry_d, 8 * SW},
      {(void **)&r.call_exit_live, v.call_exit_live, 8 * SW},
      {(void **)&r.in_region, v.in_region, v.in_region ? (size_t)v.n_blocks : 0},
      {(void **)&r.map_to, v.map_to, v.map_to ? 8 * (size_t)v.n_words : 0},
      {(void **)&r.map_from, v.map_from, v.map_from ? 8 * (size_t)v.n_words : 0},
      {(void **)&r.map_alloc, v.map_alloc, v.map_alloc ? 8 * (size_t)v.n_words : 0},
      {(void **)&r.kernel_to, v.kernel_to, v.kernel_to ? 8 * (size_t)v.n_kernels * v.n_words : 0},
      {(void **)&r.kernel_from, v.kernel_from, v.kernel_from ? 8 * (size_t)v.n_kernels * v.n_words : 0},
      {(void **)&r.firstprivate, v.firstprivate, v.firstprivate ? 8 * (size_t)v.n_kernels * v.n_words : 0},
      {(void **)&r.acc_point, v.acc_point, v.acc_point ? 4 * (size_t)v.n_acc : 0},
      {(void **)&r.region_entry_edges, v.region_entry_edges, v.region_entry_edges ? 4 * (size_t)v.n_region_entries : 0},
      {(void **)&r.region_exit_edges, v.region_exit_edges, v.region_exit_edges ? 4 * (size_t)v.n_region_exits : 0},
  };
  size_t total = 0;
  for (const Part &p : parts) total += (p.bytes + 63) & ~size_t(63);
  // a small result goes through the caller's page-locked staging buffer:
  // every copy asynchronous, one wait, then one host copy into the block
  // (copies into pageable memory each wait on their own)
  char *stage_base = stage ? (char *)stage->get(total + 64) : nullptr;
  HostBlock *blk = host_block_new(total + 64, stage_base ? false : pin);
  if (!blk) return set_err(OMPDART_E_NOMEM, "host allocation failed");
  char *base = (char *)host_block_ptr(blk);
  char *land = stage_base ? stage_base : base;
  size_t off = 0;
  cudaError_t ce = cudaSuccess;
  for (const Part &p : parts) {
    // optional arrays stay NULL when absent; the others point into the
    // block even when empty
    const bool optional = p.dst == (void **)&r.h_out || p.dst == (void **)&r.d_out || p.dst == (void **)&r.live_in ||
                          p.dst == (void **)&r.in_region || p.dst == (void **)&r.map_to ||
                          p.dst == (void **)&r.map_from || p.dst == (void **)&r.map_alloc ||
                          p.dst == (void **)&r.kernel_to || p.dst == (void **)&r.kernel_from ||
                          p.dst == (void **)&r.firstprivate || p.dst == (void **)&r.acc_point ||
                          p.dst == (void **)&r.region_entry_edges || p.dst == (void **)&r.region_exit_edges;
    if (optional && !p.src) {
      *p.dst = nullptr;
      continue;
    }
    *p.dst = base + off;
    if (p.bytes && p.src && ce == cudaSuccess)
      ce = cudaMemcpyAsync(land + off, p.src, p.bytes, cudaMemcpyDeviceToHost, s);
    off += (p.bytes + 63) & ~size_t(63);
  }
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce == cudaSuccess && stage_base) memcpy(base, stage_base, off);
  if (ce != cudaSuccess) {
    host_block_release(blk);
    return cuda_err(ce, "copy of results");
  }
  r.d2h_bytes = (long long)(2 + (v.h_out ? 2 : 0) + (v.live_in ? 1 : 0)) * NW * 8 + v.n_acc +
                (long long)sizeof(ompdart_edge_xfer) * v.n_edge_xfers + 4ll * v.n_exits + 8ll * v.n_exits * v.n_words +
                4ll * ST_COUNT + 4ll * v.n_call_sites + 40ll * SW;
  ompdart_result *res = result_in_block(r, blk);
  host_block_release(blk);  // the result holds its own reference
  if (!res) return set_err(OMPDART_E_NOMEM, "host allocation failed");
  *out = res;
  return OMPDART_OK;
}

ompdart_result *result_in_block(const ompdart_result &v, HostBlock *block) {
  ompdart_result *r = (ompdart_result *)malloc(sizeof(ompdart_result));
  if (!r) return nullptr;
  *r = v;
  r->mem = OMPDART_MEM_HOST;
  r->host_block = block;
  host_block_ref(block);
  return r;
}

int set_error(int code, const std::string &msg) { return set_err(code, msg); }

}  // namespace ompdart

// ==================================================================================
// single-CFG plan
// ==================================================================================
struct ompdart_plan {
  PlanCore core;
  cudaStream_t stream = nullptr;
  cudaStream_t last_stream = nullptr;
  int device = 0;
  int launches = 0;
  int32_t *h_status = nullptr;  // pinned
  Prof prof;
  // graph replay: the first run after enabling is captured into a CUDA
  // graph and later runs launch it whole; a run that changes the plan's
  // buffers (record streams grown after an overflow) drops it
  bool graph_on = false;
  cudaGraphExec_t gexec = nullptr;
  HostStage stage;  // small results and boundary rows pass through it
  void drop_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
  }
  ~ompdart_plan() {
    // the plan's memory goes back to the pool: its last run must be done
    if (last_stream) cudaStreamSynchronize(last_stream);
    if (stream) cudaStreamSynchronize(stream);
    drop_graph();
    if (stream) cudaStreamDestroy(stream);
    if (h_status) cudaFreeHost(h_status);
  }
};

namespace ompdart {

int plan_set_boundary(ompdart_plan *P, const ompdart_cfg *cfg, cudaStream_t s) {
  std::vector<uint64_t> top, eh, ed, xl;
  boundary_rows(cfg, P->core.g.W, &top, &eh, &ed, &xl);
  const DevPlan &d = P->core.dp;
  const size_t bytes = sizeof(uint64_t) * eh.size();
  // through the plan's page-locked staging buffer: the copies do not wait.
  // The buffer is free again here: the plan's previous run (and the copy
  // of its results) completed before this run may start.
  uint64_t *h = (uint64_t *)P->stage.get(3 * bytes);
  const uint64_t *src[3] = {eh.data(), ed.data(), xl.data()};
  if (h)
    for (int k = 0; k < 3; ++k) memcpy(h + k * eh.size(), src[k], bytes);
  uint64_t *dst[3] = {const_cast<uint64_t *>(d.entry_h), const_cast<uint64_t *>(d.entry_d),
                      const_cast<uint64_t *>(d.exit_live)};
  cudaError_t ce = cudaSuccess;
  for (int k = 0; k < 3 && ce == cudaSuccess; ++k)
    ce = cudaMemcpyAsync(dst[k], h ? h + k * eh.size() : src[k], bytes, cudaMemcpyHostToDevice, s);
  // (a copy from pageable memory has read its source when it returns)
  return ce == cudaSuccess ? OMPDART_OK : cuda_err(ce, "uploading entry and exit rows");
}

long long plan_device_bytes(const ompdart_plan *P) { return P ? P->core.dev_bytes : 0; }

}  // namespace ompdart

extern "C" {

const char *ompdart_last_error(void) { return g_err.c_str(); }

int ompdart_plan_create(const ompdart_cfg *cfg, const ompdart_opts *opts, ompdart_plan **out) {
  g_err.clear();
  if (!out) return set_err(OMPDART_E_INVALID, "plan output pointer is NULL");
  *out = nullptr;
  ompdart_opts o{};
  if (opts) o = *opts;
  StagedCfgs staged;  // device-resident inputs copied for ingestion
  if (cfg) {
    std::string serr;
    const int src = stage_cfgs(cfg, 1, &staged, &cfg, &serr);
    if (src) return set_err(src, serr);
  }
  ompdart_plan *P = new (std::nothrow) ompdart_plan();
  if (!P) return set_err(OMPDART_E_NOMEM, "host allocation failed");
  std::string err;
  TraceScope trace("ingest", cfg ? cfg->n_blocks : 0);
  // eager placement puts constants on any edge: every edge gets an entry
  // unless the sweep solver is asked for (it needs none)
  int rc = ingest(cfg, &P->core.g, &err, o.data_region != 0, o.eager_to != 0 && o.path != 1);
  trace.next("plan rows");
  if (rc) {
    delete P;
    return set_err(rc, err);
  }
  // firstprivate scalars (Sec. IV-D): their kernel reads analysed as host reads
  ompdart_cfg fpc = *cfg;
  std::vector<uint64_t> fp;
  int n_kernels = 0;
  if (o.data_region && (rc = firstprivate_view(*cfg, &staged, &fpc, &fp, &n_kernels, &err))) {
    delete P;
    return set_err(rc, err);
  }
  P->device = o.device;
  cudaError_t ce = cudaSetDevice(o.device);
  if (ce != cudaSuccess) {
    delete P;
    return cuda_err(ce, "cudaSetDevice");
  }
  if ((ce = cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking)) != cudaSuccess) {
    delete P;
    return cuda_err(ce, "cudaStreamCreate");
  }
  if ((ce = cudaMallocHost(&P->h_status, ST_COUNT * sizeof(int32_t))) != cudaSuccess) {
    delete P;
    return cuda_err(ce, "cudaMallocHost");
  }
  std::vector<uint64_t> top, eh, ed, xl;
  boundary_rows(cfg, P->core.g.W, &top, &eh, &ed, &xl);
  CallHost calls;
  calls.planes = cfg->call_planes;
  calls.rows = cfg->call_planes ? cfg->n_calls : 0;
  rc = core_build(&P->core, cfg->acc_off, fpc.acc, calls, top, eh, ed, xl, 1, {}, o, &err, fp);
  if (rc) {
    delete P;
    return set_err(rc, err);
  }
  *out = P;
  return OMPDART_OK;
}

int ompdart_plan_run(ompdart_plan *P, void *stream) {
  g_err.clear();
  if (!P) return set_err(OMPDART_E_INVALID, "plan is NULL");
  cudaStream_t s = stream ? (cudaStream_t)stream : P->stream;
  P->last_stream = s;
  (void)cudaGetLastError();  // clear a stale "not ready" of an earlier query
  Prof *pf = P->prof.on ? &P->prof : nullptr;
  if (P->graph_on && !pf) {
    if (!P->gexec) {
      cudaGraph_t g = nullptr;
      cudaError_t ce = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
      if (ce != cudaSuccess) return cuda_err(ce, "graph capture");
      P->launches = core_enqueue(&P->core, s, nullptr);
      ce = cudaStreamEndCapture(s, &g);
      if (ce == cudaSuccess) ce = cudaGraphInstantiate(&P->gexec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (ce != cudaSuccess) {
        P->gexec = nullptr;
        return cuda_err(ce, "graph capture");
      }
    }
    const cudaError_t ce = cudaGraphLaunch(P->gexec, s);
    if (ce != cudaSuccess) return cuda_err(ce, "graph launch");
    return OMPDART_OK;
  }
  if (pf) pf->collect_pending = true;
  P->launches = core_enqueue(&P->core, s, pf);
  if (pf) pf->close(s);
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) return cuda_err(ce, "kernel launch");
  return OMPDART_OK;
}

int ompdart_plan_graph(ompdart_plan *P, int enable) {
  if (!P) return set_err(OMPDART_E_INVALID, "plan is NULL");
  P->graph_on = enable != 0;
  if (!P->graph_on) {
    if (P->last_stream) cudaStreamSynchronize(P->last_stream);
    P->drop_graph();
  }
  return OMPDART_OK;
}

int ompdart_plan_sync(ompdart_plan *P) {
  if (!P) return set_err(OMPDART_E_INVALID, "plan is NULL");
  cudaStream_t s = P->last_stream ? P->last_stream : P->stream;
  cudaError_t ce = cudaMemcpyAsync(P->h_status, P->core.dp.status, ST_COUNT * sizeof(int32_t),
                                   cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return cuda_err(ce, "device run");
  if (P->prof.on && P->prof.collect_pending) {
    P->prof.collect();
    P->prof.collect_pending = false;
  }
  if (P->h_status[ST_ERROR] == ERR_NOCONVERGE)
    return set_err(OMPDART_E_NOCONVERGE, "a device fixed-point loop reached max_sweeps");
  bool rerun = false;
  int rc = core_finish(&P->core, s, P->h_status, &rerun);
  if (rerun) P->drop_graph();  // its launches hold the old buffers
  if (rc) return rc;
  if (P->h_status[ST_ERROR] == ERR_NOCONVERGE)
    return set_err(OMPDART_E_NOCONVERGE, "a device fixed-point loop reached max_sweeps");
  return OMPDART_OK;
}

int ompdart_plan_view(ompdart_plan *P, ompdart_result *v) {
  if (!P || !v) return set_err(OMPDART_E_INVALID, "NULL argument");
  core_view(P->core, P->h_status, v);
  return OMPDART_OK;
}

int ompdart_plan_launches(const ompdart_plan *P) { return P ? P->launches : 0; }

int ompdart_plan_profile(ompdart_plan *P, int enable) {
  if (!P) return set_err(OMPDART_E_INVALID, "plan is NULL");
  P->prof.on = enable != 0;
  for (double &x : P->prof.ms) x = 0.0;
  for (int &x : P->prof.cnt) x = 0;
  P->prof.used = 0;
  return OMPDART_OK;
}

int ompdart_plan_timings(ompdart_plan *P, ompdart_timing *out, int32_t max, int32_t *n) {
  if (!P || !n) return set_err(OMPDART_E_INVALID, "NULL argument");
  const int k = (int)P->prof.names.size();
  *n = k;
  for (int i = 0; i < k && i < max && out; ++i) {
    out[i].name = P->prof.names[i].c_str();
    out[i].launches = P->prof.cnt[i];
    out[i].ms = P->prof.ms[i];
  }
  return OMPDART_OK;
}

void ompdart_plan_destroy(ompdart_plan *P) { delete P; }

void ompdart_result_free(ompdart_result *r) {
  if (!r) return;
  host_block_release(static_cast<HostBlock *>(r->host_block));
  free(r);
}

int ompdart_plan_fetch(ompdart_plan *P, ompdart_result **out) {
  if (!P || !out) return set_err(OMPDART_E_INVALID, "NULL argument");
  *out = nullptr;
  ompdart_result v;
  core_view(P->core, P->h_status, &v);
  // one large block: page-locked; a small one through the plan's staging buffer
  return result_copy(v, true, P->last_stream ? P->last_stream : P->stream, out, &P->stage);
}

int ompdart_analyze(const ompdart_cfg *cfg, const ompdart_opts *opts, ompdart_result **out) {
  if (!out) return set_err(OMPDART_E_INVALID, "result output pointer is NULL");
  *out = nullptr;
  ompdart_plan *P = nullptr;
  TraceScope trace("plan create", cfg ? cfg->n_blocks : 0);
  int rc = ompdart_plan_create(cfg, opts, &P);
  if (rc) return rc;
  trace.next("plan run+sync");
  rc = ompdart_plan_run(P, nullptr);
  if (!rc) rc = ompdart_plan_sync(P);
  trace.next("plan fetch");
  if (!rc) rc = ompdart_plan_fetch(P, out);
  trace.next("plan destroy");
  ompdart_plan_destroy(P);
  return rc;
}

}  // extern "C"
