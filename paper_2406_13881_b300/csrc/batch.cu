// batch.cu -- many independent CFGs per device run (ompdart_batch_*).
//
// Host side of the batched analysis:
//   * ingestion of every CFG on a pool of host threads (one CFG per task);
//   * grouping into arenas by word count W: an arena is one plan of the
//     chunked scan solver over its CFGs laid end to end (concat_ingests),
//     with per-CFG entry/exit rows and valid-variable masks; CFGs that
//     solver cannot take get a plan of their own (sweep solver);
//   * the autotuner: per arena, (chunk_target, warps_per_cta) timed on a
//     sample of the arena's CFGs, cached per (W, size class);
//   * one CUDA graph per batch: every plan's kernel sequence captured on
//     its own forked stream, so independent arenas overlap on the GPU;
//   * per-CFG status and per-CFG result views into the arenas.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <tuple>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ompdart.h"
#include "solver.h"

using namespace ompdart;

namespace {

struct Arena {
  PlanCore core;
  int W = 0, chunk_target = 0, wpc = 0;
  std::vector<int32_t> members;                              // batch index of each CFG, arena order
  std::vector<int32_t> blk_off, acc_base, x_off, chunk_beg;  // [members + 1]
  std::vector<int32_t> n_vars, n_edges;                      // [members]
  std::vector<int32_t> site_off;                             // [members + 1] call sites of each CFG
  int32_t *site_local = nullptr;  // device [sites]: access index within its CFG
  int32_t *exit_local = nullptr;  // device [X]: exit blocks as ids local to their CFG
  int32_t *h_status = nullptr;    // host [ST_COUNT]
  int32_t *h_err = nullptr;       // host [members]
  std::vector<int32_t> rec_off;   // [members + 1] gathered record range per CFG
  int rec_run = -1;               // run whose records rec_off describes
};

struct Solo {  // a CFG on a plan of its own
  PlanCore core;
  int32_t member = -1;
  int32_t *h_status = nullptr;  // host [ST_COUNT]
};

struct Where {
  int kind = 0;  // 0 not placed (ingestion failed), 1 arena, 2 solo
  int index = 0, member = 0;
};

// ---- autotuner cache: (W, floor(log2(arena positions))) -> (chunk_target, wpc)
std::mutex g_tune_mu;
std::map<std::pair<int, int>, std::pair<int, int>> g_tune_cache;

int ilog2(long long x) {
  int r = 0;
  while (x > 1) {
    x >>= 1;
    ++r;
  }
  return r;
}

}  // namespace

struct ompdart_batch {
  int n = 0;
  ompdart_opts opts{};
  std::vector<int32_t> ingest_status, run_status;
  std::vector<Where> where;
  std::vector<std::unique_ptr<Arena>> arenas;
  std::vector<std::unique_ptr<Solo>> solos;
  std::vector<std::unique_ptr<int32_t[]>> host;
  cudaStream_t stream = nullptr, last_stream = nullptr;
  std::vector<cudaStream_t> side;  // one per plan, at most kSide
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool graph_ok = false;
  int launches = 0;
  int runs = 0;
  bool ran = false;
  Prof prof;  // per-kernel events (ompdart_batch_profile): plans run one after another on the caller's stream

  // host status words (pageable: a batch is created and destroyed often by
  // the serving loop, and freeing pinned memory can wait for the device)
  int32_t *host_ints(size_t n) {
    host.emplace_back(new (std::nothrow) int32_t[std::max<size_t>(n, 1)]());
    return host.back().get();
  }
  void drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    graph_ok = false;
  }
  ~ompdart_batch() {
    // the arenas' memory goes back to the pool: every run must be done
    if (last_stream) cudaStreamSynchronize(last_stream);
    for (cudaStream_t s : side) cudaStreamSynchronize(s);
    if (stream) cudaStreamSynchronize(stream);
    drop_graph();
    arenas.clear();
    solos.clear();
    for (cudaStream_t s : side) cudaStreamDestroy(s);
    for (cudaEvent_t e : join) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
    if (stream) cudaStreamDestroy(stream);
  }
};

namespace {

constexpr int kSide = 8;  // forked streams a run spreads its plans over

// Lay the CFGs `members` (ingested in ing) out as one arena and upload it.
int build_arena(Arena *a, const std::vector<int32_t> &members, const std::vector<const Ingest *> &ing,
                const ompdart_cfg *cfgs, const ompdart_opts &o, std::string *err,
                const std::vector<std::vector<uint64_t>> &fps) {
  a->members = members;
  std::vector<const Ingest *> parts;
  parts.reserve(members.size());
  for (int m : members) parts.push_back(ing[m]);
  TraceScope trace_cat("arena concat", (long long)members.size());
  concat_ingests(parts, &a->core.g);
  const int W = a->core.g.W;
  a->W = W;
  std::vector<int32_t> acc_off{0}, unreach_cfg, exit_local, site_local;
  std::vector<uint32_t> acc;
  std::vector<uint64_t> top, eh, ed, xl, table;
  CallHost calls;
  std::map<std::tuple<const void *, const void *, const void *, const void *, const void *, int, int, int, int>, int>
      same;
  a->site_off.assign(1, 0);
  acc_off.reserve(a->core.g.N + 1);
  acc.reserve(a->core.g.A);
  a->blk_off.assign(1, 0);
  a->acc_base.assign(1, 0);
  a->x_off.assign(1, 0);
  for (size_t k = 0; k < members.size(); ++k) {
    const ompdart_cfg &c = cfgs[members[k]];
    const Ingest &g = *ing[members[k]];
    const int32_t base = (int32_t)acc.size();
    for (int b = 0; b < g.N; ++b) acc_off.push_back(base + c.acc_off[b + 1]);
    acc.insert(acc.end(), c.acc, c.acc + c.acc_off[g.N]);
    boundary_rows(&c, W, &top, &eh, &ed, &xl);
    for (int b = 0; b < g.N; ++b)
      if (g.pos[b] < 0) unreach_cfg.push_back((int32_t)k);
    exit_local.insert(exit_local.end(), g.exit_blocks.begin(), g.exit_blocks.end());
    // a CFG given with the same arrays and call table as an earlier member
    // (one function in several contexts) shares its table rows and folds
    const auto key = std::make_tuple((const void *)c.succ_off, (const void *)c.succ, (const void *)c.acc_off,
                                     (const void *)c.acc, (const void *)c.call_planes, c.n_blocks, c.n_vars,
                                     c.entry, c.n_calls);
    const int first = same.emplace(key, (int)k).first->second;
    calls.same_as.push_back(first);
    if (first != (int)k) {
      calls.row_base.push_back(calls.row_base[first]);
    } else {
      calls.row_base.push_back(calls.rows);
      if (c.call_planes && c.n_calls > 0) {
        table.insert(table.end(), c.call_planes, c.call_planes + (size_t)c.n_calls * 7 * W);
        calls.rows += c.n_calls;
      }
    }
    if (c.call_planes)  // call accesses come with a call table (checked at ingestion)
      for (int i = 0; i < c.acc_off[g.N]; ++i)
        if (c.acc[i] >> 31) site_local.push_back(i);
    a->site_off.push_back((int32_t)site_local.size());
    a->n_vars.push_back(c.n_vars);
    a->n_edges.push_back(g.E);
    a->blk_off.push_back(a->blk_off.back() + g.N);
    a->acc_base.push_back((int32_t)acc.size());
    a->x_off.push_back(a->x_off.back() + (int32_t)g.exit_blocks.size());
  }
  trace_cat.next("arena core", (long long)members.size());
  ompdart_opts oa = o;
  oa.path = 2;
  oa.chunk_target = a->chunk_target;
  oa.warps_per_cta = a->wpc;
  calls.planes = table.empty() ? nullptr : table.data();
  std::vector<uint64_t> fp;  // firstprivate rows of the members' kernels, in kernel order
  if (!fps.empty())
    for (int m : members) fp.insert(fp.end(), fps[m].begin(), fps[m].end());
  int rc = core_build(&a->core, acc_off.data(), acc.data(), calls, top, eh, ed, xl, (int)members.size(),
                      unreach_cfg, oa, err, fp);
  if (rc) return rc;
  const std::vector<int32_t> &co = a->core.g.chunk_off, &cp = a->core.g.cfg_pos_off;
  a->chunk_beg.resize(members.size() + 1);
  for (size_t k = 0; k < members.size(); ++k)
    a->chunk_beg[k] = (int32_t)(std::lower_bound(co.begin(), co.end(), cp[k]) - co.begin());
  a->chunk_beg[members.size()] = (int32_t)co.size() - 1;
  a->exit_local = a->core.upload(exit_local);
  a->site_local = a->core.upload(site_local);
  if (!a->exit_local || !a->site_local) {
    *err = "device allocation failed";
    return OMPDART_E_NOMEM;
  }
  return OMPDART_OK;
}

// Mean device time of `reps` runs of a core (after one warm-up run), ms;
// a huge value if a run failed.
double time_core(PlanCore *c, cudaStream_t s, int reps) {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  core_enqueue(c, s, nullptr);
  cudaEventRecord(a, s);
  for (int r = 0; r < reps; ++r) core_enqueue(c, s, nullptr);
  cudaEventRecord(b, s);
  float ms = 1e30f;
  int32_t st[ST_COUNT] = {};
  bool ok = cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess &&
            cudaMemcpy(st, c->dp.status, sizeof st, cudaMemcpyDeviceToHost) == cudaSuccess && st[ST_ERROR] == 0;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ok ? ms / reps : 1e30;
}

// Pick (chunk_target, wpc) for an arena of `members`: coordinate search
// over chunk targets (16..512) at 4 warps per CTA, then 2 warps per CTA at the
// best target, each candidate a trial arena over a sample of about 2^18
// positions (every step-th CFG), timed on the device.
void tune_arena(Arena *a, const std::vector<int32_t> &members, const std::vector<const Ingest *> &ing,
                const ompdart_cfg *cfgs, const ompdart_opts &o, cudaStream_t s,
                const std::vector<std::vector<uint64_t>> &fps) {
  long long total = 0;
  for (int m : members) total += ing[m]->M;
  const std::pair<int, int> key(ing[members[0]]->W, ilog2(std::max<long long>(1, total)));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      a->chunk_target = it->second.first;
      a->wpc = it->second.second;
      return;
    }
  }
  const long long kSample = 1 << 18;
  const long long step = std::max<long long>(1, (total + kSample - 1) / kSample);
  std::vector<int32_t> sample;
  for (size_t k = 0; k < members.size(); k += (size_t)step) sample.push_back(members[k]);
  auto trial = [&](int chunk, int wpc) {
    Arena t;
    t.chunk_target = chunk;
    t.wpc = wpc;
    std::string err;
    if (build_arena(&t, sample, ing, cfgs, o, &err, fps)) return 1e30;
    return time_core(&t.core, s, 3);
  };
  int best_chunk = 128, best_wpc = 4;
  double best = 1e30;
  for (int chunk : {16, 32, 64, 128, 256, 512}) {
    const double t = trial(chunk, 4);
    if (t < best) {
      best = t;
      best_chunk = chunk;
    }
  }
  for (int wpc : {2}) {
    const double t = trial(best_chunk, wpc);
    if (t < best) {
      best = t;
      best_wpc = wpc;
    }
  }
  a->chunk_target = best_chunk;
  a->wpc = best_wpc;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = {best_chunk, best_wpc};
}

// Enqueue one run of every plan: fork from s onto the side streams, join back.
int enqueue_all(ompdart_batch *B, cudaStream_t s) {
  int n = 0, k = 0;
  cudaEventRecord(B->fork, s);
  for (cudaStream_t x : B->side) cudaStreamWaitEvent(x, B->fork, 0);
  auto next = [&]() { return B->side[(k++) % B->side.size()]; };
  for (auto &a : B->arenas) n += core_enqueue(&a->core, next(), nullptr);
  for (auto &p : B->solos) n += core_enqueue(&p->core, next(), nullptr);
  for (size_t i = 0; i < B->side.size(); ++i) {
    cudaEventRecord(B->join[i], B->side[i]);
    cudaStreamWaitEvent(s, B->join[i], 0);
  }
  return n;
}

// Gathered record range of every CFG of an arena after the last run.
int arena_records(ompdart_batch *B, Arena *a) {
  if (a->rec_run == B->runs) return OMPDART_OK;
  std::vector<int32_t> offs;
  const int32_t total = std::min(a->h_status[ST_NREC], a->core.dp.xfer_cap);
  if (!scan_chunk_record_offsets(a->core.scan, B->last_stream, &offs, total))
    return set_error(OMPDART_E_CUDA, "copy of record offsets failed");
  a->rec_off.resize(a->members.size() + 1);
  for (size_t k = 0; k <= a->members.size(); ++k) a->rec_off[k] = std::min(offs[a->chunk_beg[k]], total);
  a->rec_run = B->runs;
  return OMPDART_OK;
}

void arena_view(const Arena &a, int k, ompdart_result *v) {
  const Ingest &g = a.core.g;
  const int W = g.W;
  const DevPlan &d = a.core.dp;
  const size_t b0 = (size_t)a.blk_off[k] * W;
  memset(v, 0, sizeof *v);
  v->n_blocks = a.blk_off[k + 1] - a.blk_off[k];
  v->n_vars = a.n_vars[k];
  v->n_edges = a.n_edges[k];
  v->n_words = W;
  v->n_acc = a.acc_base[k + 1] - a.acc_base[k];
  v->n_exits = a.x_off[k + 1] - a.x_off[k];
  v->mem = OMPDART_MEM_DEVICE;
  v->h_in = d.h_in + b0;
  v->d_in = d.d_in + b0;
  v->h_out = a.core.keep_states ? d.h_out + b0 : nullptr;
  v->d_out = a.core.keep_states ? d.d_out + b0 : nullptr;
  v->live_in = a.core.keep_states ? d.live + b0 : nullptr;
  v->acc_flag = d.acc_flag + a.acc_base[k];
  v->n_edge_xfers = a.rec_off[k + 1] - a.rec_off[k];
  v->edge_xfers = reinterpret_cast<ompdart_edge_xfer *>(d.xfer) + a.rec_off[k];
  v->exit_blocks = a.exit_local + a.x_off[k];
  v->from_exit = d.from_exit + (size_t)a.x_off[k] * W;
  v->path = a.core.path;
  v->sweeps = a.h_status[ST_SWEEPS];
  const int s0 = a.site_off[k];
  v->n_call_sites = a.site_off[k + 1] - s0;
  v->call_site_acc = a.site_local + s0;
  if (v->n_call_sites) {
    const size_t o = (size_t)s0 * W;
    v->call_to = d.call_to + o;
    v->call_from = d.call_from + o;
    v->call_entry_h = d.call_entry_h + o;
    v->call_entry_d = d.call_entry_d + o;
    v->call_exit_live = d.call_exit_live + o;
  }
  v->h2d_bytes = a.core.h2d + scan_h2d_bytes(a.core.scan);
  v->d2h_bytes = 0;
  const PlanCore &c = a.core;
  if (c.region) {  // this member's slice of the arena's data-region outputs
    const size_t kb = (size_t)c.h_kern_off[k] * W;
    v->in_region = c.d_in_region + a.blk_off[k];
    v->map_to = c.cls.map_to + (size_t)k * W;
    v->map_from = c.cls.map_from + (size_t)k * W;
    v->map_alloc = c.cls.map_alloc + (size_t)k * W;
    v->n_kernels = c.h_kern_off[k + 1] - c.h_kern_off[k];
    v->kernel_to = c.cls.kernel_to + kb;
    v->kernel_from = c.cls.kernel_from + kb;
    v->firstprivate = c.d_fp + kb;
    v->acc_point = c.cls.acc_point + a.acc_base[k];
    v->n_region_entries = c.h_rin_off[k + 1] - c.h_rin_off[k];
    v->n_region_exits = c.h_rout_off[k + 1] - c.h_rout_off[k];
    v->region_entry_edges = c.d_rin + c.h_rin_off[k];
    v->region_exit_edges = c.d_rout + c.h_rout_off[k];
  }
}

}  // namespace

extern "C" {

int ompdart_batch_create(const ompdart_cfg *cfgs, int32_t n, const ompdart_opts *opts, ompdart_batch **out,
                         int32_t *status) {
  set_last_error_text("");
  if (!out) return set_error(OMPDART_E_INVALID, "batch output pointer is NULL");
  *out = nullptr;
  if (n < 0 || (n > 0 && !cfgs)) return set_error(OMPDART_E_INVALID, "bad CFG array");
  StagedCfgs staged;  // device-resident inputs copied for ingestion; a CFG that fails fails alone
  {
    std::string serr;
    const int src = stage_cfgs(cfgs, n, &staged, &cfgs, &serr, true);
    if (src) return set_error(src, serr);
  }
  ompdart_batch *B = new (std::nothrow) ompdart_batch();
  if (!B) return set_error(OMPDART_E_NOMEM, "host allocation failed");
  std::unique_ptr<ompdart_batch> hold(B);
  if (opts) B->opts = *opts;
  const ompdart_opts &o = B->opts;
  B->n = n;
  cudaError_t ce = cudaSetDevice(o.device);
  if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
  if (ce != cudaSuccess) return set_error(OMPDART_E_CUDA, std::string("CUDA setup: ") + cudaGetErrorString(ce));
  // ---- ingestion, one CFG per task.  CFGs given with the same graph and
  // access arrays (the same function analysed in several contexts: only
  // the boundary rows differ) are ingested once and share the result.
  TraceScope trace_ingest("batch ingest", n);
  std::vector<int32_t> canon(n);
  {
    std::map<std::tuple<const void *, const void *, const void *, const void *, const void *, const void *, int, int,
                        int>,
             int32_t>
        first;
    for (int i = 0; i < n; ++i) {
      const ompdart_cfg &c = cfgs[i];
      canon[i] = first.emplace(std::make_tuple((const void *)c.succ_off, (const void *)c.succ, (const void *)c.acc_off,
                                               (const void *)c.acc, (const void *)c.region,
                                               (const void *)c.scalar_vars, c.n_blocks, c.n_vars, c.entry),
                               i)
                     .first->second;
    }
  }
  std::vector<Ingest> ing(n);
  std::vector<const Ingest *> ingp(n);
  for (int i = 0; i < n; ++i) ingp[i] = &ing[canon[i]];
  B->ingest_status.assign(n, OMPDART_OK);
  B->where.assign(n, Where{});
  {
    std::atomic<int> next{0};
    auto work = [&]() {
      for (int i = next++; i < n; i = next++) {
        if (canon[i] != i) continue;
        std::string e;
        int rc = ingest(&cfgs[i], &ing[i], &e, o.data_region != 0, o.eager_to != 0);
        B->ingest_status[i] = rc;
      }
    };
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int T = (int)std::min<long long>({(long long)hw, 32ll, (long long)n / 16 + 1});
    std::vector<std::thread> pool;
    for (int t = 1; t < T; ++t) pool.emplace_back(work);
    work();
    for (auto &t : pool) t.join();
    for (int i = 0; i < n; ++i) B->ingest_status[i] = B->ingest_status[canon[i]];
    for (int i = 0; i < (int)staged.rc.size(); ++i)
      if (staged.rc[i]) B->ingest_status[i] = staged.rc[i];
  }
  // ---- firstprivate scalars (data-region mode): each ingested CFG's kernel
  // reads of read-only scalars analysed as host reads (a copy of the
  // access array; CFGs sharing arrays share the copy)
  std::vector<ompdart_cfg> fcfgs;
  std::vector<std::vector<uint64_t>> fps;
  StagedCfgs fp_bufs;
  if (o.data_region) {
    fcfgs.assign(cfgs, cfgs + n);
    fps.resize(n);
    for (int i = 0; i < n; ++i) {
      if (B->ingest_status[i]) continue;
      if (canon[i] != i) {
        fcfgs[i].acc = fcfgs[canon[i]].acc;
        fps[i] = fps[canon[i]];
        continue;
      }
      int nk = 0;
      std::string e;
      const int rc = firstprivate_view(cfgs[i], &fp_bufs, &fcfgs[i], &fps[i], &nk, &e);
      if (rc) B->ingest_status[i] = rc;
    }
    for (int i = 0; i < n; ++i)
      if (canon[i] != i && B->ingest_status[canon[i]]) B->ingest_status[i] = B->ingest_status[canon[i]];
    cfgs = fcfgs.data();
  }
  trace_ingest.next("batch arenas", n);
  // ---- grouping
  std::map<int, std::vector<int32_t>> by_w;
  std::vector<int32_t> solo_ids;
  for (int i = 0; i < n; ++i) {
    if (B->ingest_status[i]) continue;
    // (eager placement takes no calls: such a CFG fails alone on a plan of its own)
    const bool calls_eager = o.eager_to && cfgs[i].call_planes && cfgs[i].n_calls > 0;
    if (scan_supported(*ingp[i]) && !calls_eager)
      by_w[ingp[i]->W].push_back(i);
    else
      solo_ids.push_back(i);
  }
  std::string err;
  // arenas: tuned one after another (trials are timed on the device), then
  // laid out and uploaded in parallel, one host thread per arena
  std::vector<std::pair<int, std::vector<int32_t>>> groups(by_w.begin(), by_w.end());
  const int n_ar = (int)groups.size();
  std::vector<std::unique_ptr<Arena>> built(n_ar);
  for (int g = 0; g < n_ar; ++g) {
    built[g].reset(new (std::nothrow) Arena());
    if (!built[g]) return set_error(OMPDART_E_NOMEM, "host allocation failed");
    built[g]->chunk_target = o.chunk_target;
    built[g]->wpc = o.warps_per_cta;
    if (o.tune) tune_arena(built[g].get(), groups[g].second, ingp, cfgs, o, B->stream, fps);
  }
  {
    std::vector<int> rcs(n_ar, OMPDART_OK);
    std::vector<std::string> errs(n_ar);
    std::atomic<int> next{0};
    auto work = [&](bool main_thread) {
      if (!main_thread && cudaSetDevice(o.device) != cudaSuccess) {
        for (int g = next++; g < n_ar; g = next++) {
          rcs[g] = OMPDART_E_CUDA;
          errs[g] = "CUDA setup in a build thread failed";
        }
        return;
      }
      for (int g = next++; g < n_ar; g = next++)
        rcs[g] = build_arena(built[g].get(), groups[g].second, ingp, cfgs, o, &errs[g], fps);
    };
    // small batches (a serving turn) are built on the calling thread: a
    // thread of its own costs more than such an arena's build
    long long positions = 0;
    for (const auto &gr : groups)
      for (int m : gr.second) positions += ingp[m]->M;
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int T = positions < (1 << 18) ? 1 : std::min(n_ar, (int)std::min(hw, 16u));
    std::vector<std::thread> pool;
    for (int t = 1; t < T; ++t) pool.emplace_back(work, false);
    work(true);
    for (auto &t : pool) t.join();
    for (int g = 0; g < n_ar; ++g)
      if (rcs[g]) return set_error(rcs[g], errs[g]);
  }
  for (int g = 0; g < n_ar; ++g) {
    std::unique_ptr<Arena> a = std::move(built[g]);
    a->h_status = B->host_ints(ST_COUNT);
    a->h_err = B->host_ints(a->members.size());
    if (!a->h_status || !a->h_err) return set_error(OMPDART_E_NOMEM, "host allocation failed");
    const int idx = (int)B->arenas.size();
    for (size_t k = 0; k < a->members.size(); ++k) B->where[a->members[k]] = Where{1, idx, (int)k};
    B->arenas.push_back(std::move(a));
  }
  for (int i : solo_ids) {
    std::unique_ptr<Solo> p(new (std::nothrow) Solo());
    if (!p) return set_error(OMPDART_E_NOMEM, "host allocation failed");
    p->member = i;
    p->core.g = *ingp[i];  // a copy: CFGs with the same arrays share one ingestion
    std::vector<uint64_t> top, eh, ed, xl;
    boundary_rows(&cfgs[i], p->core.g.W, &top, &eh, &ed, &xl);
    ompdart_opts os = o;
    os.path = 1;
    CallHost calls;
    calls.planes = cfgs[i].call_planes;
    calls.rows = cfgs[i].call_planes ? cfgs[i].n_calls : 0;
    int rc = core_build(&p->core, cfgs[i].acc_off, cfgs[i].acc, calls, top, eh, ed, xl, 1, {}, os, &err,
                        fps.empty() ? std::vector<uint64_t>() : fps[i]);
    if (rc == OMPDART_E_INVALID) {  // this CFG alone (calls without the scan solver)
      B->ingest_status[i] = rc;
      B->where[i] = Where{};
      continue;
    }
    if (rc) return set_error(rc, err);
    p->h_status = B->host_ints(ST_COUNT);
    if (!p->h_status) return set_error(OMPDART_E_NOMEM, "host allocation failed");
    B->where[i] = Where{2, (int)B->solos.size(), 0};
    B->solos.push_back(std::move(p));
  }
  const int plans = (int)(B->arenas.size() + B->solos.size());
  const int ns = std::max(1, std::min(kSide, plans));
  for (int i = 0; i < ns; ++i) {
    cudaStream_t x = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return set_error(OMPDART_E_CUDA, "stream creation failed");
    B->side.push_back(x);
    B->join.push_back(e);
  }
  B->run_status = B->ingest_status;
  if (status) std::copy(B->ingest_status.begin(), B->ingest_status.end(), status);
  *out = hold.release();
  return OMPDART_OK;
}

int ompdart_batch_run(ompdart_batch *B, void *stream) {
  set_last_error_text("");
  if (!B) return set_error(OMPDART_E_INVALID, "batch is NULL");
  cudaStream_t s = stream ? (cudaStream_t)stream : B->stream;
  B->last_stream = s;
  // start from a clean per-thread error state: a query that answered "not
  // ready" (a poll of an earlier run) leaves that code behind
  (void)cudaGetLastError();
  cudaError_t ce;
  if (B->arenas.empty() && B->solos.empty()) {  // nothing to run (empty batch, or every CFG rejected)
    B->launches = 0;
  } else if (B->prof.on) {
    B->prof.collect_pending = true;
    int n = 0;
    for (auto &a : B->arenas) n += core_enqueue(&a->core, s, &B->prof);
    for (auto &p : B->solos) n += core_enqueue(&p->core, s, &B->prof);
    B->prof.close(s);
    B->launches = n;
  } else if (B->opts.no_graph) {
    B->launches = enqueue_all(B, s);
  } else {
    if (!B->graph_ok) {
      B->drop_graph();
      ce = cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal);
      if (ce != cudaSuccess) return set_error(OMPDART_E_CUDA, std::string("begin capture: ") + cudaGetErrorString(ce));
      B->launches = enqueue_all(B, B->stream);
      ce = cudaStreamEndCapture(B->stream, &B->graph);
      if (ce == cudaSuccess) ce = cudaGraphInstantiate(&B->exec, B->graph, 0);
      if (ce != cudaSuccess) {
        B->drop_graph();
        return set_error(OMPDART_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
      }
      B->graph_ok = true;
    }
    ce = cudaGraphLaunch(B->exec, s);
    if (ce != cudaSuccess) return set_error(OMPDART_E_CUDA, std::string("graph launch: ") + cudaGetErrorString(ce));
  }
  ce = cudaGetLastError();
  if (ce != cudaSuccess) return set_error(OMPDART_E_CUDA, std::string("kernel launch: ") + cudaGetErrorString(ce));
  ++B->runs;
  B->ran = true;
  return OMPDART_OK;
}

int ompdart_batch_sync(ompdart_batch *B, int32_t *status) {
  if (!B) return set_error(OMPDART_E_INVALID, "batch is NULL");
  if (!B->ran) return set_error(OMPDART_E_INVALID, "the batch has not run");
  cudaStream_t s = B->last_stream;
  cudaError_t ce = cudaSuccess;
  for (auto &a : B->arenas) {
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(a->h_status, a->core.dp.status, ST_COUNT * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(a->h_err, a->core.cfg_err, a->members.size() * sizeof(int32_t), cudaMemcpyDeviceToHost,
                           s);
  }
  for (auto &p : B->solos)
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(p->h_status, p->core.dp.status, ST_COUNT * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return set_error(OMPDART_E_CUDA, std::string("device run: ") + cudaGetErrorString(ce));
  if (B->prof.on && B->prof.collect_pending) {
    B->prof.collect();
    B->prof.collect_pending = false;
  }
  B->run_status = B->ingest_status;
  for (auto &a : B->arenas) {
    bool rerun = false;
    int rc = core_finish(&a->core, s, a->h_status, &rerun);
    if (rc) return rc;
    if (rerun) B->graph_ok = false;
    for (size_t k = 0; k < a->members.size(); ++k)
      if (a->h_err[k]) B->run_status[a->members[k]] = OMPDART_E_NOCONVERGE;
  }
  for (auto &p : B->solos) {
    if (p->h_status[ST_ERROR]) {
      B->run_status[p->member] = OMPDART_E_NOCONVERGE;
      continue;
    }
    bool rerun = false;
    int rc = core_finish(&p->core, s, p->h_status, &rerun);
    if (rc) return rc;
    if (rerun) B->graph_ok = false;
  }
  if (status) std::copy(B->run_status.begin(), B->run_status.end(), status);
  return OMPDART_OK;
}

int ompdart_batch_profile(ompdart_batch *B, int enable) {
  if (!B) return set_error(OMPDART_E_INVALID, "batch is NULL");
  B->prof.on = enable != 0;
  for (double &x : B->prof.ms) x = 0.0;
  for (int &x : B->prof.cnt) x = 0;
  B->prof.used = 0;
  return OMPDART_OK;
}

int ompdart_batch_timings(ompdart_batch *B, ompdart_timing *out, int32_t max, int32_t *n) {
  if (!B || !n) return set_error(OMPDART_E_INVALID, "NULL argument");
  const int k = (int)B->prof.names.size();
  *n = k;
  for (int i = 0; i < k && i < max && out; ++i) {
    out[i].name = B->prof.names[i].c_str();
    out[i].launches = B->prof.cnt[i];
    out[i].ms = B->prof.ms[i];
  }
  return OMPDART_OK;
}

int ompdart_batch_view(ompdart_batch *B, int32_t i, ompdart_result *v) {
  if (!B || !v) return set_error(OMPDART_E_INVALID, "NULL argument");
  if (i < 0 || i >= B->n) return set_error(OMPDART_E_INVALID, "CFG index out of range");
  if (!B->ran) return set_error(OMPDART_E_INVALID, "the batch has not run");
  if (B->run_status[i]) return set_error(B->run_status[i], "this CFG has no result (see its status)");
  const Where &w = B->where[i];
  if (w.kind == 2) {
    Solo &p = *B->solos[w.index];
    core_view(p.core, p.h_status, v);
    return OMPDART_OK;
  }
  Arena &a = *B->arenas[w.index];
  int rc = arena_records(B, &a);
  if (rc) return rc;
  arena_view(a, w.member, v);
  return OMPDART_OK;
}

int ompdart_batch_fetch(ompdart_batch *B, int32_t i, ompdart_result **out) {
  if (!out) return set_error(OMPDART_E_INVALID, "NULL argument");
  *out = nullptr;
  ompdart_result v;
  int rc = ompdart_batch_view(B, i, &v);
  if (rc) return rc;
  return result_copy(v, false, B->last_stream, out);
}

int ompdart_batch_info(const ompdart_batch *B, int32_t *n_arenas, int32_t *n_solo, int32_t *launches, int32_t max,
                       int32_t *arena_w, int32_t *arena_cfgs, int32_t *arena_chunk, int32_t *arena_wpc) {
  if (!B) return set_error(OMPDART_E_INVALID, "batch is NULL");
  if (n_arenas) *n_arenas = (int32_t)B->arenas.size();
  if (n_solo) *n_solo = (int32_t)B->solos.size();
  if (launches) *launches = B->launches;
  for (int k = 0; k < (int)B->arenas.size() && k < max; ++k) {
    const Arena &a = *B->arenas[k];
    if (arena_w) arena_w[k] = a.W;
    if (arena_cfgs) arena_cfgs[k] = (int32_t)a.members.size();
    if (arena_chunk) arena_chunk[k] = a.chunk_target;
    if (arena_wpc) arena_wpc[k] = a.wpc;
  }
  return OMPDART_OK;
}

void ompdart_batch_destroy(ompdart_batch *B) { delete B; }

int ompdart_analyze_batch(const ompdart_cfg *cfgs, int32_t n, const ompdart_opts *opts, ompdart_result **outs,
                          int32_t *status) {
  if (n > 0 && !outs) return set_error(OMPDART_E_INVALID, "result array is NULL");
  for (int i = 0; i < n; ++i) outs[i] = nullptr;
  ompdart_batch *B = nullptr;
  int rc = ompdart_batch_create(cfgs, n, opts, &B, status);
  if (rc) return rc;
  std::unique_ptr<ompdart_batch> hold(B);
  TraceScope trace("batch run+sync", n);
  rc = ompdart_batch_run(B, nullptr);
  if (!rc) rc = ompdart_batch_sync(B, status);
  if (rc) return rc;
  trace.next("batch fetch", n);
  rc = batch_fetch_all(B, outs);
  trace.next("batch destroy", n);
  return rc;
}

}  // extern "C"

namespace ompdart {

cudaStream_t batch_stream(const ompdart_batch *B) { return B->stream; }

long long batch_device_bytes(const ompdart_batch *B) {
  long long b = 0;
  for (auto &a : B->arenas) b += a->core.dev_bytes;
  for (auto &p : B->solos) b += p->core.dev_bytes;
  return b;
}

int batch_fetch_all(ompdart_batch *B, ompdart_result **outs) {
  int rc = OMPDART_OK;
  for (int i = 0; i < B->n; ++i) outs[i] = nullptr;
  // one bulk copy per arena into one host block; each CFG's result is a
  // view into it (the block lives until the last of them is freed)
  for (auto &ap : B->arenas) {
    Arena &a = *ap;
    rc = arena_records(B, &a);
    if (rc) return rc;
    ompdart_result whole;
    core_view(a.core, a.h_status, &whole);
    if (whole.n_call_sites != a.site_off.back())
      return set_error(OMPDART_E_INVALID, "internal: arena call sites out of step");
    whole.exit_blocks = a.exit_local;
    whole.call_site_acc = a.site_local;  // access index within each CFG
    ompdart_result *host = nullptr;
    rc = result_copy(whole, false, B->last_stream, &host);
    if (rc) return rc;
    HostBlock *blk = static_cast<HostBlock *>(host->host_block);
    const size_t W = a.W;
    const double blocks = std::max(1, a.blk_off.back());
    for (size_t k = 0; k < a.members.size(); ++k) {
      const int i = a.members[k];
      if (B->run_status[i]) continue;
      ompdart_result v;
      arena_view(a, (int)k, &v);
      // this CFG's share of the arena's host<->device copies
      const double share = (a.blk_off[k + 1] - a.blk_off[k]) / blocks;
      const size_t b0 = (size_t)a.blk_off[k] * W;
      v.h_in = host->h_in + b0;
      v.d_in = host->d_in + b0;
      v.h_out = host->h_out ? host->h_out + b0 : nullptr;
      v.d_out = host->d_out ? host->d_out + b0 : nullptr;
      v.live_in = host->live_in ? host->live_in + b0 : nullptr;
      v.acc_flag = host->acc_flag + a.acc_base[k];
      v.edge_xfers = host->edge_xfers + a.rec_off[k];
      v.exit_blocks = host->exit_blocks + a.x_off[k];
      v.from_exit = host->from_exit + (size_t)a.x_off[k] * W;
      v.call_site_acc = host->call_site_acc + a.site_off[k];
      const size_t o = (size_t)a.site_off[k] * W;
      v.call_to = host->call_to + o;
      v.call_from = host->call_from + o;
      v.call_entry_h = host->call_entry_h + o;
      v.call_entry_d = host->call_entry_d + o;
      v.call_exit_live = host->call_exit_live + o;
      v.h2d_bytes = (long long)(share * v.h2d_bytes);
      v.d2h_bytes = (long long)(share * host->d2h_bytes);
      outs[i] = result_in_block(v, blk);
      if (!outs[i]) {
        rc = set_error(OMPDART_E_NOMEM, "host allocation failed");
        break;
      }
    }
    ompdart_result_free(host);
    if (rc) return rc;
  }
  for (auto &p : B->solos) {
    if (B->run_status[p->member]) continue;
    rc = ompdart_batch_fetch(B, p->member, &outs[p->member]);
    if (rc) return rc;
  }
  return OMPDART_OK;
}

}  // namespace ompdart
