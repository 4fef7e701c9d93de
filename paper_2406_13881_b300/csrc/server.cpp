// server.cpp -- the serving loop (ompdart_server_*): continuous batching of
// analysis requests over the batched analysis, admitted by a device-memory
// budget.
//
// One worker thread owns the GPU side.  Each turn it
//   1. retires batches whose completion event fired: per-CFG status, host
//      copies of the results, the batch's device memory back to the pool
//      and to the budget, latencies recorded, waiters woken;
//   2. admits pending requests in arrival order into a new batch while the
//      number of batches on the GPU is below max_inflight, the batch is
//      below max_batch CFGs and the estimated device bytes of everything
//      admitted stay within the budget (a request larger than the whole
//      budget fails with OMPDART_E_BUDGET); the batch is ingested and
//      uploaded on the host while earlier batches run, then launched on its
//      own stream, so batches overlap on the device.
// Submitting copies the request, so callers may reuse their buffers.
//
// Resident mode (opts.resident): `workers' threads take requests in
// arrival order, up to 16 at a time each, and serve each from a cache of
// device-resident plans keyed by the CFG's content (its entry and exit rows
// excluded): a hit uploads the request's rows into the cached plan and
// replays its graph on a stream of its own, so a group runs on the device
// together; a miss builds the plan and keeps it, dropping the least
// recently used idle plans when the device budget would overflow.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ompdart.h"
#include "solver.h"

using namespace ompdart;

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kResidentGroup = 16;  // resident mode: streams (requests in flight) per worker by default

struct Request {
  int64_t id = 0;
  std::vector<int32_t> so, su, ao;
  std::vector<uint32_t> acc;
  std::vector<uint64_t> eh, ed, xl, calls, scalars;
  std::vector<int32_t> region;
  ompdart_cfg cfg{};
  long long est = 0;
  Clock::time_point t_submit, t_done;
  int status = OMPDART_OK;
  std::string err;  // why it failed
  ompdart_result *res = nullptr;
  bool done = false;
};
using ReqPtr = std::shared_ptr<Request>;

struct InFlight {
  ompdart_batch *b = nullptr;
  std::vector<ReqPtr> reqs;
  long long bytes = 0;
  cudaEvent_t ev = nullptr;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct ompdart_server {
  ompdart_server_opts o{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<ReqPtr> pending;
  std::map<int64_t, ReqPtr> live;  // submitted and not yet collected by a wait
  std::vector<InFlight> inflight;  // worker thread only
  int n_inflight = 0;              // guarded by mu (for drain)
  std::thread worker;
  bool stop = false;
  int64_t next_id = 1;
  long long bytes_in_use = 0, peak_bytes = 0;
  int64_t submitted = 0, completed = 0, failed = 0, batches = 0, batched_cfgs = 0;
  std::vector<double> lat_ms;
  // ---- resident mode
  struct Cached {
    ompdart_plan *plan = nullptr;
    std::mutex run;         // runs of one plan are serialised
    long long bytes = 0;
    uint64_t last_use = 0;  // LRU clock (guarded by cache_mu)
    ~Cached() { ompdart_plan_destroy(plan); }
  };
  struct KeyHash {
    size_t operator()(const std::pair<uint64_t, uint64_t> &k) const { return (size_t)(k.first ^ (k.second * 31)); }
  };
  std::vector<std::thread> workers;
  // the workers' streams (a group's worth each), owned by the server: a
  // cached plan synchronises the stream it last ran on when it is
  // destroyed, so the streams outlive the cache
  std::vector<cudaStream_t> worker_streams;
  std::mutex cache_mu;
  std::unordered_map<std::pair<uint64_t, uint64_t>, std::shared_ptr<Cached>, KeyHash> cache;
  long long cache_bytes = 0;
  uint64_t lru_clock = 0;
  int64_t cache_hits = 0, cache_misses = 0;
};

namespace {

void finish_request(ompdart_server *S, const ReqPtr &r, int status, ompdart_result *res, Clock::time_point now,
                    const std::string &err = std::string()) {
  r->status = status;
  r->err = err;
  r->res = res;
  r->t_done = now;
  r->done = true;
  S->lat_ms.push_back(ms_between(r->t_submit, now));
  if (status == OMPDART_OK)
    ++S->completed;
  else
    ++S->failed;
}

// Retire a batch whose work is done (the event fired or failed).
void retire(ompdart_server *S, InFlight &f, cudaError_t q) {
  const size_t n = f.reqs.size();
  std::vector<int32_t> st(n, OMPDART_OK);
  std::vector<ompdart_result *> outs(n, nullptr);
  int rc = q == cudaSuccess ? ompdart_batch_sync(f.b, st.data())
                            : set_error(OMPDART_E_CUDA, std::string("batch run: ") + cudaGetErrorString(q));
  if (!rc && S->o.keep_results) rc = batch_fetch_all(f.b, outs.data());
  const std::string err = rc ? ompdart_last_error() : "";
  ompdart_batch_destroy(f.b);
  cudaEventDestroy(f.ev);
  const Clock::time_point now = Clock::now();
  std::lock_guard<std::mutex> lk(S->mu);
  S->bytes_in_use -= f.bytes;
  --S->n_inflight;
  for (size_t k = 0; k < n; ++k) {
    if (rc && outs[k]) {
      ompdart_result_free(outs[k]);
      outs[k] = nullptr;
    }
    const int code = rc ? rc : st[k];
    finish_request(S, f.reqs[k], code, outs[k], now, rc ? err : code ? "the CFG was rejected or did not converge" : "");
  }
  S->cv_done.notify_all();
}

// Build and launch one batch of admitted requests (reserved: their estimate).
void launch(ompdart_server *S, std::vector<ReqPtr> &take, long long reserved) {
  const int n = (int)take.size();
  std::vector<ompdart_cfg> cfgs(n);
  for (int k = 0; k < n; ++k) cfgs[k] = take[k]->cfg;
  std::vector<int32_t> st(n, OMPDART_OK);
  ompdart_batch *b = nullptr;
  int rc = ompdart_batch_create(cfgs.data(), n, &S->o.opts, &b, st.data());
  cudaEvent_t ev = nullptr;
  if (!rc) rc = ompdart_batch_run(b, nullptr);
  if (!rc && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) rc = OMPDART_E_CUDA;
  if (!rc && cudaEventRecord(ev, batch_stream(b)) != cudaSuccess) rc = OMPDART_E_CUDA;
  if (rc) {
    const std::string err = ompdart_last_error();
    if (ev) cudaEventDestroy(ev);
    if (b) ompdart_batch_destroy(b);
    const Clock::time_point now = Clock::now();
    std::lock_guard<std::mutex> lk(S->mu);
    S->bytes_in_use -= reserved;
    --S->n_inflight;
    for (int k = 0; k < n; ++k) finish_request(S, take[k], rc, nullptr, now, err);
    S->cv_done.notify_all();
    return;
  }
  const long long actual = batch_device_bytes(b);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->bytes_in_use += actual - reserved;  // charge what the batch really holds
    S->peak_bytes = std::max(S->peak_bytes, S->bytes_in_use);
    ++S->batches;
    S->batched_cfgs += n;
  }
  InFlight f;
  f.b = b;
  f.reqs = std::move(take);
  f.bytes = actual;
  f.ev = ev;
  S->inflight.push_back(std::move(f));
}

// ---- resident mode ---------------------------------------------------------------
// 128-bit content key of a CFG: its graph, accesses, call table, kernels and
// scalars (two independent word-wise mixes)
struct Mix {
  uint64_t a = 0x9e3779b97f4a7c15ull, b = 0xc2b2ae3d27d4eb4full;
  void add(uint64_t x) {
    a = (a ^ x) * 0x100000001b3ull;
    a ^= a >> 29;
    b = (b + x) * 0xff51afd7ed558ccdull;
    b ^= b >> 33;
  }
  template <class T>
  void add(const T *p, size_t n) {
    add((uint64_t)n);
    if (!p) return add(0x5bd1e995ull);
    const unsigned char *c = reinterpret_cast<const unsigned char *>(p);
    const size_t bytes = n * sizeof(T);
    size_t i = 0;
    for (; i + 8 <= bytes; i += 8) {
      uint64_t x;
      memcpy(&x, c + i, 8);
      add(x);
    }
    uint64_t t = 0;
    memcpy(&t, c + i, bytes - i);
    add(t);
  }
};
std::pair<uint64_t, uint64_t> content_key(const ompdart_cfg &c) {
  Mix m;
  const size_t N = (size_t)c.n_blocks, W = (size_t)(c.n_vars + 63) / 64;
  m.add((uint64_t)c.n_blocks);
  m.add((uint64_t)c.n_vars);
  m.add((uint64_t)c.entry);
  m.add(c.succ_off, N + 1);
  m.add(c.succ, (size_t)c.succ_off[N]);
  m.add(c.acc_off, N + 1);
  m.add(c.acc, (size_t)c.acc_off[N]);
  m.add(c.call_planes, c.call_planes ? (size_t)c.n_calls * 7 * W : 0);
  m.add(c.region, c.region ? N : 0);
  m.add(c.scalar_vars, c.scalar_vars ? W : 0);
  return {m.a, m.b};
}

void finish_one(ompdart_server *S, const ReqPtr &r, int rc, ompdart_result *res, const std::string &err) {
  const Clock::time_point now = Clock::now();
  std::lock_guard<std::mutex> lk(S->mu);
  --S->n_inflight;
  finish_request(S, r, rc, res, now, err);
  S->cv_done.notify_all();
}

// Make room for `need' more device bytes of cached plans by dropping idle
// plans, least recently used first.  cache_mu held.
void evict_for(ompdart_server *S, long long need) {
  while (S->cache_bytes + need > S->o.hbm_budget_bytes) {
    auto victim = S->cache.end();
    for (auto it = S->cache.begin(); it != S->cache.end(); ++it) {
      if (it->second.use_count() > 1) continue;  // a worker holds it
      if (victim == S->cache.end() || it->second->last_use < victim->second->last_use) victim = it;
    }
    if (victim == S->cache.end()) return;
    S->cache_bytes -= victim->second->bytes;
    S->cache.erase(victim);
  }
}

// The cached plan of a request's CFG, ingested and cached on a miss; NULL
// (the request finished with the error) when it cannot be built.
std::shared_ptr<ompdart_server::Cached> resident_plan(ompdart_server *S, const ReqPtr &r) {
  TraceScope trace("resident: lookup", r->cfg.n_blocks);
  const auto key = content_key(r->cfg);
  std::shared_ptr<ompdart_server::Cached> c;
  {
    std::lock_guard<std::mutex> lk(S->cache_mu);
    auto it = S->cache.find(key);
    if (it != S->cache.end()) {
      c = it->second;
      c->last_use = ++S->lru_clock;
      ++S->cache_hits;
    } else {
      ++S->cache_misses;
    }
  }
  if (c) return c;
  // ingest and build it (outside the locks)
  c = std::make_shared<ompdart_server::Cached>();
  const int rc = ompdart_plan_create(&r->cfg, &S->o.opts, &c->plan);
  if (rc) {
    c->plan = nullptr;
    finish_one(S, r, rc, nullptr, ompdart_last_error());
    return nullptr;
  }
  ompdart_plan_graph(c->plan, 1);  // every later hit replays one graph
  c->bytes = plan_device_bytes(c->plan);
  std::lock_guard<std::mutex> lk(S->cache_mu);
  auto it = S->cache.find(key);
  if (it != S->cache.end()) return it->second;  // another worker built it meanwhile
  evict_for(S, c->bytes);
  if (S->cache_bytes + c->bytes <= S->o.hbm_budget_bytes) {  // else a plan of its own, freed after the run
    S->cache.emplace(key, c);
    S->cache_bytes += c->bytes;
  }
  c->last_use = ++S->lru_clock;
  return c;
}

// A resident worker takes up to one request per stream it owns at a time.
// Each runs on a stream of its own -- upload of its rows, then its cached
// plan's graph -- so the group runs on the device together; then the
// worker waits for each and copies its results back.  Requests for one
// plan run in successive rounds (runs of one plan are serialised), and a
// plan another worker is running is taken in a later round (try_lock: a
// worker never waits for a plan while holding another).
void resident_worker(ompdart_server *S, const cudaStream_t *streams, int n_streams) {
  cudaSetDevice(S->o.device);
  struct Job {
    ReqPtr r;
    std::shared_ptr<ompdart_server::Cached> c;
    int rc = OMPDART_OK;
  };
  for (;;) {
    std::vector<ReqPtr> take;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty(); });
      if (S->pending.empty()) break;  // stopping with nothing left
      while (!S->pending.empty() && (int)take.size() < n_streams) {
        const ReqPtr r = S->pending.front();
        S->pending.pop_front();
        ++S->n_inflight;
        if (r->est > S->o.hbm_budget_bytes) {
          --S->n_inflight;
          finish_request(S, r, OMPDART_E_BUDGET, nullptr, Clock::now(),
                         "the request needs more device memory than the whole budget");
          S->cv_done.notify_all();
          continue;
        }
        take.push_back(r);
      }
    }
    std::vector<Job> jobs;
    jobs.reserve(take.size());
    for (const ReqPtr &r : take) {
      auto c = resident_plan(S, r);
      if (c) jobs.push_back(Job{r, std::move(c)});
    }
    std::vector<Job *> rest;
    for (Job &j : jobs) rest.push_back(&j);
    while (!rest.empty()) {
      std::vector<Job *> round, later;
      for (Job *j : rest) {
        bool dup = false;
        for (Job *x : round) dup = dup || x->c == j->c;
        if (!dup && j->c->run.try_lock())
          round.push_back(j);
        else
          later.push_back(j);
      }
      if (round.empty()) {  // every plan is busy elsewhere: wait for the first, holding none
        later.front()->c->run.lock();
        round.push_back(later.front());
        later.erase(later.begin());
      }
      {
        TraceScope trace("resident: launch", (long long)round.size());
        for (size_t k = 0; k < round.size(); ++k) {
          Job *j = round[k];
          const cudaStream_t st = streams[k % n_streams];
          j->rc = plan_set_boundary(j->c->plan, &j->r->cfg, st);
          if (!j->rc) j->rc = ompdart_plan_run(j->c->plan, st);
        }
      }
      for (Job *j : round) {
        TraceScope trace("resident: wait+fetch", j->r->cfg.n_blocks);
        ompdart_result *res = nullptr;
        int rc = j->rc;
        if (!rc) rc = ompdart_plan_sync(j->c->plan);
        if (!rc && S->o.keep_results) rc = ompdart_plan_fetch(j->c->plan, &res);
        const std::string err = rc ? ompdart_last_error() : "";
        j->c->run.unlock();
        j->c.reset();  // an uncached plan dies with its last reference
        finish_one(S, j->r, rc, res, err);
      }
      rest.swap(later);
    }
  }
}

void worker_main(ompdart_server *S) {
  cudaSetDevice(S->o.device);
  for (;;) {
    bool progressed = false;
    for (size_t i = 0; i < S->inflight.size();) {
      const cudaError_t q = cudaEventQuery(S->inflight[i].ev);
      if (q == cudaErrorNotReady) {
        (void)cudaGetLastError();  // "not ready" is an answer, not an error
        ++i;
        continue;
      }
      retire(S, S->inflight[i], q);
      S->inflight.erase(S->inflight.begin() + (long)i);
      progressed = true;
    }
    std::vector<ReqPtr> take;
    long long est = 0;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      if (S->stop && S->pending.empty() && S->inflight.empty()) break;
      const Clock::time_point now = Clock::now();
      if ((int)S->inflight.size() < S->o.max_inflight) {
        while (!S->pending.empty() && (int)take.size() < S->o.max_batch) {
          const ReqPtr r = S->pending.front();
          if (r->est > S->o.hbm_budget_bytes) {  // can never fit
            S->pending.pop_front();
            finish_request(S, r, OMPDART_E_BUDGET, nullptr, now,
                           "the request needs more device memory than the whole budget");
            S->cv_done.notify_all();
            continue;
          }
          if (S->bytes_in_use + est + r->est > S->o.hbm_budget_bytes) break;
          est += r->est;
          take.push_back(r);
          S->pending.pop_front();
        }
        if (!take.empty()) {
          S->bytes_in_use += est;
          ++S->n_inflight;
        }
      }
      if (take.empty() && !progressed) {
        if (S->inflight.empty())
          S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty(); });
        else
          S->cv_work.wait_for(lk, std::chrono::microseconds(20));
        continue;
      }
    }
    if (!take.empty()) launch(S, take, est);
  }
}

}  // namespace

extern "C" {

int ompdart_server_create(const ompdart_server_opts *opts, ompdart_server **out) {
  set_last_error_text("");
  if (!out) return set_error(OMPDART_E_INVALID, "server output pointer is NULL");
  *out = nullptr;
  ompdart_server *S = new (std::nothrow) ompdart_server();
  if (!S) return set_error(OMPDART_E_NOMEM, "host allocation failed");
  if (opts) S->o = *opts;
  if (S->o.hbm_budget_bytes <= 0) S->o.hbm_budget_bytes = 40ll << 30;
  // resident mode: max_batch is the group a worker launches at once
  const int group = S->o.max_batch > 0 ? std::min(S->o.max_batch, 256) : kResidentGroup;
  if (S->o.max_batch <= 0) S->o.max_batch = 4096;
  if (S->o.max_inflight <= 0) S->o.max_inflight = 2;
  S->o.opts.device = S->o.device;
  // a serving batch runs once: capturing it into a graph would cost more
  // than it saves, so its kernels are launched directly
  S->o.opts.no_graph = 1;
  if (cudaSetDevice(S->o.device) != cudaSuccess) {
    delete S;
    return set_error(OMPDART_E_CUDA, "cudaSetDevice failed");
  }
  if (S->o.resident) {
    const int nw = S->o.workers > 0 ? S->o.workers : 4;
    for (int k = 0; k < nw * group; ++k) {
      cudaStream_t x = nullptr;
      if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess) {
        for (cudaStream_t y : S->worker_streams) cudaStreamDestroy(y);
        delete S;
        return set_error(OMPDART_E_CUDA, "stream creation failed");
      }
      S->worker_streams.push_back(x);
    }
    for (int k = 0; k < nw; ++k)
      S->workers.emplace_back(resident_worker, S, S->worker_streams.data() + (size_t)k * group, group);
  } else {
    S->worker = std::thread(worker_main, S);
  }
  *out = S;
  return OMPDART_OK;
}

int ompdart_server_submit(ompdart_server *S, const ompdart_cfg *c, int64_t *ticket) {
  if (!S || !c || !ticket) return set_error(OMPDART_E_INVALID, "NULL argument");
  StagedCfgs staged;  // a CFG in device memory: its arrays copied to the host first
  {
    std::string serr;
    const int src = stage_cfgs(c, 1, &staged, &c, &serr);
    if (src) return set_error(src, serr);
  }
  if (c->n_blocks < 1 || !c->succ_off || !c->acc_off || c->n_vars < 1)
    return set_error(OMPDART_E_INVALID, "malformed CFG header");
  ReqPtr r = std::make_shared<Request>();
  const int N = c->n_blocks, W = (c->n_vars + 63) / 64;
  const int E = c->succ_off[N], A = c->acc_off[N];
  if (E < 0 || A < 0 || (E && !c->succ) || (A && !c->acc)) return set_error(OMPDART_E_INVALID, "malformed CSR");
  r->so.assign(c->succ_off, c->succ_off + N + 1);
  r->su.assign(c->succ, c->succ + E);
  r->ao.assign(c->acc_off, c->acc_off + N + 1);
  r->acc.assign(c->acc, c->acc + A);
  if (c->entry_host_valid) r->eh.assign(c->entry_host_valid, c->entry_host_valid + W);
  if (c->entry_dev_valid) r->ed.assign(c->entry_dev_valid, c->entry_dev_valid + W);
  if (c->exit_host_live) r->xl.assign(c->exit_host_live, c->exit_host_live + W);
  if (c->call_planes && c->n_calls > 0) r->calls.assign(c->call_planes, c->call_planes + (size_t)c->n_calls * 7 * W);
  if (c->region) r->region.assign(c->region, c->region + N);
  if (c->scalar_vars) r->scalars.assign(c->scalar_vars, c->scalar_vars + W);
  r->cfg = *c;
  r->cfg.succ_off = r->so.data();
  r->cfg.succ = r->su.data();
  r->cfg.acc_off = r->ao.data();
  r->cfg.acc = r->acc.data();
  r->cfg.entry_host_valid = c->entry_host_valid ? r->eh.data() : nullptr;
  r->cfg.entry_dev_valid = c->entry_dev_valid ? r->ed.data() : nullptr;
  r->cfg.exit_host_live = c->exit_host_live ? r->xl.data() : nullptr;
  r->cfg.call_planes = r->calls.empty() ? nullptr : r->calls.data();
  r->cfg.region = c->region ? r->region.data() : nullptr;
  r->cfg.scalar_vars = c->scalar_vars ? r->scalars.data() : nullptr;
  r->est = estimate_device_bytes(r->cfg, S->o.opts.keep_states);
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->stop) return set_error(OMPDART_E_INVALID, "server is shutting down");
  r->id = S->next_id++;
  r->t_submit = Clock::now();
  S->pending.push_back(r);
  S->live[r->id] = r;
  ++S->submitted;
  *ticket = r->id;
  S->cv_work.notify_one();
  return OMPDART_OK;
}

int ompdart_server_replay(ompdart_server *S, const ompdart_cfg *cfgs, int32_t n, const double *arrival_us,
                          int64_t *tickets) {
  if (!S || (n > 0 && (!cfgs || !arrival_us || !tickets))) return set_error(OMPDART_E_INVALID, "NULL argument");
  const Clock::time_point t0 = Clock::now();
  for (int i = 0; i < n; ++i) {
    const Clock::time_point due = t0 + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double, std::micro>(arrival_us[i]));
    while (Clock::now() < due) {
      const auto left = due - Clock::now();
      if (left > std::chrono::microseconds(200)) std::this_thread::sleep_for(left - std::chrono::microseconds(100));
    }
    tickets[i] = -1;
    const int rc = ompdart_server_submit(S, &cfgs[i], &tickets[i]);
    if (rc) return rc;
  }
  return OMPDART_OK;
}

int ompdart_server_wait(ompdart_server *S, int64_t ticket, int32_t timeout_ms, ompdart_result **out,
                        int32_t *status, double *latency_ms) {
  if (!S) return set_error(OMPDART_E_INVALID, "server is NULL");
  if (out) *out = nullptr;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->live.find(ticket);
  if (it == S->live.end()) return set_error(OMPDART_E_INVALID, "unknown or already collected ticket");
  ReqPtr r = it->second;
  const auto pred = [&] { return r->done; };
  if (timeout_ms < 0)
    S->cv_done.wait(lk, pred);
  else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
    return set_error(OMPDART_E_TIMEOUT, "the request is not done yet");
  if (status) *status = r->status;
  if (latency_ms) *latency_ms = ms_between(r->t_submit, r->t_done);
  set_last_error_text(r->err);  // why the request failed, for ompdart_last_error
  if (out)
    *out = r->res;
  else if (r->res)
    ompdart_result_free(r->res);
  r->res = nullptr;
  S->live.erase(it);
  return OMPDART_OK;
}

int ompdart_server_drain(ompdart_server *S, int32_t timeout_ms) {
  if (!S) return set_error(OMPDART_E_INVALID, "server is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  const auto pred = [&] { return S->pending.empty() && S->n_inflight == 0; };
  if (timeout_ms < 0)
    S->cv_done.wait(lk, pred);
  else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
    return set_error(OMPDART_E_TIMEOUT, "requests still pending");
  return OMPDART_OK;
}

int ompdart_server_get_stats(ompdart_server *S, ompdart_server_stats *out) {
  if (!S || !out) return set_error(OMPDART_E_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  memset(out, 0, sizeof *out);
  out->submitted = S->submitted;
  out->completed = S->completed;
  out->failed = S->failed;
  out->batches = S->batches;
  out->mean_batch = S->batches ? (double)S->batched_cfgs / S->batches : 0.0;
  out->peak_bytes = S->peak_bytes;
  out->bytes_in_use = S->bytes_in_use;
  {
    std::lock_guard<std::mutex> ck(S->cache_mu);
    out->cache_hits = S->cache_hits;
    out->cache_misses = S->cache_misses;
    out->cached_plans = (int64_t)S->cache.size();
    if (S->o.resident) {
      out->bytes_in_use = S->cache_bytes;
      out->peak_bytes = std::max<int64_t>(out->peak_bytes, S->cache_bytes);
    }
  }
  std::vector<double> l = S->lat_ms;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    auto q = [&](double p) { return l[std::min(l.size() - 1, (size_t)(p * (l.size() - 1) + 0.5))]; };
    out->p50_ms = q(0.50);
    out->p99_ms = q(0.99);
    out->max_ms = l.back();
  }
  return OMPDART_OK;
}

void ompdart_server_destroy(ompdart_server *S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();  // finishes what was submitted
  for (auto &t : S->workers) t.join();
  S->cache.clear();  // the cached plans (each synchronises its last stream)
  for (cudaStream_t x : S->worker_streams) cudaStreamDestroy(x);
  for (auto &kv : S->live)
    if (kv.second->res) ompdart_result_free(kv.second->res);
  delete S;
}

}  // extern "C"
