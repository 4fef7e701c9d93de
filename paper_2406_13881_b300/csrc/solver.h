// solver.h -- internal interfaces between the files of libompdart.
#pragma once
#include <cuda_runtime.h>

#include <chrono>
#include <cstdint>
#include <cstdio>
#include <deque>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ompdart.h"
#include "ingest.h"
#include "plan.cuh"

namespace ompdart {

struct HostBlock;

// ---- host-side tracing: with OMPDART_TRACE=1 in the environment, phases
// of plan and batch construction print their wall time to stderr
bool trace_on();
struct TraceScope {
  const char *name;
  long long n;
  std::chrono::steady_clock::time_point t0;
  explicit TraceScope(const char *nm, long long count = -1)
      : name(nm), n(count), t0(std::chrono::steady_clock::now()) {}
  // report the phase so far and start the next one
  void next(const char *nm, long long count = -1) {
    report();
    name = nm;
    n = count;
    t0 = std::chrono::steady_clock::now();
  }
  ~TraceScope() { report(); }

 private:
  void report() const {
    if (!trace_on()) return;
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    std::fprintf(stderr, "[ompdart] %-22s %9.3f ms  (%lld)\n", name, ms, n);
  }
};

// ---- staging.cpp: CFGs given in device memory (ompdart_cfg.mem =
// OMPDART_MEM_DEVICE) copied to host buffers for ingestion
struct StagedCfgs {
  std::vector<ompdart_cfg> cfgs;           // the CFGs with host pointers
  std::deque<std::vector<uint8_t>> bufs;   // host copies of the device arrays
  std::map<std::pair<const void *, size_t>, const void *> seen;  // one copy per device array
  std::vector<int> rc;                     // per CFG (per_cfg mode): its staging error or OK
  std::vector<std::string> err;
};
// *out = in when every CFG is in host memory, else st->cfgs.  A CFG that
// cannot be staged fails the call (per_cfg false) or, with per_cfg, is
// replaced by an empty CFG that ingestion rejects and its code is left in
// st->rc[i] for the caller to report.
int stage_cfgs(const ompdart_cfg *in, int n, StagedCfgs *st, const ompdart_cfg **out, std::string *err,
               bool per_cfg = false);

// ---- api.cu: thread-local error text of ompdart_last_error
void set_last_error_text(const std::string &msg);
int set_error(int code, const std::string &msg);  // sets the text, returns code

// ---- sweep.cu: the general solver (any CFG, one CFG per plan)
int enqueue_local_summary(const DevPlan &p, cudaStream_t s, Prof *pf);
int enqueue_fill_unreachable(const DevPlan &p, cudaStream_t s, int keep_states, Prof *pf);
int enqueue_sweep_solver(const DevPlan &p, cudaStream_t s, int n_fin, Prof *pf);
int enqueue_sweep_edges(const DevPlan &p, cudaStream_t s, int n_fin);

// Call table of a plan (Sec. IV-C): rows of 7 planes of W words (ReqH,
// ReqD, GenH, KillH, GenD, KillD, MustDef) on the host; a batch lays its
// CFGs' tables end to end and a call access's row is local to its CFG.
struct CallHost {
  const uint64_t *planes = nullptr;  // [rows][7][W]
  int rows = 0;
  std::vector<int32_t> row_base;     // per CFG of the plan (empty: 0)
  // per CFG of the plan: the first CFG given with the same arrays and call
  // table (its blocks fold to the same records), itself if none; empty: all
  // distinct
  std::vector<int32_t> same_as;
};

// ---- calls.cu: the call-site pass (after the host-validity pass)
int enqueue_call_sites(const DevPlan &p, cudaStream_t s, Prof *pf);

// ---- scan.cu: the chunked scan solver (reducible CFGs with contiguous
// loop bodies; one CFG or a batch of CFGs laid end to end)
int scan_supported(const Ingest &g);
struct ScanState;
// acc_off/acc: accesses of the plan's blocks (CSR over g's block ids);
// cfg_err: device [n_cfg] per-CFG error flags or null; wpc: warps per CTA
// of the chain kernels (0 = default)
ScanState *scan_create(const Ingest &g, const int32_t *acc_off, const uint32_t *acc, const CallHost &calls,
                       int32_t *cfg_err, DevPlan &p, int chunk_target, int keep_states, std::string *err, int wpc);
bool scan_grow_streams(ScanState *st);
long long scan_h2d_bytes(const ScanState *st);
int enqueue_scan_solver(ScanState *st, const DevPlan &p, cudaStream_t s, Prof *pf);
int enqueue_scan_edges(ScanState *st, const DevPlan &p, cudaStream_t s, Prof *pf);
// after a completed run: index of the first gathered transfer record of
// every chunk, and `total` at index C
bool scan_chunk_record_offsets(const ScanState *st, cudaStream_t s, std::vector<int32_t> *out, int32_t total);
long long scan_device_bytes(const ScanState *st);
void scan_destroy(ScanState *st);

// ---- classify.cu: directive classification of the data-region mode
// (device arrays of one plan; per-CFG arrays indexed by the CFG of a batch)
struct ClsDev {
  long long A;
  int W, n_cfg, n_k, n_rin;
  const uint32_t *acc;       // [A] the accesses the analysis read
  const int32_t *acc_off;    // [N+1]
  const int32_t *acc_blk;    // [A] block of each access
  const int32_t *pos;        // [N] position or -1 (unreachable)
  const int32_t *kern;       // [N] plan-wide kernel index or -1
  const int32_t *blk_cfg;    // [N] CFG of each block
  const int32_t *acc_base;   // [n_cfg] first access of each CFG
  const uint8_t *acc_flag;   // [A]
  uint64_t *kw_h, *kw_d;     // [n_k][W] written by kernel k on the host / device (scratch)
  uint64_t *kernel_to, *kernel_from;  // [n_k][W]
  uint64_t *dev_touched;     // [n_cfg][W] (scratch)
  int32_t *acc_point;        // [A] insertion point (index local to the CFG) or -1
  const int32_t *rin_off, *rout_off;  // [n_cfg+1] boundary rows: entry rows, then n_rin + exit rows
  const int32_t *xin_off, *xin;       // [n_cfg+1], exit indices of the exits inside the region
  const uint8_t *has_r, *entry_in_r;  // [n_cfg]
  const int32_t *start_k;    // [n_cfg] kernel whose entry opens the region, or -1
  const uint64_t *bnd_to, *bnd_from, *from_exit;
  uint64_t *map_to, *map_from, *map_alloc;  // [n_cfg][W]
};
int enqueue_classify(const ClsDev &c, cudaStream_t s, Prof *pf);

// ---- staging.cpp: firstprivate (Sec. IV-D, scalar paragraph).  With
// cfg.region and cfg.scalar_vars: the device reads of a scalar that a kernel
// reads and never writes are relabelled as host reads in a copy of the
// access array kept in *st (*out points at it); fp receives the
// [n_kernels * W] firstprivate rows, *n_kernels = max kernel id + 1 (0
// without region).  Returns OMPDART_E_INVALID for a kernel id outside
// [-1, n_blocks).  The CFG must have passed ingestion's format checks.
int firstprivate_view(const ompdart_cfg &in, StagedCfgs *st, ompdart_cfg *out, std::vector<uint64_t> *fp,
                      int *n_kernels, std::string *err);

// ---- api.cu: one device plan over one CFG or a batch of CFGs of equal
// word count (shared by the single-CFG plan and the batch)
struct PlanCore {
  Ingest g;
  DevPlan dp{};
  std::vector<void *> allocs;
  int path = 1;  // 1 sweep, 2 scan
  int n_fin = 0;
  int keep_states = 0;
  long long h2d = 0;
  ScanState *scan = nullptr;
  int32_t *cfg_err = nullptr;  // device [n_cfg] (scan path)
  std::vector<int32_t> site_acc;   // host copy: access index of each call site
  // data region and directives (region mode): device arrays and the host
  // per-CFG offsets views need
  bool region = false;
  ClsDev cls{};
  uint8_t *d_in_region = nullptr;
  int32_t *d_rin = nullptr, *d_rout = nullptr;
  uint64_t *d_fp = nullptr;
  std::vector<int32_t> h_kern_off, h_rin_off, h_rout_off, h_acc_base;

  long long dev_bytes = 0;  // device bytes this core holds (with its scan state)

  template <class T>
  T *dalloc(size_t n) {
    const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
    void *ptr = dev_malloc(bytes);
    if (!ptr) return nullptr;
    allocs.push_back(ptr);
    dev_bytes += (long long)bytes;
    return static_cast<T *>(ptr);
  }
  template <class T>
  T *upload(const T *src, size_t n) {
    T *d = dalloc<T>(n);
    if (d && n && cudaMemcpy(d, src, n * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
    h2d += (long long)(n * sizeof(T));
    return d;
  }
  template <class T>
  T *upload(const std::vector<T> &v) {
    return upload(v.data(), v.size());
  }
  PlanCore() = default;
  PlanCore(const PlanCore &) = delete;
  PlanCore &operator=(const PlanCore &) = delete;
  ~PlanCore();
};

// Boundary rows of one CFG (Sec. IV-D entry states and region-exit
// liveness), padding bits cleared: appended to top, eh, ed, xl.
void boundary_rows(const ompdart_cfg *cfg, int W, std::vector<uint64_t> *top, std::vector<uint64_t> *eh,
                   std::vector<uint64_t> *ed, std::vector<uint64_t> *xl);

// Upload c->g (ingested; a batch concatenated) and its accesses, choose the
// solver (path 0 auto, 1 sweep, 2 scan; a batch must take the scan) and
// allocate every plane.  unreach_cfg: CFG of each unreachable block in
// ascending block order (empty for one CFG).  Returns an OMPDART_* code.
// fp: the firstprivate rows of every kernel ([n_kernels][W], kernels
// numbered plan-wide by Ingest::kern_off; empty = none).
int core_build(PlanCore *c, const int32_t *acc_off, const uint32_t *acc, const CallHost &calls,
               const std::vector<uint64_t> &top, const std::vector<uint64_t> &eh, const std::vector<uint64_t> &ed,
               const std::vector<uint64_t> &xl, int n_cfg, const std::vector<int32_t> &unreach_cfg,
               const ompdart_opts &o, std::string *err, const std::vector<uint64_t> &fp = {});
// Enqueue one full run on s; returns the number of kernels launched.
int core_enqueue(PlanCore *c, cudaStream_t s, Prof *pf);
// After the stream finished a run (h_status: its ST_COUNT status words):
// regrow overflowed record buffers and redo the emission (synchronously).
// *rerun is set when buffers changed (captured graphs must be rebuilt).
int core_finish(PlanCore *c, cudaStream_t s, int32_t *h_status, bool *rerun);
// Device view of a core's results (h_status: the status words of its last run).
void core_view(const PlanCore &c, const int32_t *h_status, ompdart_result *v);
// Copy the device arrays a view points at into a new host result
// (ompdart_result_free) whose arrays share one host block (page-locked if
// `pin`), on stream s.
// A page-locked staging buffer owned by one user (a plan): small copies to
// and from the device land here asynchronously.  get(bytes) returns a
// buffer of at least `bytes' (grown on demand), or NULL for a request above
// kMax or when page-locking fails (the caller then copies directly).
struct HostStage {
  static constexpr size_t kMax = size_t(4) << 20;
  void *p = nullptr;
  size_t cap = 0;
  void *get(size_t bytes) {
    if (bytes > kMax) return nullptr;
    if (bytes > cap) {
      if (p) cudaFreeHost(p);
      p = nullptr;
      cap = 0;
      size_t want = 4096;
      while (want < bytes) want <<= 1;
      if (cudaHostAlloc(&p, want, cudaHostAllocPortable) != cudaSuccess) {
        (void)cudaGetLastError();
        p = nullptr;
        return nullptr;
      }
      cap = want;
    }
    return p;
  }
  ~HostStage() {
    if (p) cudaFreeHost(p);
  }
};
int result_copy(const ompdart_result &v, bool pin, cudaStream_t s, ompdart_result **out, HostStage *stage = nullptr);
// A new host result whose arrays are v's, all inside `block` (one more
// reference to it); NULL if the host allocation fails.
ompdart_result *result_in_block(const ompdart_result &v, HostBlock *block);

// ---- api.cu: hooks of the serving loop's resident mode on a plan
// Upload the entry / exit rows of `cfg' (a CFG with the plan's graph) into
// the plan's device rows on `stream'.
int plan_set_boundary(ompdart_plan *plan, const ompdart_cfg *cfg, cudaStream_t stream);
// Device bytes a plan holds.
long long plan_device_bytes(const ompdart_plan *plan);

// ---- hostmem.cpp: reference-counted host blocks for host results
// (page-locked or pageable; cached by size class once released when large)
HostBlock *host_block_new(size_t bytes, bool pin);  // one reference; NULL on failure
void *host_block_ptr(HostBlock *b);
void host_block_ref(HostBlock *b);
void host_block_release(HostBlock *b);  // frees or caches at the last reference

// ---- batch.cu helpers for the serving loop
// host copies of every CFG's results after ompdart_batch_sync (outs[n];
// NULL where a CFG's status is an error)
int batch_fetch_all(ompdart_batch *B, ompdart_result **outs);
long long batch_device_bytes(const ompdart_batch *B);
cudaStream_t batch_stream(const ompdart_batch *B);
// device bytes a plan of this CFG is expected to hold (admission estimate)
long long estimate_device_bytes(const ompdart_cfg &c, int keep_states);

// ---- summary.cu: callee summaries (rows[i]: 7 * W_i words, callee numbering)
int summarize_run(const ompdart_cfg *cfgs, int n, const ompdart_opts &o, uint64_t *const *rows, int32_t *status);
void map_summary(const uint64_t *sum, int callee_vars, const int32_t *var_map, int caller_vars, uint64_t *row);

}  // namespace ompdart
