/*
 * ompdart.h -- C ABI of libompdart.so: host/device validity data-flow of
 * OpenMP offload programs on one NVIDIA B300 (sm_103a).
 *
 * The analysis is the one of Marzen et al., "Static Generation of Efficient
 * OpenMP Offload Data Mappings" (SC24):
 *   - Sec. IV-D: data is valid in a memory space if it was last written
 *     there; a write in one space makes the other stale; a read that may see
 *     stale data is a true (read-after-write) dependency and needs one of
 *     the Table II constructs; WAR/WAW need nothing.
 *   - Sec. IV-D (loops) and Algorithm 1: a need inside a loop is met before
 *     the loop when the data stays valid to the end of the loop body,
 *     otherwise inside the loop.
 *   - Sec. IV-D (last paragraph) and Sec. II-B: at the region exit, data the
 *     host may read afterwards must be valid on the host (`from').
 *   - Sec. IV-C: call sites carry the callee's side effects on globals and
 *     pointer parameters (see ompdart_summarize_callee).
 *
 * INPUT FORMAT (the same for every entry point)
 *   A CFG is n_blocks basic blocks, block `entry' has no predecessors.
 *   succ_off[n_blocks+1], succ[n_edges]: CSR successor lists; the edge id
 *       of succ[k] is k.  Duplicate edges are allowed (each is its own edge).
 *   acc_off[n_blocks+1], acc[n_acc]: the ordered accesses of each block
 *       (Sec. IV-B classification), packed as uint32:
 *         bits  0-23  variable id (< n_vars)
 *         bits 24-25  kind: 1 read, 2 write, 3 read-then-write (also used
 *                     for "unknown", which the paper treats pessimistically)
 *         bit  26     space: 0 host, 1 target (inside an offload kernel)
 *         bits 27-30  zero
 *         bit  31     call pseudo-access: bits 0-30 index the call table
 *   Variable sets are bit planes of W = ceil(n_vars/64) uint64 words:
 *   variable v is bit (v % 64) of word (v / 64); bits >= n_vars are zero.
 *
 * OUTPUT (ompdart_result)
 *   h_in, d_in [n_blocks*W]: at the entry of each block, the variables
 *       whose latest value is on the host / on the device (after the edge
 *       transfers into the block).  Blocks unreachable from the entry are
 *       all-ones.  h_out, d_out likewise at block exit (opts.keep_states).
 *   acc_flag [n_acc]: 0 nothing, 1 `update to' (host->device) right before
 *       this access, 2 `update from' (device->host) right before it.
 *   edge_xfers [n_edge_xfers]: {edge, word, to_bits, from_bits} records for
 *       transfers on CFG edges (hoisted before a loop, Sec. IV-D, or at a
 *       join where the incoming paths disagree); order unspecified; only
 *       words with a nonzero transfer appear.
 *   exit_blocks [n_exits], from_exit [n_exits*W]: `from' at the end of each
 *       reachable block without successors (region exit liveness).
 *   Call sites (Sec. IV-C), one per call pseudo-access in access order:
 *       call_to / call_from [n_call_sites*W]: the callee's requirements met
 *       right before the call (ReqD stale on the device -> `to', ReqH stale
 *       on the host -> `from'); acc_flag of the call access is 1 | 2 as
 *       either is nonzero; call_entry_h / call_entry_d: the validity the
 *       callee starts from (the context for its own analysis);
 *       call_exit_live: variables live (read in either space before being
 *       written) right after the call.
 *
 * CALLS
 *   A call pseudo-access applies row r of the call table: requirements
 *   first (ReqH / ReqD: the callee reads them there before writing them),
 *   then the net effect (GenS valid, else KillS stale, else unchanged;
 *   MustDef ends liveness), as ompdart_summarize_callee computes them.  CFGs
 *   with calls take the chunked scan solver (reducible CFG, loop bodies
 *   contiguous in loop order); others return OMPDART_E_INVALID.
 *
 * DATA REGION AND DIRECTIVES (opts.data_region, cfg.region)
 *   The constructs of Table II.  The single target data region R of the
 *   function (Sec. IV-D) is the set of blocks b with S dom b, E pdom b and
 *   b != E, where S is the nearest common dominator of the kernel blocks
 *   and of the headers of the natural loops whose body holds a kernel
 *   block ("begin before any loop capturing the first kernel"), and E the
 *   nearest common post-dominator (towards one virtual exit fed by every
 *   block without successors) of the blocks those kernel blocks and loop
 *   bodies lead to outside themselves ("end after any loop capturing the
 *   last kernel"; E is the virtual exit when there is none).  On every edge
 *   leaving R the host copy of each variable live at its target is made
 *   valid (a `from' there: "if stale data may be read on the host after
 *   exit from a target data region, the from map-type is included"); this
 *   is the one change the mode makes to the analysis.  Then:
 *     map_to      `to's made on every way into R (every edge entering R, or
 *                 the `to's of the kernel whose entry edges are R's);
 *     map_from    `from's made on every way out of R (every edge leaving R
 *                 and every function exit inside R);
 *     map_alloc   variables a kernel accesses on the device with neither;
 *                 tofrom = map_to & map_from;
 *     kernel_to / kernel_from   the `to's (`from's) right before accesses
 *                 inside kernel k, made right before the kernel instead (no
 *                 host code runs in a kernel), less what map_to carries;
 *     acc_point   Sec. IV-F consolidation: a transfer right before a host
 *                 access moves up to just after the previous access of the
 *                 same variable in the block (or to the block's first
 *                 access); all transfers of one direction at one point form
 *                 one `target update'; a call keeps its own;
 *   edge records and exit sets stay as they are: on an edge entering or
 *   leaving R (region_entry_edges / region_exit_edges) and at exits inside
 *   R, the bits in map_to / map_from are carried by the map clauses.
 *
 * ERRORS
 *   Every call returns OMPDART_OK (0) or a negative code; the text of the
 *   last error of the calling thread is ompdart_last_error().  Invalid
 *   inputs never reach the GPU.  Device loops are bounded (max_sweeps); a
 *   bound that runs out makes the call return OMPDART_E_NOCONVERGE and
 *   never traps.
 *
 * OWNERSHIP
 *   Inputs are caller-owned and only read.  Plans and results are
 *   library-owned and freed with ompdart_plan_destroy / ompdart_result_free.
 */
#ifndef OMPDART_H
#define OMPDART_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OMPDART_OK 0
#define OMPDART_E_INVALID (-1)    /* malformed CFG, ids out of range, entry with predecessors */
#define OMPDART_E_NOMEM (-2)      /* host or device allocation failed                         */
#define OMPDART_E_BUDGET (-3)     /* the request does not fit the device memory budget        */
#define OMPDART_E_NOCONVERGE (-4) /* a device loop hit max_sweeps before its fixed point      */
#define OMPDART_E_CUDA (-5)       /* a CUDA runtime call failed (no device, launch failure)   */
#define OMPDART_E_TIMEOUT (-6)    /* a bounded device wait gave up                            */

#define OMPDART_MEM_HOST 0
#define OMPDART_MEM_DEVICE 1

/* One CFG (see INPUT FORMAT).  `mem' says where its arrays live:
   OMPDART_MEM_HOST (0, a zero-initialised struct) for host memory, or
   OMPDART_MEM_DEVICE for device memory of the current CUDA device (every
   non-NULL array pointer must then be a device or managed allocation, else
   OMPDART_E_INVALID).  Ingestion runs on the host, so an entry point given
   device arrays first copies them to host buffers it owns (a device array
   shared by several CFGs of one call is copied once); the caller's arrays
   are only read, and may be reused as soon as the call returns. */
typedef struct {
  int32_t n_blocks, n_vars, entry;
  const int32_t *succ_off, *succ;
  const int32_t *acc_off;
  const uint32_t *acc;
  const uint64_t *entry_host_valid; /* [W]; NULL = every variable valid on the host */
  const uint64_t *entry_dev_valid;  /* [W]; NULL = nothing valid on the device      */
  const uint64_t *exit_host_live;   /* [W]; NULL = every variable live after exit   */
  /* call table for call pseudo-accesses: row r = 7 planes of W words, in
     order ReqH, ReqD, GenH, KillH, GenD, KillD, MustDef (the layout
     ompdart_summarize_callee writes after mapping to caller variables).
     NULL when no access has bit 31 set. */
  const uint64_t *call_planes;
  int32_t n_calls;
  int32_t mem;                      /* OMPDART_MEM_HOST or OMPDART_MEM_DEVICE        */
  /* offload kernels (Sec. IV-B offloaded nodes): region[b] = id (0 ..
     n_blocks-1) of the kernel block b belongs to, or -1 for host code;
     NULL = no kernel information (no data region, no directives). */
  const int32_t *region;
  /* [W] scalar variables (Sec. IV-D firstprivate paragraph); NULL = none.
     With region: a scalar that a kernel reads on the device and never
     writes is passed to that kernel as firstprivate -- its device reads
     there read the private copy made from the host value at the launch,
     so they need the host copy valid and leave the device copy as it was
     (they are analysed as host reads), and the kernel gets a firstprivate
     clause instead of a `to'. */
  const uint64_t *scalar_vars;
} ompdart_cfg;

typedef struct {
  int32_t max_sweeps;   /* bound on device fixed-point sweeps; 0 = 1<<20           */
  int32_t keep_states;  /* nonzero: also produce h_out / d_out                     */
  int32_t path;         /* 0 auto, 1 general sweep solver, 2 chunked scan solver   */
  int32_t chunk_target; /* blocks per chunk for the scan solver; 0 = automatic     */
  int32_t device;       /* CUDA device ordinal                                     */
  int32_t warps_per_cta; /* warps per CTA of the scan solver's walk kernels, 1-4
                            (larger values count as 4); 0 = automatic (4, or
                            the batch autotuner's choice)                        */
  int32_t tune;         /* batches: nonzero = let the autotuner pick chunk_target
                           and warps_per_cta per arena (ompdart_batch_create)     */
  int32_t no_graph;     /* batches: nonzero = launch kernels directly instead of
                           replaying a captured CUDA graph                        */
  int32_t data_region;  /* nonzero (CFGs with region): the single target data
                           region of Sec. IV-D and the directives (see
                           DATA REGION AND DIRECTIVES)                            */
  int32_t eager_to;     /* nonzero: eager `to' placement (see EAGER `TO')        */
} ompdart_opts;

/* EAGER `TO' (opts.eager_to; Sec. IV-E, Algorithm 1: a `target update to'
   follows the host write that produced the data, moved past the loops that
   sweep the array).  By default a `to' is lazy: right before the device
   read that finds the device copy stale, or hoisted onto a loop's entry
   edges.  The eager placement first computes AntDm, the variables that
   every path from a point reads on the device before any write of them
   (a path that leaves the function first does not count), and then makes
   the device copy valid on every edge p->b for AntDm_in[b] & Hp_out[p]
   (Hp: the host copy is the latest one with no transfer).  The `to' thus
   sits on the first edge after the producing write from which every path
   reads the data on the device: a write inside a host loop gets it on the
   loop's exit edges, a branch that reads nothing on the device gets none,
   and no path makes more `to's than the lazy placement.  These transfers
   are edge records (ompdart_edge_xfer.to_bits); a device read that still
   finds its copy stale keeps its access flag.  On the chunked scan solver
   (the default for reducible CFGs) every edge gets an edge constant:
   AntDm comes from a second backward walk (its complement is a may-problem
   shaped like liveness), and a back edge's constant is taken where the
   loop closes; path = 1 runs the sweep solver instead (any CFG, far
   slower).  A CFG with call pseudo-accesses is OMPDART_E_INVALID. */

typedef struct {
  int32_t edge, word;
  uint64_t to_bits, from_bits;
} ompdart_edge_xfer;

typedef struct {
  int32_t n_blocks, n_vars, n_words, n_edges, n_acc, n_exits;
  int32_t mem;                 /* OMPDART_MEM_HOST or OMPDART_MEM_DEVICE       */
  uint64_t *h_in, *d_in;       /* [n_blocks*n_words]                           */
  uint64_t *h_out, *d_out;     /* [n_blocks*n_words] or NULL                   */
  uint8_t *acc_flag;           /* [n_acc]                                      */
  int32_t n_edge_xfers;
  ompdart_edge_xfer *edge_xfers;
  int32_t *exit_blocks;        /* [n_exits]                                    */
  uint64_t *from_exit;         /* [n_exits*n_words]                            */
  int32_t path;                /* solver that ran: 1 sweep, 2 chunked scan      */
  int32_t sweeps;              /* device sweeps executed (diagnostic)           */
  int64_t h2d_bytes;           /* bytes the plan copied host->device            */
  int64_t d2h_bytes;           /* bytes copied device->host for this result     */
  uint64_t *live_in;           /* [n_blocks*n_words] or NULL (keep_states):
                                  variables the host or the device may read
                                  before they are written, from the block entry
                                  on (Sec. II-B); zero for unreachable blocks   */
  int32_t n_call_sites;        /* call pseudo-accesses (see CALLS)             */
  int32_t *call_site_acc;      /* [n_call_sites] access index of each          */
  uint64_t *call_to, *call_from;          /* [n_call_sites*n_words]            */
  uint64_t *call_entry_h, *call_entry_d;  /* [n_call_sites*n_words]            */
  uint64_t *call_exit_live;               /* [n_call_sites*n_words]            */
  /* data region and directives (opts.data_region with cfg.region, else
     NULL / 0; see DATA REGION AND DIRECTIVES) */
  uint8_t *in_region;          /* [n_blocks] inside the target data region   */
  uint64_t *map_to, *map_from, *map_alloc;  /* [n_words] map clauses        */
  int32_t n_kernels;           /* kernel ids 0 .. n_kernels-1                 */
  uint64_t *kernel_to;         /* [n_kernels*n_words] update to before kernel k */
  uint64_t *kernel_from;       /* [n_kernels*n_words] update from before kernel k */
  uint64_t *firstprivate;      /* [n_kernels*n_words] firstprivate on kernel k  */
  int32_t *acc_point;          /* [n_acc] insertion point of the transfer
                                  flagged at this access, or -1             */
  int32_t n_region_entries, n_region_exits;
  int32_t *region_entry_edges; /* [n_region_entries] edge ids into the region */
  int32_t *region_exit_edges;  /* [n_region_exits] edge ids out of it        */
  void *host_block;            /* library-internal: the host allocation that
                                  holds a host result's arrays (shared by the
                                  results of one batch arena); NULL in views  */
} ompdart_result;

typedef struct ompdart_plan ompdart_plan;

/* Ingest one CFG on the host (validation, predecessor lists, loop-ordered
   reverse post-order, dominators, natural loops, chunking) and upload it.
   Sec. IV-B (CFG, loops), Sec. IV-D (forward traversal). */
int ompdart_plan_create(const ompdart_cfg *cfg, const ompdart_opts *opts, ompdart_plan **plan);

/* Enqueue the whole analysis of a plan on `stream' (cudaStream_t, NULL =
   the plan's own stream).  Inputs and outputs stay on the device; returns
   after enqueueing.  Sec. IV-D and Algorithm 1. */
int ompdart_plan_run(ompdart_plan *plan, void *stream);

/* Wait for the plan's last run and report its device status
   (OMPDART_E_NOCONVERGE if a bounded loop ran out). */
int ompdart_plan_sync(ompdart_plan *plan);

/* Device-resident results of the last run (pointers owned by the plan,
   valid until the next run or destroy; mem = OMPDART_MEM_DEVICE). */
int ompdart_plan_view(ompdart_plan *plan, ompdart_result *view);

/* Copy the results of the plan's last run to host memory; *out is
   library-owned (ompdart_result_free), mem = OMPDART_MEM_HOST. */
int ompdart_plan_fetch(ompdart_plan *plan, ompdart_result **out);

/* Graph replay of a plan's runs (enable != 0): the next ompdart_plan_run
   captures the whole enqueue (every kernel, memset and the fork onto the
   plan's side streams) into a CUDA graph on its stream and launches it;
   later runs launch the same graph, on any stream, in one call.  A run
   whose ompdart_plan_sync had to grow a buffer (an overflowed transfer
   record stream) drops the graph and the next run captures it again.
   Profiling (ompdart_plan_profile) takes precedence: profiled runs are
   enqueued kernel by kernel.  enable = 0 waits for the last run and frees
   the graph. */
int ompdart_plan_graph(ompdart_plan *plan, int enable);

/* Number of kernel launches one ompdart_plan_run enqueues. */
int ompdart_plan_launches(const ompdart_plan *plan);

/* Per-kernel device time.  After ompdart_plan_profile(plan, 1), every run
   records a CUDA event on its stream before each kernel launch and after
   the last; ompdart_plan_sync charges the time between consecutive events
   to the kernel launched between them and accumulates it per kernel name.
   ompdart_plan_timings copies up to `max' entries (name strings owned by
   the plan) and sets *n to the number of distinct kernels.  Enabling or
   disabling resets the totals. */
typedef struct {
  const char *name;
  int32_t launches;
  double ms;
} ompdart_timing;
int ompdart_plan_profile(ompdart_plan *plan, int enable);
int ompdart_plan_timings(ompdart_plan *plan, ompdart_timing *out, int32_t max, int32_t *n);

void ompdart_plan_destroy(ompdart_plan *plan);

/* One call: plan, run, copy every output to host memory.  *out is
   library-owned (ompdart_result_free). */
int ompdart_analyze(const ompdart_cfg *cfg, const ompdart_opts *opts, ompdart_result **out);

void ompdart_result_free(ompdart_result *res);

/* Host results of at least 1 MiB live in memory kept for reuse once freed
   (up to OMPDART_HOST_CACHE_MB, default 4096 MiB, of cached blocks per
   kind): page-locked for a plan's result (ompdart_plan_fetch,
   ompdart_analyze), pageable for batch and serving results.  Releases
   every cached block; returns the bytes released. */
size_t ompdart_host_cache_trim(void);

/* Text of the calling thread's last error ("" if none). */
const char *ompdart_last_error(void);

/* ---- batches: many independent CFGs in one device run ------------------
   (no paper counterpart: the paper's tool analyses one translation unit at
   a time, Sec. V; a batch runs the same analysis for thousands of CFGs at
   once.)  The CFGs are grouped by word count W; every group becomes one
   arena: its CFGs laid end to end in one plan of the chunked scan solver
   (chunks never span two CFGs, each CFG starts from its own entry values
   and ends at its own region exit).  A CFG that solver cannot take
   (irreducible, or loop bodies not contiguous in loop order) gets a plan
   of its own with the general sweep solver.  A run is one CUDA graph: the
   arenas' kernel sequences are captured once on forked streams, so they
   overlap on the GPU, and every later run replays the graph.  The walk
   kernels of an arena are persistent: each warp takes (chunk, word group)
   items from a device work queue, longest chunks first. */
typedef struct ompdart_batch ompdart_batch;

/* Ingest n CFGs (host threads, one CFG per task) and upload the arenas.
   status[n] (may be NULL) receives each CFG's ingestion code; a CFG that
   fails (OMPDART_E_INVALID, ...) is left out and the rest proceed.  With
   opts->tune the autotuner times candidate (chunk_target, warps_per_cta)
   pairs on a sample of each arena and builds the arena with the fastest;
   choices are cached per (W, size class) for the life of the process.
   Returns OMPDART_OK unless the batch itself could not be built (n < 0,
   NULL pointers, allocation failure: OMPDART_E_NOMEM). */
int ompdart_batch_create(const ompdart_cfg *cfgs, int32_t n, const ompdart_opts *opts, ompdart_batch **batch,
                         int32_t *status);

/* Enqueue one run of every CFG of the batch on `stream' (cudaStream_t,
   NULL = the batch's own stream) and return. */
int ompdart_batch_run(ompdart_batch *batch, void *stream);

/* Wait for the last run.  status[n] (may be NULL): per CFG OMPDART_OK, its
   ingestion error, or OMPDART_E_NOCONVERGE.  Returns OMPDART_OK, or the
   error of the device run itself (OMPDART_E_CUDA, OMPDART_E_NOMEM). */
int ompdart_batch_sync(ompdart_batch *batch, int32_t *status);

/* Results of CFG i of the last run, as for ompdart_plan_view (device
   pointers into the batch's arenas, edge ids local to CFG i) and
   ompdart_plan_fetch (host copy, ompdart_result_free).  A CFG whose status
   is an error returns that error. */
int ompdart_batch_view(ompdart_batch *batch, int32_t i, ompdart_result *view);
int ompdart_batch_fetch(ompdart_batch *batch, int32_t i, ompdart_result **out);

/* Batch shape: number of arenas (each one device plan over many CFGs),
   number of CFGs on a plan of their own, kernel launches per run, and per
   arena its W, CFG count, chunk_target and warps_per_cta (arrays of at
   least max entries; NULL to skip). */
int ompdart_batch_info(const ompdart_batch *batch, int32_t *n_arenas, int32_t *n_solo, int32_t *launches,
                       int32_t max, int32_t *arena_w, int32_t *arena_cfgs, int32_t *arena_chunk,
                       int32_t *arena_wpc);

/* Per-kernel device time of a batch's runs, as ompdart_plan_profile /
   ompdart_plan_timings do for a plan: while profiling is on, a run
   launches every plan of the batch directly, one after another on the
   run's stream (no graph, no overlap between arenas), with a CUDA event
   before each kernel; ompdart_batch_sync charges the time between
   consecutive events to the kernel between them, summed per kernel name
   over all arenas.  Enabling or disabling resets the totals. */
int ompdart_batch_profile(ompdart_batch *batch, int enable);
int ompdart_batch_timings(ompdart_batch *batch, ompdart_timing *out, int32_t max, int32_t *n);

void ompdart_batch_destroy(ompdart_batch *batch);

/* One call: batch, run, copy every CFG's outputs to host memory.
   outs[n] receives library-owned results (NULL for a CFG whose status is
   an error); status[n] (may be NULL) as for ompdart_batch_sync.  Each
   result's h2d_bytes / d2h_bytes is its share (by blocks) of its arena's
   copies. */
int ompdart_analyze_batch(const ompdart_cfg *cfgs, int32_t n, const ompdart_opts *opts, ompdart_result **outs,
                          int32_t *status);

/* ---- interprocedural: callee summaries (Sec. IV-C) -----------------------
   The paper's side-effect analysis records, per function, which data it
   reads or writes on the host or the device and applies that at every call
   site.  A summary is 7 planes of the callee's W words, in the call-table
   row order: ReqH, ReqD (anticipated at the entry with nothing live after
   the exit: read in that space before being written, on some path), GenH,
   KillH, GenD, KillD (plain validity at the reachable exits, the local rule
   along paths without transfers: Gen = valid at every exit from an
   all-stale entry, Kill = stale at some exit from an all-valid entry),
   MustDef (written on every path to a reachable exit).  A callee without a
   reachable exit gets zero Gen/Kill/MustDef.  Callees may hold calls
   themselves (their own call tables); any CFG shape is accepted. */

/* Summaries of n callees in one device run: rows[i] receives 7 * W_i words
   in callee i's own numbering; status[i] (may be NULL) its code
   (OMPDART_E_INVALID for a malformed CFG, OMPDART_E_NOCONVERGE if
   opts->max_sweeps ran out).  Returns OMPDART_OK unless the run failed. */
int ompdart_summarize_batch(const ompdart_cfg *callees, int32_t n, const ompdart_opts *opts, uint64_t *const *rows,
                            int32_t *status);

/* One callee's summary mapped into a caller's numbering, ready to be a row
   of the caller's call table: var_map[v] (callee variable v) is the caller
   variable it denotes (a global, or the actual argument of a pointer
   parameter) or -1 (a local, dropped); NULL = identity.  caller_row
   receives 7 * ceil(caller_n_vars / 64) words.  Callee variables that
   denote the same caller variable combine into the tightest row that is
   sound for every callee with these per-variable summaries: Req, Kill,
   MustDef and Gen of any alias carry over, and a kill of one alias
   overrides a gen of another. */
int ompdart_summarize_callee(const ompdart_cfg *callee, const int32_t *var_map, int32_t caller_n_vars,
                             uint64_t *caller_row, const ompdart_opts *opts);

/* ---- interprocedural: a whole program ----------------------------------
   Functions and their call sites.  Function f's CFG holds its calls as
   call pseudo-accesses whose row index k (bits 0-30) names its k-th call
   site, site_off[f] + k; its call_planes are ignored (the driver fills the
   table from the callees' summaries).  Site s calls site_callee[s];
   var_map[map_off[s] ...] gives, per callee variable, the caller variable
   it denotes (a global, or the actual argument of a pointer parameter) or
   -1 (a local of the callee).  The call graph must be acyclic.
   ompdart_analyze_program
     1. computes the summaries bottom-up, one device run per call-DAG height
        (leaves first), each call site's row being its callee's summary
        mapped into the caller (as ompdart_summarize_callee);
     2. analyses every function top-down, one batch per height: a function
        nobody calls runs in its own boundary rows; a called function runs
        once per distinct context its call sites pass on: the caller's state
        at the call (call_entry_h / call_entry_d as the callee's entry rows,
        call_exit_live as its exit_host_live) mapped into the callee's
        numbering (a callee local starts valid on the host only and is dead
        after the exit).  A site passes on at most max_contexts contexts
        (0 = 4): sorted, the excess merged into the last by the meet
        (validity AND, liveness OR), which lies below every context it
        absorbs, so the merged instance's transfers serve each of them;
        a context whose meet would leave a variable valid nowhere that one
        of them holds somewhere (a host-only and a device-only copy) is not
        merged and runs as a context of its own. */
typedef struct {
  int32_t n_funcs;
  const ompdart_cfg *funcs;    /* [n_funcs]                                     */
  const int32_t *site_off;     /* [n_funcs+1]                                   */
  const int32_t *site_callee;  /* [n_sites]                                     */
  const int32_t *map_off;      /* [n_sites+1]                                   */
  const int32_t *var_map;      /* [map_off[n_sites]]                            */
  int32_t max_contexts;        /* per call site; 0 = 4                          */
} ompdart_program;

typedef struct {
  int32_t func;                /* the function analysed                          */
  int32_t status;              /* OMPDART_OK or why it has no (exact) result     */
  uint64_t *entry_h, *entry_d, *exit_live; /* [W_func] its context               */
  ompdart_result *result;      /* host result (NULL if the analysis failed)      */
} ompdart_instance;

typedef struct {
  int32_t n_instances;
  ompdart_instance *inst;      /* grouped by height, highest first               */
  int32_t levels;              /* call-DAG heights                                */
  int32_t *height;             /* [n_funcs]                                       */
  int32_t *status;             /* [n_funcs] summary status                        */
  uint64_t *summaries;         /* 7 * W_f words per function, in its numbering    */
  int64_t *summary_off;        /* [n_funcs]                                       */
} ompdart_program_result;

int ompdart_analyze_program(const ompdart_program *prog, const ompdart_opts *opts, ompdart_program_result **out);
void ompdart_program_result_free(ompdart_program_result *res);

/* ---- serving: continuous batching of analysis requests -----------------
   (no paper counterpart: the paper's tool runs once per translation unit;
   this is the request loop of a service that analyses CFGs as they
   arrive.)  A worker thread admits pending requests in arrival order into
   batches (ompdart_batch_*) while at most max_inflight batches are on the
   GPU and the estimated device bytes of all admitted work stay within
   hbm_budget_bytes; a batch is ingested and uploaded while earlier ones
   run and is launched on its own stream, so batches overlap on the device.
   When a batch finishes, its results are copied to the host, its device
   memory is released and the next pending requests are admitted.
   A serving batch runs once, so its kernels are launched directly (no
   graph capture).  max_batch = 1 is the plain form: one plan and one
   launch sequence per request.

   RESIDENT MODE (resident != 0): CFGs stay on the device between requests.
   `workers' threads take requests in arrival order, up to max_batch (16
   by default) at a time each.  A request's CFG is looked up by its content (graph, accesses,
   call table, kernels and scalars; not the entry and exit rows, which can
   differ per request) in a cache of device-resident plans: a hit uploads
   the request's entry and exit rows into the cached plan and runs it; a
   miss ingests the CFG into a new plan first (ompdart_plan_create) and
   keeps it.  A cached plan replays its run as one CUDA graph
   (ompdart_plan_graph).  Each request of a group runs on a stream of its
   own, so the group runs on the device together; the worker then waits
   for each in turn and copies its results back.  Runs of one cached plan
   are serialised; different plans run concurrently.  The plans' device bytes stay within hbm_budget_bytes:
   the least recently used idle plans are dropped to make room, and a
   request that still does not fit runs on a plan of its own that is
   freed afterwards.  max_batch is the group a worker launches at once
   (0 = 16, at most 256); max_inflight is not used. */
typedef struct ompdart_server ompdart_server;
typedef struct {
  int64_t hbm_budget_bytes; /* device bytes admitted work may hold; 0 = 40 GiB     */
  int32_t max_batch;        /* CFGs per batch; 0 = 4096 (resident: group, 0 = 16)  */
  int32_t max_inflight;     /* batches on the GPU at once; 0 = 2                    */
  int32_t device;           /* CUDA device ordinal                                  */
  int32_t keep_results;     /* nonzero: copy each result to the host for the waiter */
  ompdart_opts opts;        /* analysis options of every batch                      */
  int32_t resident;         /* nonzero: resident mode (see below)                   */
  int32_t workers;          /* resident mode: worker threads; 0 = 4                 */
} ompdart_server_opts;

typedef struct {
  int64_t submitted, completed, failed, batches;
  double mean_batch;               /* CFGs per batch                              */
  double p50_ms, p99_ms, max_ms;   /* latency: submission to result on the host   */
  int64_t peak_bytes, bytes_in_use; /* device bytes held by admitted batches       */
  int64_t cache_hits, cache_misses; /* resident mode: requests served by a cached
                                       plan / that had to build one              */
  int64_t cached_plans;            /* resident mode: plans held now                */
} ompdart_server_stats;

int ompdart_server_create(const ompdart_server_opts *opts, ompdart_server **server);

/* Queue one CFG (copied; the caller may reuse its buffers) and return its
   ticket at once.  Malformed CFGs are reported by the wait (status). */
int ompdart_server_submit(ompdart_server *server, const ompdart_cfg *cfg, int64_t *ticket);

/* Submit cfgs[i] at arrival_us[i] microseconds after the call (a load
   generator for capacity tests: sleeps and spins on the host clock); the
   tickets go to tickets[n].  Returns when the last one is submitted. */
int ompdart_server_replay(ompdart_server *server, const ompdart_cfg *cfgs, int32_t n, const double *arrival_us,
                          int64_t *tickets);

/* Wait up to timeout_ms (< 0: no limit) for a ticket: its status, its
   latency (submission to result on the host) and, if out is not NULL and
   keep_results was set, its result (caller-owned, ompdart_result_free).
   OMPDART_E_TIMEOUT if it is not done in time (the ticket stays valid);
   a collected ticket is forgotten.  For a failed request, the calling
   thread's ompdart_last_error() says why. */
int ompdart_server_wait(ompdart_server *server, int64_t ticket, int32_t timeout_ms, ompdart_result **out,
                        int32_t *status, double *latency_ms);

/* Wait until every submitted request is done (OMPDART_E_TIMEOUT after
   timeout_ms, < 0: no limit). */
int ompdart_server_drain(ompdart_server *server, int32_t timeout_ms);
int ompdart_server_get_stats(ompdart_server *server, ompdart_server_stats *out);

/* Finish every submitted request, then stop the worker and free all. */
void ompdart_server_destroy(ompdart_server *server);

/* Liveness of one CFG, allocating nothing (no paper counterpart: an
   addition for callers that cannot allocate device memory, for instance
   code running inside another runtime's memory pool, or that must not
   trigger the implicit synchronisation of cudaMalloc/cudaFree).
   Every argument is already in device memory, in the INPUT FORMAT above;
   exit_host_live may be NULL (all live).  On return live_in[n_blocks*W]
   holds, per block, the variables the host or the device may read before
   they are written from the block's entry on (the same plane as
   ompdart_result.live_in); unreachable blocks are zero.
   Limits: n_blocks <= 65536, n_vars <= 4096, accesses <= 2^20; larger
   inputs return OMPDART_E_BUDGET with a message, call pseudo-accesses
   OMPDART_E_INVALID.  The liveness sweeps visit the reachable blocks in
   breadth-first order from the entry, farthest first; a call that runs
   for more than 20 s of device time stops and returns OMPDART_E_TIMEOUT.
   Scratch: one static device array of 4.5 MiB per device, resident until
   the process exits; its device address is looked up
   (cudaGetSymbolAddress) on the first call on each device, which should
   come before any stream capture (a failed lookup is retried by the next
   call).  Calls share that array: calls that overlap on the GPU race and
   must be serialised by the caller.  The call enqueues on `stream'
   (cudaStream_t) and waits for that stream to finish before it returns. */
int ompdart_liveness_noalloc(int32_t n_blocks, int32_t n_vars, int32_t entry, const int32_t *succ_off,
                             const int32_t *succ, const int32_t *acc_off, const uint32_t *acc,
                             const uint64_t *exit_host_live, uint64_t *live_in, void *stream);

#ifdef __cplusplus
}
#endif
#endif
