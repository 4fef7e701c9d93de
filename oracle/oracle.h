/*
 * oracle.h -- CPU oracle for the OMPDart host/device validity data-flow.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link
 * or call this file: only tests/, the smoke check and the bench's CPU
 * baseline leg use it.  It shares no code, header or constant with the
 * CUDA library under paper_2406_13881_b300/; the only thing the two have
 * in common is the documented input format (CSR CFG + packed access
 * words), which both sides decode with their own code.
 *
 * Method (Marzen et al., "Static Generation of Efficient OpenMP Offload
 * Data Mappings", SC24):
 *   - validity of each variable in each memory space, tracked per CFG node
 *     (Sec. IV-D, definition of valid/stale);
 *   - only true (read-after-write) dependencies need a transfer (Sec. IV-D);
 *   - loops: a need inside a loop is satisfied before the loop when the data
 *     stays valid to the end of the body, else inside it (Sec. IV-D, loop
 *     paragraph; Algorithm 1's outward walk);
 *   - region-exit liveness decides the final `from' (Sec. IV-D, last
 *     paragraph; Sec. II-B liveness);
 *   - constructs are those of Table II (to / from / update).
 *
 * Every phase is a monotone bit-vector problem with a unique extremal fixed
 * point, solved here by a FIFO worklist over all reachable blocks.  All
 * planes are uint64 rows of W = ceil(n_vars/64) words, bit (v mod 64) of
 * word (v/64) for variable v; bits past n_vars are always 0.
 *
 * Parity: every function here is pinned by the -m "not gpu" tests (step
 * simulation of the local rule, brute-force meet-over-paths on acyclic
 * CFGs, the loop closed form, path simulation with version counters, the
 * paper's listings hand-translated to access form).
 */
#ifndef OMPDART_ORACLE_H
#define OMPDART_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define ORACLE_OK 0
#define ORACLE_E_INVALID (-1)
#define ORACLE_E_NOMEM (-2)

typedef struct {
  int32_t n_blocks, n_vars, entry;
  const int32_t *succ_off;  /* [n_blocks+1] */
  const int32_t *succ;      /* [n_edges]; edge id = position here */
  const int32_t *acc_off;   /* [n_blocks+1] */
  const uint32_t *acc;      /* packed: bits 0-23 var, 24-25 kind (1 R, 2 W,
                               3 RW), bit 26 space (0 host, 1 target),
                               bit 31 call (bits 0-30 = call table row) */
  const uint64_t *entry_host_valid; /* [W] or NULL = all valid   */
  const uint64_t *entry_dev_valid;  /* [W] or NULL = none valid  */
  const uint64_t *exit_host_live;   /* [W] or NULL = all live    */
  /* call table: row c holds 7 planes of W words in the caller's variable
     numbering, in the order ReqH, ReqD, GenH, KillH, GenD, KillD, MustDef
     (see oracle_summarize for their meaning).  May be NULL if no access
     has bit 31 set. */
  const uint64_t *call_planes;
  int32_t n_calls;
  /* kernels (Sec. IV-B offloaded nodes): region[b] = id of the offload
     kernel block b belongs to, or -1 for host code; NULL = no kernels. */
  const int32_t *region;
  /* nonzero: the single target data region of Sec. IV-D.  The region R is
     the set of blocks b with S dom b, E pdom b and b != E, where S is the
     nearest common dominator of the kernel blocks and the headers of every
     natural loop whose body holds a kernel block ("begin before any loop
     capturing the first kernel"), and E the nearest common post-dominator
     of the blocks those kernel blocks and loop bodies lead to outside
     themselves ("end after any loop capturing the last kernel";
     post-dominance towards one virtual exit fed by every block without
     successors; E is that virtual exit when there is no such block).  On every edge leaving R the
     host copy of each variable live at its target is made valid ("if
     stale data may be read on the host after exit from a target data
     region, the from map-type is included"). */
  int32_t data_region;
  /* nonzero: eager `to' placement (Sec. IV-E: a `target update to' follows
     the host write that produced the data, Algorithm 1 moving it past the
     loops that sweep the array).  Read here as the earliest point after
     the producing write from which EVERY path reads the variable on the
     device before any write of it: AntDm (device-read must-anticipation,
     ant_dm_in) holds there.  On every edge p->b the device copy is made
     valid for AntDm_in[b] & Hp_out[p] (the host copy is the only latest
     one), so a write inside a host loop gets its `to' on the loop's exit
     edges, and a branch that leads to no device read gets none.  The
     lazy rule (a `to' right before a device read that finds the device
     copy stale) covers what is left, e.g. data valid on the host at the
     function's entry. */
  int32_t eager_to;
} oracle_cfg;

/* Every pointer is caller-allocated; any may be NULL (then not written).
   N = n_blocks, E = n_edges, A = n_acc, W = words per plane. */
typedef struct {
  uint8_t *reachable;         /* [N] */
  uint8_t *is_header;         /* [N] natural-loop header */
  uint8_t *is_loop_entry;     /* [E] edge p->h, h header, p not in body(h) */
  uint64_t *gen_h, *kill_h, *gen_d, *kill_d, *ue_h, *ue_d, *def; /* [N*W] */
  uint64_t *ant_h_in, *ant_d_in, *live_in;       /* [N*W] */
  uint64_t *hp_in, *hp_out;                      /* [N*W] */
  uint64_t *mask_h, *mask_d;                     /* [N*W], rows of headers */
  uint64_t *d_in, *d_out, *hm, *h_in, *h_out;    /* [N*W] */
  uint64_t *to_edge, *from_edge;                 /* [E*W] */
  uint64_t *from_exit;                           /* [N*W], rows of exits */
  uint8_t *acc_flag;                             /* [A]: 0, 1 = to, 2 = from;
                                                    a call: 1 | 2 as needed */
  /* call sites, numbered by access index order (S = number of call
     accesses; rows of calls in unreachable blocks stay zero): */
  uint64_t *call_to, *call_from;                 /* [S*W] transfers right before the call */
  uint64_t *call_entry_h, *call_entry_d;         /* [S*W] validity the callee starts from */
  uint64_t *call_exit_live;                      /* [S*W] Live (AntH | AntD) right after it */
  /* data region (cfg->data_region with kernels; zero otherwise) */
  uint8_t *in_region;                            /* [N] block in R                   */
  uint8_t *region_exit;                          /* [E] edge from R to a block not in R */
  /* eager `to' (cfg->eager_to; zero otherwise) */
  uint64_t *ant_dm_in;                           /* [N*W] AntDm at block entry */
} oracle_out;

int oracle_solve(const oracle_cfg *cfg, oracle_out *out);

/* Side-effect summary of a callee (Sec. IV-C: per function, which data it
   reads or writes on the host or the device), in the callee's own variable
   numbering, written to planes[7*W] in the order
     ReqH    AntH at the entry with nothing live after the exit: read on the
             host before any write on some path;
     ReqD    the same on the device;
     GenH    valid on the host at every reachable exit whatever held at the
             entry (plain validity: the local rule along paths, no transfers);
     KillH   stale on the host at some reachable exit although valid
             everywhere at the entry;
     GenD, KillD  the same for the device;
     MustDef written on every path from the entry to a reachable exit.
   A callee with no reachable exit gets all-zero Gen/Kill/MustDef. */
int oracle_summarize(const oracle_cfg *callee, uint64_t *planes);


#ifdef __cplusplus
}
#endif
#endif
