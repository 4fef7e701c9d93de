// ingest.h -- host-side ingestion of one CFG (internal to libompdart).
//
// Turns the caller's CSR CFG into what the device solvers need:
//   * validation of the input format (ompdart.h);
//   * reachability, predecessor lists with edge ids;
//   * dominators (Lengauer-Tarjan) and natural loops (Sec. IV-B: loops are
//     recognised; Sec. IV-D: revisiting a node means a loop);
//   * a loop-ordered reverse post-order: every natural-loop body is a
//     contiguous run of positions starting at its header whenever the CFG
//     allows it (the DFS leaves loops before it enters their bodies);
//   * single-entry cut points of that order and the chunks built on them,
//     used by the chunked scan solver.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ompdart.h"

namespace ompdart {

struct Ingest {
  int N = 0, E = 0, A = 0, V = 0, W = 0, entry = 0;
  int M = 0;                        // reachable blocks
  std::vector<int32_t> order;       // [M] block at each position
  std::vector<int32_t> pos;         // [N] position of each block, -1 if unreachable
  // forward in-edges of each position (reachable sources only), CSR
  std::vector<int32_t> fin_off;     // [M+1]
  std::vector<int32_t> fin_src;     // source block
  std::vector<int32_t> fin_eid;     // edge id
  std::vector<int32_t> fin_ent;     // loop-entry edge index or -1
  // out-edges of each position (reachable targets are all reachable), CSR
  std::vector<int32_t> out_off;     // [M+1]
  std::vector<int32_t> out_dst;     // target block
  std::vector<uint8_t> is_exit;     // [M] no successor
  std::vector<int32_t> exit_blocks; // reachable blocks without successors, ascending id
  // natural loops (one per header), numbered by header position
  int L = 0;
  std::vector<int32_t> loop_head;   // [L] header block
  std::vector<int32_t> loop_parent; // [L] enclosing loop or -1
  std::vector<int32_t> loop_depth;  // [L] 1 = outermost
  std::vector<int32_t> body_off;    // [L+1]
  std::vector<int32_t> body_blk;    // blocks of each body, ascending position
  std::vector<int32_t> inner_loop;  // [N] innermost loop of each block or -1
  std::vector<int32_t> loop_end;    // [L] one past the last body position (contiguous order)
  // edges with constants: loop-entry edges p->h (h header, p outside
  // body(h)), reachable p only, then (region mode) the edges leaving the
  // data region that are not loop-entry edges (ent_loop -1)
  int K = 0;
  std::vector<int32_t> ent_loop, ent_src, ent_eid;
  std::vector<int32_t> ent_dst;     // [K] target block
  std::vector<uint8_t> ent_rx;      // [K] the edge leaves the data region
  // ---- the single target data region of each CFG (Sec. IV-D; region
  // mode only, see ingest()): per-CFG lists are concatenated for a batch
  bool region_mode = false;
  std::vector<uint8_t> in_region;   // [N] block in its CFG's region
  std::vector<int32_t> kernel;      // [N] kernel id (local to its CFG) or -1
  std::vector<int32_t> kern_off;    // [n_cfg+1] kernels of CFG c: kern_off[c] + local id
  std::vector<int32_t> rin_eid, rout_eid;  // edges entering / leaving a region (edge ids local to the CFG)
  std::vector<int32_t> rin_off, rout_off;  // [n_cfg+1]
  std::vector<int32_t> start_kernel;       // [n_cfg] local kernel id whose entry opens the region, or -1
  std::vector<uint8_t> entry_in_region;    // [n_cfg] the region starts at the CFG's entry
  bool reducible = true;            // every retreating edge is a back edge
  bool contiguous = true;           // every loop body is a run of positions
  // chunks of the order for the scan solver: chunk c = positions
  // [chunk_off[c], chunk_off[c+1]); each boundary is a single-entry cut
  std::vector<int32_t> chunk_off;
  int max_chunk = 0;
  // a batch of independent CFGs laid end to end: CFG k owns positions
  // [cfg_pos_off[k], cfg_pos_off[k+1]) (one CFG: {0, M}) and blocks
  // [cfg_blk_off[k], cfg_blk_off[k+1]) (one CFG: {0, N})
  std::vector<int32_t> cfg_pos_off;
  std::vector<int32_t> cfg_blk_off;
};

// Lay independent ingested CFGs end to end: block, position, loop and
// loop-entry ids are offset per part; edge ids (fin_eid) stay local to
// their part.  Every part must have been ingested on its own with the same
// W; edges never cross parts.
void concat_ingests(const std::vector<const Ingest *> &parts, Ingest *out);

// Returns OMPDART_OK or OMPDART_E_INVALID (message in *err).
// data_region (with cfg->region): also the single target data region of
// Sec. IV-D.  Its blocks are those b with S dom b, E pdom b and b != E:
// S is the nearest common dominator of the kernel blocks and of the
// headers of the natural loops whose body holds a kernel block, E the
// nearest common post-dominator (towards one virtual exit fed by every
// block without successors) of the blocks those kernel blocks and loop
// bodies lead to outside themselves, or the virtual exit if there is none.
// The edges leaving the region join the edge constants (ent_rx).
// all_edges: every reachable edge gets an edge-constant entry (eager `to'
// placement puts constants on any edge); the loop-entry ones come first.
int ingest(const ompdart_cfg *cfg, Ingest *g, std::string *err, bool data_region = false, bool all_edges = false);

// Build chunks of about `target` positions at single-entry cut points.
void make_chunks(Ingest *g, int target);

}  // namespace ompdart
