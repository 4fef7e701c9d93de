/*
 * oracle.c -- CPU oracle for the OMPDart validity data-flow (TEST
 * INFRASTRUCTURE ONLY; see oracle.h).  Plain, single-threaded C11: FIFO
 * worklists over explicit bit planes, no blocking, no reordering beyond the
 * phase order the method fixes.
 *
 * Phase order (each phase needs only earlier ones):
 *   1. local rule per block (Sec. IV-D: a write in one space makes the other
 *      stale; a read needs a valid copy; Sec. IV-B: R / W / RW / unknown=RW)
 *   2. backward anticipation AntH, AntD and Live = AntH | AntD (Sec. II-B
 *      liveness; Sec. IV-D region-exit liveness)
 *   3. plain host validity Hp, forward must (Sec. IV-D)
 *   4. loop masks: needed by a node of the loop and never made stale in
 *      the body (Sec. IV-D loop rule; Algorithm 1's outward walk)
 *   5. device validity D, forward must, with the masks as hoisted `to' on
 *      loop-entry edges (eager placement: the must-anticipation of device
 *      reads first, and its `to' on every edge)
 *   6. host validity H, forward must, hoisted `from' on loop-entry edges and
 *      a live join where neither space is valid resolved toward the host
 *   7. emission of the Table II transfers from the final states.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

/* ---- access word decoding (the documented input format) --------------- */
#define A_KIND_R 1
#define A_KIND_W 2
#define A_KIND_RW 3
#define SPACE_HOST 0
#define SPACE_DEV 1

static int a_var(uint32_t a) { return (int)(a & 0xFFFFFFu); }
static int a_kind(uint32_t a) { return (int)((a >> 24) & 3u); }
static int a_space(uint32_t a) { return (int)((a >> 26) & 1u); }
static int a_is_call(uint32_t a) { return (int)(a >> 31); }
static int a_call_row(uint32_t a) { return (int)(a & 0x7FFFFFFFu); }

/* ---- bit rows ---------------------------------------------------------- */
static int get_bit(const uint64_t *row, int v) { return (int)((row[v >> 6] >> (v & 63)) & 1u); }
static void set_bit(uint64_t *row, int v, int x) {
  uint64_t m = (uint64_t)1 << (v & 63);
  if (x) row[v >> 6] |= m; else row[v >> 6] &= ~m;
}

typedef struct {
  int N, E, A, W, V, entry;
  const int32_t *so, *s, *ao;
  const uint32_t *acc;
  int32_t *po, *ps, *pe;   /* predecessor CSR: source block, edge id */
  uint8_t *reach;
  uint64_t *top;           /* [W] all variables set */
} graph;

static void *xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }

/* ---- validation --------------------------------------------------------- */
static int validate(const oracle_cfg *c) {
  if (!c || c->n_blocks < 1 || c->n_vars < 1 || c->n_vars > (1 << 24)) return ORACLE_E_INVALID;
  if (c->entry < 0 || c->entry >= c->n_blocks) return ORACLE_E_INVALID;
  if (!c->succ_off || !c->acc_off) return ORACLE_E_INVALID;
  if (c->succ_off[0] != 0 || c->acc_off[0] != 0) return ORACLE_E_INVALID;
  for (int b = 0; b < c->n_blocks; ++b)
    if (c->succ_off[b + 1] < c->succ_off[b] || c->acc_off[b + 1] < c->acc_off[b]) return ORACLE_E_INVALID;
  int E = c->succ_off[c->n_blocks], A = c->acc_off[c->n_blocks];
  if ((E && !c->succ) || (A && !c->acc)) return ORACLE_E_INVALID;
  for (int e = 0; e < E; ++e) {
    if (c->succ[e] < 0 || c->succ[e] >= c->n_blocks) return ORACLE_E_INVALID;
    if (c->succ[e] == c->entry) return ORACLE_E_INVALID; /* entry has no predecessors */
  }
  for (int i = 0; i < A; ++i) {
    uint32_t a = c->acc[i];
    if (a_is_call(a)) {
      if (!c->call_planes || a_call_row(a) >= c->n_calls) return ORACLE_E_INVALID;
    } else {
      if ((a >> 27) & 0xFu) return ORACLE_E_INVALID;
      if (a_var(a) >= c->n_vars || a_kind(a) == 0) return ORACLE_E_INVALID;
    }
  }
  return ORACLE_OK;
}

/* ---- predecessors and reachability -------------------------------------- */
static int build_graph(const oracle_cfg *c, graph *g) {
  memset(g, 0, sizeof *g);
  g->N = c->n_blocks; g->V = c->n_vars; g->W = (c->n_vars + 63) / 64; g->entry = c->entry;
  g->so = c->succ_off; g->s = c->succ; g->ao = c->acc_off; g->acc = c->acc;
  g->E = c->succ_off[g->N]; g->A = c->acc_off[g->N];
  g->po = xcalloc((size_t)g->N + 1, sizeof(int32_t));
  g->ps = xcalloc((size_t)g->E, sizeof(int32_t));
  g->pe = xcalloc((size_t)g->E, sizeof(int32_t));
  g->reach = xcalloc((size_t)g->N, 1);
  g->top = xcalloc((size_t)g->W, sizeof(uint64_t));
  if (!g->po || !g->ps || !g->pe || !g->reach || !g->top) return ORACLE_E_NOMEM;
  for (int e = 0; e < g->E; ++e) g->po[g->s[e] + 1]++;
  for (int b = 0; b < g->N; ++b) g->po[b + 1] += g->po[b];
  int32_t *fill = xcalloc((size_t)g->N, sizeof(int32_t));
  if (!fill) return ORACLE_E_NOMEM;
  for (int b = 0; b < g->N; ++b)
    for (int e = g->so[b]; e < g->so[b + 1]; ++e) {
      int t = g->s[e], k = g->po[t] + fill[t]++;
      g->ps[k] = b; g->pe[k] = e;
    }
  free(fill);
  for (int v = 0; v < g->V; ++v) set_bit(g->top, v, 1);
  /* breadth-first reachability from the entry */
  int32_t *q = xcalloc((size_t)g->N, sizeof(int32_t));
  if (!q) return ORACLE_E_NOMEM;
  int qh = 0, qt = 0;
  q[qt++] = g->entry; g->reach[g->entry] = 1;
  while (qh < qt) {
    int b = q[qh++];
    for (int e = g->so[b]; e < g->so[b + 1]; ++e)
      if (!g->reach[g->s[e]]) { g->reach[g->s[e]] = 1; q[qt++] = g->s[e]; }
  }
  free(q);
  return ORACLE_OK;
}

static void free_graph(graph *g) {
  free(g->po); free(g->ps); free(g->pe); free(g->reach); free(g->top);
}

/* ---- step 1: local rule -------------------------------------------------
 * Per block and variable, scanning the accesses in order (RW = read then
 * write; a call row contributes its reads, then its net effect):
 *   events touching space S: an S-read, an S-write, a write in the other
 *   space.  GenS = last such event is an S-access; KillS = it is a write in
 *   the other space.  UES = the first event among {S-read, any write} is an
 *   S-read.  Def = some (must-)write.
 * Implemented as a tiny state machine per variable: last[S] in {0 none,
 * 1 S-access, 2 other-space write}; ue[S] in {0 undecided, 1 read first,
 * 2 write first}. */
typedef struct { uint8_t last[2], ue[2], def; } lstate;

static void ev_read(lstate *st, int S) {
  st->last[S] = 1;
  if (st->ue[S] == 0) st->ue[S] = 1;
}
static void ev_write(lstate *st, int S) {
  st->last[S] = 1;
  st->last[1 - S] = 2;
  if (st->ue[0] == 0) st->ue[0] = 2;
  if (st->ue[1] == 0) st->ue[1] = 2;
  st->def = 1;
}

/* planes of call row r, plane k (0 ReqH,1 ReqD,2 GenH,3 KillH,4 GenD,5 KillD,6 MustDef) */
static const uint64_t *call_plane(const oracle_cfg *c, int W, int r, int k) {
  return c->call_planes + ((size_t)r * 7 + (size_t)k) * (size_t)W;
}

static void local_rule(const oracle_cfg *c, const graph *g, uint64_t *GH, uint64_t *KH, uint64_t *GD,
                       uint64_t *KD, uint64_t *UH, uint64_t *UD, uint64_t *DF) {
  int W = g->W;
  lstate *st = xcalloc((size_t)g->V, sizeof(lstate));
  uint8_t *touched = xcalloc((size_t)g->V, 1);
  int32_t *list = xcalloc((size_t)g->V, sizeof(int32_t));
  for (int b = 0; b < g->N; ++b) {
    int nt = 0;
    for (int i = g->ao[b]; i < g->ao[b + 1]; ++i) {
      uint32_t a = g->acc[i];
      if (a_is_call(a)) {
        int r = a_call_row(a);
        for (int v = 0; v < g->V; ++v) {
          int rq_h = get_bit(call_plane(c, W, r, 0), v), rq_d = get_bit(call_plane(c, W, r, 1), v);
          int gh = get_bit(call_plane(c, W, r, 2), v), kh = get_bit(call_plane(c, W, r, 3), v);
          int gd = get_bit(call_plane(c, W, r, 4), v), kd = get_bit(call_plane(c, W, r, 5), v);
          int md = get_bit(call_plane(c, W, r, 6), v);
          if (!(rq_h | rq_d | gh | kh | gd | kd | md)) continue;
          if (!touched[v]) { touched[v] = 1; list[nt++] = v; memset(&st[v], 0, sizeof(lstate)); }
          lstate *s = &st[v];
          if (rq_h) ev_read(s, SPACE_HOST);
          if (rq_d) ev_read(s, SPACE_DEV);
          /* net effect on each space after the callee body */
          if (gh) s->last[SPACE_HOST] = 1; else if (kh) s->last[SPACE_HOST] = 2;
          if (gd) s->last[SPACE_DEV] = 1; else if (kd) s->last[SPACE_DEV] = 2;
          if (md) {
            s->def = 1;
            if (s->ue[0] == 0) s->ue[0] = 2;
            if (s->ue[1] == 0) s->ue[1] = 2;
          }
        }
        continue;
      }
      int v = a_var(a), k = a_kind(a), S = a_space(a);
      if (!touched[v]) { touched[v] = 1; list[nt++] = v; memset(&st[v], 0, sizeof(lstate)); }
      if (k & A_KIND_R) ev_read(&st[v], S);
      if (k & A_KIND_W) ev_write(&st[v], S);
    }
    size_t o = (size_t)b * W;
    for (int j = 0; j < nt; ++j) {
      int v = list[j];
      lstate *s = &st[v];
      if (GH) set_bit(GH + o, v, s->last[SPACE_HOST] == 1);
      if (KH) set_bit(KH + o, v, s->last[SPACE_HOST] == 2);
      if (GD) set_bit(GD + o, v, s->last[SPACE_DEV] == 1);
      if (KD) set_bit(KD + o, v, s->last[SPACE_DEV] == 2);
      if (UH) set_bit(UH + o, v, s->ue[SPACE_HOST] == 1);
      if (UD) set_bit(UD + o, v, s->ue[SPACE_DEV] == 1);
      if (DF) set_bit(DF + o, v, s->def);
      touched[v] = 0;
    }
  }
  free(st); free(touched); free(list);
}

/* ---- FIFO worklist ------------------------------------------------------ */
typedef struct { int32_t *q; uint8_t *in; int n, head, count; } wlist;
static int wl_init(wlist *w, int n) {
  w->q = xcalloc((size_t)n, sizeof(int32_t)); w->in = xcalloc((size_t)n, 1);
  w->n = n; w->head = 0; w->count = 0;
  return (w->q && w->in) ? ORACLE_OK : ORACLE_E_NOMEM;
}
static void wl_push(wlist *w, int b) {
  if (w->in[b]) return;
  w->in[b] = 1; w->q[(w->head + w->count) % w->n] = b; w->count++;
}
static int wl_pop(wlist *w) {
  int b = w->q[w->head]; w->head = (w->head + 1) % w->n; w->count--; w->in[b] = 0;
  return b;
}
static void wl_free(wlist *w) { free(w->q); free(w->in); }

/* ---- step 2: backward anticipation (least fixed point) ------------------
 * AntS_out[b] = OR over successors s of AntS_in[s]; a block with no
 * successor sees the region exit, where AntH = exit_host_live, AntD = 0.
 * AntS_in[b] = UES[b] | (AntS_out[b] & ~Def[b]).  Over reachable blocks. */
static int anticipation(const graph *g, const uint64_t *UES, const uint64_t *DF, const uint64_t *exit_live,
                        uint64_t *ant_in) {
  int W = g->W;
  wlist wl;
  if (wl_init(&wl, g->N)) return ORACLE_E_NOMEM;
  uint64_t *out = xcalloc((size_t)W, sizeof(uint64_t));
  memset(ant_in, 0, (size_t)g->N * W * sizeof(uint64_t));
  for (int b = g->N - 1; b >= 0; --b) if (g->reach[b]) wl_push(&wl, b);
  while (wl.count) {
    int b = wl_pop(&wl);
    if (g->so[b] == g->so[b + 1]) {
      for (int w = 0; w < W; ++w) out[w] = exit_live ? exit_live[w] : 0;
    } else {
      memset(out, 0, (size_t)W * sizeof(uint64_t));
      for (int e = g->so[b]; e < g->so[b + 1]; ++e)
        for (int w = 0; w < W; ++w) out[w] |= ant_in[(size_t)g->s[e] * W + w];
    }
    int changed = 0;
    for (int w = 0; w < W; ++w) {
      size_t o = (size_t)b * W + w;
      uint64_t nv = UES[o] | (out[w] & ~DF[o]);
      if (nv != ant_in[o]) { ant_in[o] = nv; changed = 1; }
    }
    if (changed)
      for (int k = g->po[b]; k < g->po[b + 1]; ++k)
        if (g->reach[g->ps[k]]) wl_push(&wl, g->ps[k]);
  }
  free(out); wl_free(&wl);
  return ORACLE_OK;
}

/* ---- eager `to': must-anticipation of a device read (Sec. IV-E) ----------
 * AntDm_in[b] = UED[b] | (AntDm_out[b] & ~Def[b]); AntDm_out[b] = AND over
 * successors s of AntDm_in[s]; a block without successors: nothing (a path
 * that leaves the function first does not read the copy).  Greatest fixed
 * point over reachable blocks: v is in AntDm at a point when every path
 * from there reads v on the device before any write of v. */
static int must_anticipation(const graph *g, const uint64_t *UES, const uint64_t *DF, uint64_t *am_in) {
  int W = g->W;
  wlist wl;
  if (wl_init(&wl, g->N)) return ORACLE_E_NOMEM;
  uint64_t *out = xcalloc((size_t)W, sizeof(uint64_t));
  if (!out) { wl_free(&wl); return ORACLE_E_NOMEM; }
  for (int b = 0; b < g->N; ++b)
    for (int w = 0; w < W; ++w) am_in[(size_t)b * W + w] = g->reach[b] ? g->top[w] : 0;
  for (int b = g->N - 1; b >= 0; --b) if (g->reach[b]) wl_push(&wl, b);
  while (wl.count) {
    int b = wl_pop(&wl);
    if (g->so[b] == g->so[b + 1]) {
      memset(out, 0, (size_t)W * sizeof(uint64_t));
    } else {
      for (int w = 0; w < W; ++w) out[w] = g->top[w];
      for (int e = g->so[b]; e < g->so[b + 1]; ++e)
        for (int w = 0; w < W; ++w) out[w] &= am_in[(size_t)g->s[e] * W + w];
    }
    int changed = 0;
    for (int w = 0; w < W; ++w) {
      size_t o = (size_t)b * W + w;
      uint64_t nv = UES[o] | (out[w] & ~DF[o]);
      if (nv != am_in[o]) { am_in[o] = nv; changed = 1; }
    }
    if (changed)
      for (int k = g->po[b]; k < g->po[b + 1]; ++k)
        if (g->reach[g->ps[k]]) wl_push(&wl, g->ps[k]);
  }
  free(out); wl_free(&wl);
  return ORACLE_OK;
}

/* ---- steps 3, 5, 6: forward must problems (greatest fixed point) --------
 * x_in[entry] = init; x_in[b] = AND over reachable predecessors p of
 *   (x_out[p] | edge_gen(p->b)); then x_in[b] |= node_gen[b] (H only);
 * x_out[b] = Gen[b] | (x_in[b] & ~Kill[b]).  Unreachable blocks stay at
 * the top element and never enter a meet. */
typedef struct {
  const uint64_t *gen, *kill, *init;       /* init [W]                      */
  const uint8_t *is_entry_edge;            /* [E] loop-entry edge flags      */
  const uint64_t *edge_mask;               /* [N*W] mask row of the header   */
  const uint64_t *edge_src;                /* [N*W] source-valid test of p   */
  const uint64_t *node_gen;                /* [N*W] or NULL                  */
  uint64_t *x_in, *x_out, *x_meet;         /* x_meet may be NULL             */
  const uint8_t *is_exit_edge;             /* [E] edges leaving the data region, or NULL */
  const uint64_t *exit_gen;                /* [N*W] added along such an edge p->b: row b */
  const uint64_t *any_mask, *any_src;      /* [N*W] or NULL: added along every edge
                                              p->b: any_mask row b & any_src row p */
} fwd_problem;

static int forward_must(const graph *g, fwd_problem *P) {
  int W = g->W;
  wlist wl;
  if (wl_init(&wl, g->N)) return ORACLE_E_NOMEM;
  uint64_t *m = xcalloc((size_t)W, sizeof(uint64_t));
  for (int b = 0; b < g->N; ++b)
    for (int w = 0; w < W; ++w) {
      P->x_in[(size_t)b * W + w] = g->top[w];
      P->x_out[(size_t)b * W + w] = g->top[w];
      if (P->x_meet) P->x_meet[(size_t)b * W + w] = g->top[w];
    }
  for (int b = 0; b < g->N; ++b) if (g->reach[b]) wl_push(&wl, b);
  while (wl.count) {
    int b = wl_pop(&wl);
    if (b == g->entry) {
      for (int w = 0; w < W; ++w) m[w] = P->init ? P->init[w] : g->top[w];
    } else {
      for (int w = 0; w < W; ++w) m[w] = g->top[w];
      for (int k = g->po[b]; k < g->po[b + 1]; ++k) {
        int p = g->ps[k];
        if (!g->reach[p]) continue;
        int e = g->pe[k];
        for (int w = 0; w < W; ++w) {
          uint64_t ev = P->x_out[(size_t)p * W + w];
          if (P->is_entry_edge && P->is_entry_edge[e])
            ev |= P->edge_mask[(size_t)b * W + w] & P->edge_src[(size_t)p * W + w];
          if (P->is_exit_edge && P->is_exit_edge[e]) ev |= P->exit_gen[(size_t)b * W + w];
          if (P->any_mask) ev |= P->any_mask[(size_t)b * W + w] & P->any_src[(size_t)p * W + w];
          m[w] &= ev;
        }
      }
    }
    int changed = 0;
    for (int w = 0; w < W; ++w) {
      size_t o = (size_t)b * W + w;
      if (P->x_meet) P->x_meet[o] = m[w];
      uint64_t in = m[w] | (P->node_gen ? P->node_gen[o] : 0);
      P->x_in[o] = in;
      uint64_t nv = P->gen[o] | (in & ~P->kill[o]);
      if (nv != P->x_out[o]) { P->x_out[o] = nv; changed = 1; }
    }
    if (changed)
      for (int e = g->so[b]; e < g->so[b + 1]; ++e) wl_push(&wl, g->s[e]);
  }
  free(m); wl_free(&wl);
  return ORACLE_OK;
}

/* ---- dominators (Cooper, Harvey and Kennedy's iterative algorithm) ------- */
static int dominators(const graph *g, int32_t *idom, int32_t *rpo_num) {
  int N = g->N;
  int32_t *order = xcalloc((size_t)N, sizeof(int32_t));
  int32_t *stk = xcalloc((size_t)N, sizeof(int32_t));
  int32_t *it = xcalloc((size_t)N, sizeof(int32_t));
  uint8_t *seen = xcalloc((size_t)N, 1);
  if (!order || !stk || !it || !seen) return ORACLE_E_NOMEM;
  /* iterative depth-first search, post-order numbering */
  int sp = 0, npost = 0;
  stk[sp++] = g->entry; seen[g->entry] = 1; it[g->entry] = g->so[g->entry];
  while (sp) {
    int b = stk[sp - 1];
    if (it[b] < g->so[b + 1]) {
      int t = g->s[it[b]++];
      if (!seen[t]) { seen[t] = 1; it[t] = g->so[t]; stk[sp++] = t; }
    } else {
      order[npost++] = b; --sp;
    }
  }
  for (int b = 0; b < N; ++b) rpo_num[b] = -1;
  for (int i = 0; i < npost; ++i) rpo_num[order[i]] = npost - 1 - i;
  int32_t *rpo = stk;  /* reuse */
  for (int i = 0; i < npost; ++i) rpo[npost - 1 - i] = order[i];
  for (int b = 0; b < N; ++b) idom[b] = -1;
  idom[g->entry] = g->entry;
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int i = 1; i < npost; ++i) {
      int b = rpo[i], nd = -1;
      for (int k = g->po[b]; k < g->po[b + 1]; ++k) {
        int p = g->ps[k];
        if (!g->reach[p] || idom[p] < 0) continue;
        if (nd < 0) { nd = p; continue; }
        int f1 = p, f2 = nd;  /* intersect along the dominator tree */
        while (f1 != f2) {
          while (rpo_num[f1] > rpo_num[f2]) f1 = idom[f1];
          while (rpo_num[f2] > rpo_num[f1]) f2 = idom[f2];
        }
        nd = f1;
      }
      if (nd >= 0 && idom[b] != nd) { idom[b] = nd; changed = 1; }
    }
  }
  free(order); free(stk); free(it); free(seen);
  return ORACLE_OK;
}

/* Dominator-tree interval numbering: a dom b  iff  pre[a] <= pre[b] and
   post[b] <= post[a]. */
static int dom_intervals(const graph *g, const int32_t *idom, int32_t *pre, int32_t *post) {
  int N = g->N;
  int32_t *co = xcalloc((size_t)N + 1, sizeof(int32_t));
  int32_t *ch = xcalloc((size_t)N, sizeof(int32_t));
  int32_t *fill = xcalloc((size_t)N, sizeof(int32_t));
  int32_t *stk = xcalloc((size_t)N, sizeof(int32_t));
  int32_t *it = xcalloc((size_t)N, sizeof(int32_t));
  if (!co || !ch || !fill || !stk || !it) return ORACLE_E_NOMEM;
  for (int b = 0; b < N; ++b)
    if (g->reach[b] && b != g->entry) co[idom[b] + 1]++;
  for (int b = 0; b < N; ++b) co[b + 1] += co[b];
  for (int b = 0; b < N; ++b)
    if (g->reach[b] && b != g->entry) ch[co[idom[b]] + fill[idom[b]]++] = b;
  int sp = 0, clock = 0;
  stk[sp++] = g->entry; it[g->entry] = co[g->entry]; pre[g->entry] = clock++;
  while (sp) {
    int b = stk[sp - 1];
    if (it[b] < co[b + 1]) {
      int c = ch[it[b]++];
      pre[c] = clock++; it[c] = co[c]; stk[sp++] = c;
    } else {
      post[b] = clock++; --sp;
    }
  }
  free(co); free(ch); free(fill); free(stk); free(it);
  return ORACLE_OK;
}

/* ---- natural loops and loop masks -----------------------------------------
 * Back edge t->h: both reachable and h dominates t.  body(h) = {h} plus
 * every reachable block that reaches a latch of h without passing through
 * h.  Entry edges of h: p->h with p outside body(h).
 * For every header and space S:
 *   LantS[h] = variables that some node of the loop reads in S before any
 *              write, on a path from h that stays inside body(h) within one
 *              iteration (least fixed point of the anticipation equations
 *              restricted to body(h), edges back into h and edges leaving
 *              the body dropped) -- "a node that is part of a loop needs
 *              the data";
 *   KOS[h]   = OR over body(h) of KillS -- the loop makes S stale somewhere;
 *   MaskS[h] = LantS[h] & ~KOS[h] -- the need can be met before the loop. */
static int natural_loops(const graph *g, const uint64_t *KH, const uint64_t *KD, const uint64_t *UH,
                         const uint64_t *UD, const uint64_t *DF, uint8_t *is_header, uint8_t *is_entry_edge,
                         uint64_t *MH, uint64_t *MD) {
  int N = g->N, W = g->W, rc;
  int32_t *idom = xcalloc((size_t)N, sizeof(int32_t));
  int32_t *rpo_num = xcalloc((size_t)N, sizeof(int32_t));
  int32_t *pre = xcalloc((size_t)N, sizeof(int32_t));
  int32_t *post = xcalloc((size_t)N, sizeof(int32_t));
  int32_t *stamp = xcalloc((size_t)N, sizeof(int32_t));
  int32_t *stk = xcalloc((size_t)N, sizeof(int32_t));
  int32_t *body = xcalloc((size_t)N, sizeof(int32_t));
  uint64_t *LH = xcalloc((size_t)N * W, sizeof(uint64_t)), *LD = xcalloc((size_t)N * W, sizeof(uint64_t));
  uint64_t *koh = xcalloc((size_t)W, sizeof(uint64_t)), *kod = xcalloc((size_t)W, sizeof(uint64_t));
  uint64_t *oh = xcalloc((size_t)W, sizeof(uint64_t)), *od = xcalloc((size_t)W, sizeof(uint64_t));
  wlist wl;
  if (!idom || !rpo_num || !pre || !post || !stamp || !stk || !body || !LH || !LD || !koh || !kod || !oh ||
      !od || wl_init(&wl, N))
    return ORACLE_E_NOMEM;
  if ((rc = dominators(g, idom, rpo_num))) return rc;
  if ((rc = dom_intervals(g, idom, pre, post))) return rc;
  for (int b = 0; b < N; ++b) stamp[b] = -1;
  for (int b = 0; b < N; ++b) is_header[b] = 0;
  for (int e = 0; e < g->E; ++e) is_entry_edge[e] = 0;
  for (int h = 0; h < N; ++h) {
    if (!g->reach[h]) continue;
    int sp = 0, nb = 0;
    for (int k = g->po[h]; k < g->po[h + 1]; ++k) {
      int t = g->ps[k];
      if (!g->reach[t]) continue;
      int dom = pre[h] <= pre[t] && post[t] <= post[h];
      if (!dom) continue;
      is_header[h] = 1;
      if (t != h && stamp[t] != h) { stamp[t] = h; stk[sp++] = t; }
    }
    if (!is_header[h]) continue;
    stamp[h] = h;
    body[nb++] = h;
    /* collect the body by a backward walk from the latches */
    while (sp) {
      int b = stk[--sp];
      body[nb++] = b;
      for (int k = g->po[b]; k < g->po[b + 1]; ++k) {
        int p = g->ps[k];
        if (g->reach[p] && stamp[p] != h) { stamp[p] = h; stk[sp++] = p; }
      }
    }
    for (int k = g->po[h]; k < g->po[h + 1]; ++k)
      if (stamp[g->ps[k]] != h) is_entry_edge[g->pe[k]] = 1;
    /* kills anywhere in the body */
    memset(koh, 0, (size_t)W * sizeof(uint64_t));
    memset(kod, 0, (size_t)W * sizeof(uint64_t));
    for (int i = 0; i < nb; ++i)
      for (int w = 0; w < W; ++w) {
        koh[w] |= KH[(size_t)body[i] * W + w];
        kod[w] |= KD[(size_t)body[i] * W + w];
      }
    /* anticipation restricted to the body, one iteration from h */
    for (int i = 0; i < nb; ++i) {
      memset(LH + (size_t)body[i] * W, 0, (size_t)W * sizeof(uint64_t));
      memset(LD + (size_t)body[i] * W, 0, (size_t)W * sizeof(uint64_t));
      wl_push(&wl, body[i]);
    }
    while (wl.count) {
      int b = wl_pop(&wl);
      memset(oh, 0, (size_t)W * sizeof(uint64_t));
      memset(od, 0, (size_t)W * sizeof(uint64_t));
      for (int e = g->so[b]; e < g->so[b + 1]; ++e) {
        int s = g->s[e];
        if (s == h || stamp[s] != h) continue;
        for (int w = 0; w < W; ++w) {
          oh[w] |= LH[(size_t)s * W + w];
          od[w] |= LD[(size_t)s * W + w];
        }
      }
      int changed = 0;
      for (int w = 0; w < W; ++w) {
        size_t o = (size_t)b * W + w;
        uint64_t nh = UH[o] | (oh[w] & ~DF[o]), nd = UD[o] | (od[w] & ~DF[o]);
        if (nh != LH[o] || nd != LD[o]) { LH[o] = nh; LD[o] = nd; changed = 1; }
      }
      if (changed && b != h)
        for (int k = g->po[b]; k < g->po[b + 1]; ++k)
          if (stamp[g->ps[k]] == h) wl_push(&wl, g->ps[k]);
    }
    for (int w = 0; w < W; ++w) {
      size_t o = (size_t)h * W + w;
      MH[o] = LH[o] & ~koh[w];
      MD[o] = LD[o] & ~kod[w];
    }
  }
  free(idom); free(rpo_num); free(pre); free(post); free(stamp); free(stk); free(body);
  free(LH); free(LD); free(koh); free(kod); free(oh); free(od); wl_free(&wl);
  return ORACLE_OK;
}

/* ---- the single target data region (Sec. IV-D) ---------------------------
 * Post-dominators: Cooper, Harvey and Kennedy's iterative algorithm on the
 * reversed graph, rooted at a virtual exit (node N) whose reversed edges
 * lead to every reachable block without successors.  Blocks that reach no
 * exit get no post-dominator (-1). */
static int post_dominators(const graph *g, int32_t *ipdom, int32_t *prpo) {
  int N = g->N, X = N;  /* X: the virtual exit */
  int32_t *order = xcalloc((size_t)N + 1, sizeof(int32_t));
  int32_t *stk = xcalloc((size_t)N + 1, sizeof(int32_t));
  int32_t *it = xcalloc((size_t)N + 1, sizeof(int32_t));
  uint8_t *seen = xcalloc((size_t)N + 1, 1);
  int32_t *xs = xcalloc((size_t)N + 1, sizeof(int32_t));  /* exit blocks */
  if (!order || !stk || !it || !seen || !xs) return ORACLE_E_NOMEM;
  int nx = 0;
  for (int b = 0; b < N; ++b)
    if (g->reach[b] && g->so[b] == g->so[b + 1]) xs[nx++] = b;
  /* depth-first search over reversed edges from X: X's successors are the
     exit blocks, a block's successors are its reachable predecessors */
  int sp = 0, npost = 0;
  stk[sp++] = X; seen[X] = 1; it[X] = 0;
  while (sp) {
    int b = stk[sp - 1], nxt = -1;
    if (b == X) {
      if (it[X] < nx) nxt = xs[it[X]++];
    } else {
      while (it[b] < g->po[b + 1] - g->po[b]) {
        int p = g->ps[g->po[b] + it[b]++];
        if (g->reach[p]) { nxt = p; break; }
      }
    }
    if (nxt >= 0) {
      if (!seen[nxt]) { seen[nxt] = 1; it[nxt] = 0; stk[sp++] = nxt; }
    } else {
      order[npost++] = b; --sp;
    }
  }
  for (int b = 0; b <= N; ++b) { prpo[b] = -1; ipdom[b] = -1; }
  for (int i = 0; i < npost; ++i) prpo[order[i]] = npost - 1 - i;
  int32_t *rpo = stk;
  for (int i = 0; i < npost; ++i) rpo[npost - 1 - i] = order[i];
  ipdom[X] = X;
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int i = 1; i < npost; ++i) {
      int b = rpo[i], nd = -1;
      /* reversed predecessors of b = its successors, or X for an exit block */
      int ns = g->so[b + 1] - g->so[b];
      for (int k = 0; k < (ns ? ns : 1); ++k) {
        int q = ns ? g->s[g->so[b] + k] : X;
        if (ipdom[q] < 0) continue;
        if (nd < 0) { nd = q; continue; }
        int f1 = q, f2 = nd;
        while (f1 != f2) {
          while (prpo[f1] > prpo[f2]) f1 = ipdom[f1];
          while (prpo[f2] > prpo[f1]) f2 = ipdom[f2];
        }
        nd = f1;
      }
      if (nd >= 0 && ipdom[b] != nd) { ipdom[b] = nd; changed = 1; }
    }
  }
  free(order); free(stk); free(it); free(seen); free(xs);
  return ORACLE_OK;
}

/* Interval numbering of a tree given by parent[] over nodes [0, n) with
   `root' (nodes with parent < 0 other than the root are left out):
   a is an ancestor-or-self of b iff pre[a] <= pre[b] and post[b] <= post[a]. */
static int tree_intervals(int n, const int32_t *parent, int root, int32_t *pre, int32_t *post) {
  int32_t *co = xcalloc((size_t)n + 1, sizeof(int32_t));
  int32_t *ch = xcalloc((size_t)n, sizeof(int32_t));
  int32_t *fill = xcalloc((size_t)n, sizeof(int32_t));
  int32_t *stk = xcalloc((size_t)n, sizeof(int32_t));
  int32_t *it = xcalloc((size_t)n, sizeof(int32_t));
  if (!co || !ch || !fill || !stk || !it) return ORACLE_E_NOMEM;
  for (int b = 0; b < n; ++b) { pre[b] = -1; post[b] = -1; }
  for (int b = 0; b < n; ++b)
    if (b != root && parent[b] >= 0) co[parent[b] + 1]++;
  for (int b = 0; b < n; ++b) co[b + 1] += co[b];
  for (int b = 0; b < n; ++b)
    if (b != root && parent[b] >= 0) ch[co[parent[b]] + fill[parent[b]]++] = b;
  int sp = 0, clock = 0;
  stk[sp++] = root; it[root] = co[root]; pre[root] = clock++;
  while (sp) {
    int b = stk[sp - 1];
    if (it[b] < co[b + 1]) {
      int c = ch[it[b]++];
      pre[c] = clock++; it[c] = co[c]; stk[sp++] = c;
    } else {
      post[b] = clock++; --sp;
    }
  }
  free(co); free(ch); free(fill); free(stk); free(it);
  return ORACLE_OK;
}

/* nearest common ancestor of a and b in a tree with CHK numbering */
static int tree_meet(int a, int b, const int32_t *parent, const int32_t *num) {
  while (a != b) {
    while (num[a] > num[b]) a = parent[a];
    while (num[b] > num[a]) b = parent[b];
  }
  return a;
}

/* R (see oracle_cfg.data_region) into in_r[N]; its exit edges into
   exit_e[E].  Nothing when no reachable block belongs to a kernel. */
static int data_region(const oracle_cfg *c, const graph *g, uint8_t *in_r, uint8_t *exit_e) {
  int N = g->N, rc;
  memset(in_r, 0, (size_t)N);
  memset(exit_e, 0, (size_t)g->E);
  int32_t *idom = xcalloc((size_t)N, sizeof(int32_t)), *num = xcalloc((size_t)N, sizeof(int32_t));
  int32_t *pre = xcalloc((size_t)N, sizeof(int32_t)), *post = xcalloc((size_t)N, sizeof(int32_t));
  int32_t *ipd = xcalloc((size_t)N + 1, sizeof(int32_t)), *pnum = xcalloc((size_t)N + 1, sizeof(int32_t));
  int32_t *ppre = xcalloc((size_t)N + 1, sizeof(int32_t)), *ppost = xcalloc((size_t)N + 1, sizeof(int32_t));
  int32_t *stamp = xcalloc((size_t)N, sizeof(int32_t)), *stk = xcalloc((size_t)N, sizeof(int32_t));
  int32_t *body = xcalloc((size_t)N, sizeof(int32_t));
  uint8_t *cap = xcalloc((size_t)N, 1);  /* block in a loop body that holds a kernel block, or a kernel block */
  uint8_t *hcap = xcalloc((size_t)N, 1); /* header of such a loop */
  if (!idom || !num || !pre || !post || !ipd || !pnum || !ppre || !ppost || !stamp || !stk || !body || !cap ||
      !hcap)
    return ORACLE_E_NOMEM;
  int nk = 0;
  for (int b = 0; b < N; ++b)
    if (g->reach[b] && c->region[b] >= 0) { cap[b] = 1; ++nk; }
  if (!nk) goto out;
  if ((rc = dominators(g, idom, num))) return rc;
  if ((rc = dom_intervals(g, idom, pre, post))) return rc;
  if ((rc = post_dominators(g, ipd, pnum))) return rc;
  if ((rc = tree_intervals(N + 1, ipd, N, ppre, ppost))) return rc;
  /* natural loops whose body holds a kernel block: their headers and bodies */
  for (int b = 0; b < N; ++b) stamp[b] = -1;
  for (int h = 0; h < N; ++h) {
    if (!g->reach[h]) continue;
    int sp = 0, nb = 0, is_h = 0;
    for (int k = g->po[h]; k < g->po[h + 1]; ++k) {
      int t = g->ps[k];
      if (!g->reach[t] || !(pre[h] <= pre[t] && post[t] <= post[h])) continue;
      is_h = 1;
      if (t != h && stamp[t] != h) { stamp[t] = h; stk[sp++] = t; }
    }
    if (!is_h) continue;
    stamp[h] = h;
    body[nb++] = h;
    while (sp) {
      int b = stk[--sp];
      body[nb++] = b;
      for (int k = g->po[b]; k < g->po[b + 1]; ++k) {
        int p = g->ps[k];
        if (g->reach[p] && stamp[p] != h) { stamp[p] = h; stk[sp++] = p; }
      }
    }
    int holds = 0;
    for (int i = 0; i < nb; ++i) holds |= c->region[body[i]] >= 0;
    if (!holds) continue;
    hcap[h] = 1;
    for (int i = 0; i < nb; ++i) cap[body[i]] = 2 | (cap[body[i]] & 1);
  }
  /* S: nearest common dominator of the kernel blocks and the capturing
     headers (the region begins at S); E: nearest common post-dominator of
     the blocks that the kernel blocks and the capturing bodies lead to
     outside themselves (the region ends where E begins; the virtual exit
     if there is none, or one of them reaches no exit) */
  int S = -1, E = -1;
  for (int b = 0; b < N; ++b) {
    if ((cap[b] & 1) || hcap[b]) S = S < 0 ? b : tree_meet(S, b, idom, num);
    if (!cap[b]) continue;
    for (int e = g->so[b]; e < g->so[b + 1]; ++e) {
      int t = g->s[e];
      if (cap[t]) continue;
      if (ipd[t] < 0) E = N;
      else if (E != N) E = E < 0 ? t : tree_meet(E, t, ipd, pnum);
    }
  }
  if (E < 0) E = N;
  for (int b = 0; b < N; ++b) {
    if (!g->reach[b] || b == E) continue;
    int sdom = pre[S] <= pre[b] && post[b] <= post[S];
    int epdom = E == N || (ppre[b] >= 0 && ppre[E] <= ppre[b] && ppost[b] <= ppost[E]);
    in_r[b] = (uint8_t)(sdom && epdom);
  }
  for (int b = 0; b < N; ++b)
    for (int e = g->so[b]; e < g->so[b + 1]; ++e)
      exit_e[e] = (uint8_t)(g->reach[b] && in_r[b] && !in_r[g->s[e]]);
out:
  free(idom); free(num); free(pre); free(post); free(ipd); free(pnum); free(ppre); free(ppost);
  free(stamp); free(stk); free(body); free(cap); free(hcap);
  return ORACLE_OK;
}

/* ---- step 7: access flags --------------------------------------------------
 * Replay each reachable block from (H_in, D_in): an S-read that finds S
 * stale gets a transfer right before it (`to' for a device read, `from'
 * for a host read), after which S is valid; an S-write makes S valid and
 * the other space stale.  This covers both the transfers at the top of the
 * block (upward-exposed reads) and those after a write in the other space
 * inside the block. */
/* call-site rows: site k = the k-th call access in access order */
typedef struct { uint64_t *to, *from, *entry_h, *entry_d, *exit_live; } call_rows;

static void access_flags(const oracle_cfg *c, const graph *g, const uint64_t *h_in, const uint64_t *d_in,
                         uint8_t *flag, const int32_t *site_of, call_rows *cr) {
  int W = g->W;
  uint64_t *h = xcalloc((size_t)W, sizeof(uint64_t)), *d = xcalloc((size_t)W, sizeof(uint64_t));
  memset(flag, 0, (size_t)g->A);
  for (int b = 0; b < g->N; ++b) {
    if (!g->reach[b]) continue;
    memcpy(h, h_in + (size_t)b * W, (size_t)W * sizeof(uint64_t));
    memcpy(d, d_in + (size_t)b * W, (size_t)W * sizeof(uint64_t));
    for (int i = g->ao[b]; i < g->ao[b + 1]; ++i) {
      uint32_t a = g->acc[i];
      if (a_is_call(a)) {
        /* the callee's requirements are met right before the call (`from'
           for ReqH stale on the host, `to' for ReqD stale on the device),
           then its net effect applies */
        int r = a_call_row(a);
        size_t o = (size_t)site_of[i] * W;
        for (int w = 0; w < W; ++w) {
          uint64_t rqh = call_plane(c, W, r, 0)[w], rqd = call_plane(c, W, r, 1)[w];
          uint64_t fr = rqh & ~h[w], to = rqd & ~d[w];
          if (fr) flag[i] |= 2;
          if (to) flag[i] |= 1;
          h[w] |= rqh; d[w] |= rqd;
          if (cr->to) cr->to[o + w] = to;
          if (cr->from) cr->from[o + w] = fr;
          if (cr->entry_h) cr->entry_h[o + w] = h[w];
          if (cr->entry_d) cr->entry_d[o + w] = d[w];
          h[w] = call_plane(c, W, r, 2)[w] | (h[w] & ~call_plane(c, W, r, 3)[w]);
          d[w] = call_plane(c, W, r, 4)[w] | (d[w] & ~call_plane(c, W, r, 5)[w]);
        }
        continue;
      }
      int v = a_var(a), k = a_kind(a), S = a_space(a);
      uint64_t *own = S == SPACE_DEV ? d : h, *oth = S == SPACE_DEV ? h : d;
      if (k & A_KIND_R) {
        if (!get_bit(own, v)) { flag[i] = S == SPACE_DEV ? 1 : 2; set_bit(own, v, 1); }
      }
      if (k & A_KIND_W) { set_bit(own, v, 1); set_bit(oth, v, 0); }
    }
  }
  free(h); free(d);
}

/* Liveness right after each call (Live = AntH | AntD, Sec. II-B): from Live
   at the block exit (OR of the successors' Live_in, or exit_host_live at a
   region exit), fold the block's later accesses backward: a read in either
   space makes the variable live, a write ends it; a call makes ReqH | ReqD
   live after ending what it must write. */
static void call_exit_live(const oracle_cfg *c, const graph *g, const uint64_t *LV, const uint64_t *xlive,
                           const int32_t *site_of, uint64_t *rows) {
  int W = g->W;
  uint64_t *x = xcalloc((size_t)W, sizeof(uint64_t));
  for (int b = 0; b < g->N; ++b) {
    if (!g->reach[b]) continue;
    int has_call = 0;
    for (int i = g->ao[b]; i < g->ao[b + 1]; ++i) has_call |= a_is_call(g->acc[i]);
    if (!has_call) continue;
    if (g->so[b] == g->so[b + 1]) {
      for (int w = 0; w < W; ++w) x[w] = xlive[w];
    } else {
      memset(x, 0, (size_t)W * sizeof(uint64_t));
      for (int e = g->so[b]; e < g->so[b + 1]; ++e)
        for (int w = 0; w < W; ++w) x[w] |= LV[(size_t)g->s[e] * W + w];
    }
    for (int i = g->ao[b + 1] - 1; i >= g->ao[b]; --i) {
      uint32_t a = g->acc[i];
      if (a_is_call(a)) {
        int r = a_call_row(a);
        memcpy(rows + (size_t)site_of[i] * W, x, (size_t)W * sizeof(uint64_t));
        for (int w = 0; w < W; ++w)
          x[w] = call_plane(c, W, r, 0)[w] | call_plane(c, W, r, 1)[w] | (x[w] & ~call_plane(c, W, r, 6)[w]);
        continue;
      }
      int v = a_var(a), k = a_kind(a);
      if (k & A_KIND_W) set_bit(x, v, 0);
      if (k & A_KIND_R) set_bit(x, v, 1);
    }
  }
  free(x);
}

int oracle_solve(const oracle_cfg *c, oracle_out *out) {
  int rc = validate(c);
  if (rc) return rc;
  graph g;
  if ((rc = build_graph(c, &g))) { free_graph(&g); return rc; }
  int N = g.N, W = g.W, E = g.E;
  size_t NW = (size_t)N * W;
  uint64_t *pl[26];
  for (int i = 0; i < 26; ++i) {
    pl[i] = xcalloc(NW, sizeof(uint64_t));
    if (!pl[i]) { for (int j = 0; j < i; ++j) free(pl[j]); free_graph(&g); return ORACLE_E_NOMEM; }
  }
  uint64_t *GH = pl[0], *KH = pl[1], *GD = pl[2], *KD = pl[3], *UH = pl[4], *UD = pl[5], *DF = pl[6];
  uint64_t *AH = pl[7], *AD = pl[8], *LV = pl[9], *HPI = pl[10], *HPO = pl[11];
  uint64_t *AM = pl[12], *MH = pl[14], *MD = pl[15];
  uint64_t *DI = pl[16], *DO = pl[17], *HM = pl[18], *HI = pl[19], *HO = pl[20], *FX = pl[21];
  uint8_t *hdr = xcalloc((size_t)N, 1), *ent = xcalloc((size_t)E, 1);
  uint8_t *inr = xcalloc((size_t)N, 1), *rxe = xcalloc((size_t)E, 1);
  uint64_t *TE = xcalloc((size_t)E * W, sizeof(uint64_t)), *FE = xcalloc((size_t)E * W, sizeof(uint64_t));
  uint8_t *fl = xcalloc((size_t)g.A, 1);
  uint64_t *init_h = xcalloc((size_t)W, sizeof(uint64_t)), *init_d = xcalloc((size_t)W, sizeof(uint64_t));
  uint64_t *xlive = xcalloc((size_t)W, sizeof(uint64_t));
  if (!hdr || !ent || !inr || !rxe || !TE || !FE || !fl || !init_h || !init_d || !xlive) {
    rc = ORACLE_E_NOMEM;
    goto done;
  }
  const int region_mode = c->data_region && c->region;
  if (region_mode && (rc = data_region(c, &g, inr, rxe))) goto done;
  for (int w = 0; w < W; ++w) {
    init_h[w] = (c->entry_host_valid ? c->entry_host_valid[w] : ~(uint64_t)0) & g.top[w];
    init_d[w] = (c->entry_dev_valid ? c->entry_dev_valid[w] : 0) & g.top[w];
    xlive[w] = (c->exit_host_live ? c->exit_host_live[w] : ~(uint64_t)0) & g.top[w];
  }

  /* 1. local rule */
  local_rule(c, &g, GH, KH, GD, KD, UH, UD, DF);
  /* 2. anticipation and liveness */
  if ((rc = anticipation(&g, UH, DF, xlive, AH))) goto done;
  if ((rc = anticipation(&g, UD, DF, NULL, AD))) goto done;
  for (size_t i = 0; i < NW; ++i) LV[i] = AH[i] | AD[i];
  /* 3. plain host validity */
  {
    fwd_problem P = {GH, KH, init_h, NULL, NULL, NULL, NULL, HPI, HPO, NULL};
    if ((rc = forward_must(&g, &P))) goto done;
  }
  /* 4. loops and masks */
  if ((rc = natural_loops(&g, KH, KD, UH, UD, DF, hdr, ent, MH, MD))) goto done;
  /* 5. device validity: hoisted `to' on loop-entry edges where the host
        copy is valid (plain host validity as the source test); eager
        placement: on every edge, what every path on reads on the device
        first, where the host copy is the latest */
  const int eager = c->eager_to != 0;
  if (eager && (rc = must_anticipation(&g, UD, DF, AM))) goto done;
  {
    fwd_problem P = {GD, KD, init_d, ent, MD, HPO, NULL, DI, DO, NULL};
    if (eager) {
      P.any_mask = AM;
      P.any_src = HPO;
    }
    if ((rc = forward_must(&g, &P))) goto done;
  }
  /* 6. host validity: hoisted `from' on loop-entry edges where the device
        copy is valid; live and valid in neither space -> host */
  {
    uint64_t *C = pl[22];
    for (size_t i = 0; i < NW; ++i) C[i] = LV[i] & ~DI[i];
    fwd_problem P = {GH, KH, init_h, ent, MH, DO, C, HI, HO, HM, NULL, NULL};
    if (region_mode) {  /* leaving the data region: live data made valid on the host */
      P.is_exit_edge = rxe;
      P.exit_gen = LV;
    }
    if ((rc = forward_must(&g, &P))) goto done;
  }
  /* 7. emission */
  for (int b = 0; b < N; ++b) {
    if (!g.reach[b]) continue;
    for (int k = g.po[b]; k < g.po[b + 1]; ++k) {
      int p = g.ps[k], e = g.pe[k];
      if (!g.reach[p]) continue;
      for (int w = 0; w < W; ++w) {
        size_t ob = (size_t)b * W + w, op = (size_t)p * W + w, oe = (size_t)e * W + w;
        uint64_t hedge = HO[op];
        if (eager) TE[oe] = AM[ob] & ~DO[op] & HPO[op];
        if (ent[e]) {
          TE[oe] |= MD[ob] & ~DO[op] & HPO[op];
          FE[oe] = MH[ob] & ~HO[op] & DO[op];
          hedge |= MH[ob] & DO[op];
        }
        if (rxe[e]) {  /* the data region's exit: `from' for live data stale on the host */
          FE[oe] |= LV[ob] & ~HO[op];
          hedge |= LV[ob];
        }
        FE[oe] |= (LV[ob] & ~DI[ob] & ~HM[ob]) & ~hedge;
      }
    }
    if (g.so[b] == g.so[b + 1])
      for (int w = 0; w < W; ++w) FX[(size_t)b * W + w] = xlive[w] & ~HO[(size_t)b * W + w];
  }
  {
    int32_t *site_of = xcalloc((size_t)g.A, sizeof(int32_t));
    int S = 0;
    for (int i = 0; i < g.A; ++i) site_of[i] = a_is_call(g.acc[i]) ? S++ : -1;
    call_rows cr = {out->call_to, out->call_from, out->call_entry_h, out->call_entry_d, out->call_exit_live};
    size_t SW = (size_t)S * W * sizeof(uint64_t);
    if (cr.to) memset(cr.to, 0, SW);
    if (cr.from) memset(cr.from, 0, SW);
    if (cr.entry_h) memset(cr.entry_h, 0, SW);
    if (cr.entry_d) memset(cr.entry_d, 0, SW);
    if (cr.exit_live) memset(cr.exit_live, 0, SW);
    access_flags(c, &g, HI, DI, fl, site_of, &cr);
    if (cr.exit_live) call_exit_live(c, &g, LV, xlive, site_of, cr.exit_live);
    free(site_of);
  }

  /* copy out */
#define CP(dst, src, n) do { if (dst) memcpy((dst), (src), (n) * sizeof(*(src))); } while (0)
  CP(out->reachable, g.reach, (size_t)N);
  CP(out->is_header, hdr, (size_t)N);
  CP(out->is_loop_entry, ent, (size_t)E);
  CP(out->gen_h, GH, NW); CP(out->kill_h, KH, NW); CP(out->gen_d, GD, NW); CP(out->kill_d, KD, NW);
  CP(out->ue_h, UH, NW); CP(out->ue_d, UD, NW); CP(out->def, DF, NW);
  CP(out->ant_h_in, AH, NW); CP(out->ant_d_in, AD, NW); CP(out->live_in, LV, NW);
  CP(out->hp_in, HPI, NW); CP(out->hp_out, HPO, NW);
  CP(out->mask_h, MH, NW); CP(out->mask_d, MD, NW);
  CP(out->d_in, DI, NW); CP(out->d_out, DO, NW); CP(out->hm, HM, NW);
  CP(out->h_in, HI, NW); CP(out->h_out, HO, NW);
  CP(out->to_edge, TE, (size_t)E * W); CP(out->from_edge, FE, (size_t)E * W);
  CP(out->from_exit, FX, NW);
  CP(out->acc_flag, fl, (size_t)g.A);
  CP(out->in_region, inr, (size_t)N);
  CP(out->region_exit, rxe, (size_t)E);
  CP(out->ant_dm_in, AM, NW);
#undef CP
  rc = ORACLE_OK;
done:
  for (int i = 0; i < 26; ++i) free(pl[i]);
  free(hdr); free(ent); free(inr); free(rxe); free(TE); free(FE); free(fl); free(init_h); free(init_d);
  free(xlive);
  free_graph(&g);
  return rc;
}

/* ---- callee summaries (Sec. IV-C side effects) ----------------------------
 * Requirements: anticipation at the entry with nothing live after the exit.
 * Net effects: plain validity (the local rule along paths, no transfers)
 * from an all-stale and from an all-valid entry, met over the reachable
 * exits.  Must-writes: forward must problem "written so far", met over the
 * reachable exits. */
int oracle_summarize(const oracle_cfg *c, uint64_t *planes) {
  int rc = validate(c);
  if (rc) return rc;
  graph g;
  if ((rc = build_graph(c, &g))) { free_graph(&g); return rc; }
  int N = g.N, W = g.W;
  size_t NW = (size_t)N * W;
  uint64_t *pl[14];
  for (int i = 0; i < 14; ++i) pl[i] = xcalloc(NW, sizeof(uint64_t));
  uint64_t *zero = xcalloc((size_t)W, sizeof(uint64_t)), *nokill = pl[13];
  uint64_t *GH = pl[0], *KH = pl[1], *GD = pl[2], *KD = pl[3], *UH = pl[4], *UD = pl[5], *DF = pl[6];
  uint64_t *AH = pl[7], *AD = pl[8], *XI = pl[9], *XO = pl[10];
  local_rule(c, &g, GH, KH, GD, KD, UH, UD, DF);
  memset(planes, 0, (size_t)7 * W * sizeof(uint64_t));
  if ((rc = anticipation(&g, UH, DF, NULL, AH)) || (rc = anticipation(&g, UD, DF, NULL, AD))) goto done;
  for (int w = 0; w < W; ++w) {
    planes[0 * W + w] = AH[(size_t)g.entry * W + w];
    planes[1 * W + w] = AD[(size_t)g.entry * W + w];
  }
  {
    int n_exit = 0;
    for (int b = 0; b < N; ++b) n_exit += g.reach[b] && g.so[b] == g.so[b + 1];
    if (!n_exit) { rc = ORACLE_OK; goto done; }
    /* met over exits: Gen = AND of valid (entry all stale); Kill = OR of
       stale (entry all valid); MustDef = AND of written (entry nothing) */
    const uint64_t *gens[2] = {GH, GD}, *kills[2] = {KH, KD};
    for (int S = 0; S < 2; ++S) {
      fwd_problem P0 = {gens[S], kills[S], zero, NULL, NULL, NULL, NULL, XI, XO, NULL};
      if ((rc = forward_must(&g, &P0))) goto done;
      uint64_t *gen = planes + (size_t)(2 + 2 * S) * W, *kill = planes + (size_t)(3 + 2 * S) * W;
      for (int w = 0; w < W; ++w) gen[w] = g.top[w];
      for (int b = 0; b < N; ++b)
        if (g.reach[b] && g.so[b] == g.so[b + 1])
          for (int w = 0; w < W; ++w) gen[w] &= XO[(size_t)b * W + w];
      fwd_problem P1 = {gens[S], kills[S], g.top, NULL, NULL, NULL, NULL, XI, XO, NULL};
      if ((rc = forward_must(&g, &P1))) goto done;
      for (int b = 0; b < N; ++b)
        if (g.reach[b] && g.so[b] == g.so[b + 1])
          for (int w = 0; w < W; ++w) kill[w] |= g.top[w] & ~XO[(size_t)b * W + w];
    }
    fwd_problem PM = {DF, nokill, zero, NULL, NULL, NULL, NULL, XI, XO, NULL};
    if ((rc = forward_must(&g, &PM))) goto done;
    uint64_t *md = planes + (size_t)6 * W;
    for (int w = 0; w < W; ++w) md[w] = g.top[w];
    for (int b = 0; b < N; ++b)
      if (g.reach[b] && g.so[b] == g.so[b + 1])
        for (int w = 0; w < W; ++w) md[w] &= XO[(size_t)b * W + w];
  }
  rc = ORACLE_OK;
done:
  for (int i = 0; i < 14; ++i) free(pl[i]);
  free(zero);
  free_graph(&g);
  return rc;
}
