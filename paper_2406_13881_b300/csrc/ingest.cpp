// ingest.cpp -- host-side ingestion of one CFG (see ingest.h).
#include "ingest.h"
#include "parallel.h"
#include "solver.h"

#include <algorithm>
#include <cstring>

namespace ompdart {

namespace {

constexpr int kNone = -1;

bool fail(std::string *err, const char *msg) {
  if (err) *err = msg;
  return false;
}

// Items per host thread below which a pass of the ingestion stays on the
// calling thread (batches ingest many small CFGs on a pool already).
#ifndef OMPDART_INGEST_PAR_MIN
#define OMPDART_INGEST_PAR_MIN (1 << 16)
#endif
constexpr int kParMin = OMPDART_INGEST_PAR_MIN;
constexpr int kParMax = 16;

// The first i in [0, n) with bad(i), else n (ranges scanned in parallel).
template <class F>
int first_bad(int n, F bad) {
  int first[kParMax];
  const int T = parallel_ranges(n, kParMin, kParMax, [&](int t, int lo, int hi) {
    first[t] = n;
    for (int i = lo; i < hi; ++i)
      if (bad(i)) {
        first[t] = i;
        return;
      }
  });
  for (int t = 0; t < T; ++t)
    if (first[t] < n) return first[t];
  return n;
}

bool check_format(const ompdart_cfg *c, std::string *err) {
  if (!c) return fail(err, "cfg is NULL");
  if (c->n_blocks < 1) return fail(err, "n_blocks must be >= 1");
  if (c->n_vars < 1 || c->n_vars > (1 << 24)) return fail(err, "n_vars must be in [1, 2^24]");
  if (c->entry < 0 || c->entry >= c->n_blocks) return fail(err, "entry out of range");
  if (!c->succ_off || !c->acc_off) return fail(err, "succ_off / acc_off missing");
  if (c->succ_off[0] != 0 || c->acc_off[0] != 0) return fail(err, "CSR offsets must start at 0");
  if (first_bad(c->n_blocks, [&](int b) {
        return c->succ_off[b + 1] < c->succ_off[b] || c->acc_off[b + 1] < c->acc_off[b];
      }) < c->n_blocks)
    return fail(err, "CSR offsets must be non-decreasing");
  const int E = c->succ_off[c->n_blocks], A = c->acc_off[c->n_blocks];
  if ((E && !c->succ) || (A && !c->acc)) return fail(err, "succ / acc missing");
  // the first bad edge and the first bad access decide the message
  const int e = first_bad(E, [&](int k) { return c->succ[k] < 0 || c->succ[k] >= c->n_blocks || c->succ[k] == c->entry; });
  if (e < E) {
    if (c->succ[e] < 0 || c->succ[e] >= c->n_blocks) return fail(err, "successor id out of range");
    return fail(err, "the entry block must have no predecessors");
  }
  auto acc_msg = [&](int i) -> const char * {
    const uint32_t a = c->acc[i];
    if (a >> 31) {
      if (!c->call_planes || (int)(a & 0x7FFFFFFFu) >= c->n_calls) return "call access without a matching call-table row";
      return nullptr;
    }
    if ((a >> 27) & 0xFu) return "reserved access bits 27-30 must be zero";
    if ((int)(a & 0xFFFFFFu) >= c->n_vars) return "access variable out of range";
    if (((a >> 24) & 3u) == 0) return "access kind must be 1, 2 or 3";
    return nullptr;
  };
  const int a = first_bad(A, [&](int i) { return acc_msg(i) != nullptr; });
  if (a < A) return fail(err, acc_msg(a));
  return true;
}

// Lengauer-Tarjan immediate dominators over blocks reachable from `entry`.
// preorder[] lists reachable blocks in DFS preorder, dfn[] is each block's
// index there (-1 if unreachable), and idom[] the DFS number of each DFS
// number's immediate dominator (idom[0] = 0, the entry).
void lengauer_tarjan(int N, int entry, const std::vector<int32_t> &so, const int32_t *succ,
                     const std::vector<int32_t> &po, const std::vector<int32_t> &psrc,
                     std::vector<int32_t> *preorder_out, std::vector<int32_t> *dfn_out,
                     std::vector<int32_t> *idom_out) {
  std::vector<int32_t> dfn(N, kNone), vert, parent(N, kNone);
  vert.reserve(N);
  {  // iterative DFS, preorder numbering
    std::vector<std::pair<int32_t, int32_t>> st;
    st.push_back({entry, so[entry]});
    dfn[entry] = 0;
    vert.push_back(entry);
    while (!st.empty()) {
      auto &top = st.back();
      if (top.second < so[top.first + 1]) {
        int t = succ[top.second++];
        if (dfn[t] == kNone) {
          dfn[t] = (int32_t)vert.size();
          vert.push_back(t);
          parent[t] = top.first;
          st.push_back({t, so[t]});
        }
      } else {
        st.pop_back();
      }
    }
  }
  const int n = (int)vert.size();
  // work on dfs numbers 0..n-1
  std::vector<int32_t> semi(n), label(n), anc(n, kNone), idom(n, kNone), par(n, kNone);
  std::vector<int32_t> bucket_head(n, kNone), bucket_next(n, kNone);
  for (int i = 0; i < n; ++i) {
    semi[i] = i;
    label[i] = i;
    if (i) par[i] = dfn[parent[vert[i]]];
  }
  std::vector<int32_t> path;
  auto eval = [&](int v) -> int {
    if (anc[v] == kNone) return v;
    // iterative path compression
    path.clear();
    int x = v;
    while (anc[anc[x]] != kNone) {
      path.push_back(x);
      x = anc[x];
    }
    for (int k = (int)path.size() - 1; k >= 0; --k) {
      int y = path[k];
      if (semi[label[anc[y]]] < semi[label[y]]) label[y] = label[anc[y]];
      anc[y] = anc[anc[y]];
    }
    return label[v];
  };
  // the reachable predecessors of each DFS number, as DFS numbers (one
  // gather up front keeps the sequential part on dense arrays)
  std::vector<int32_t> qoff(n + 1, 0), qdfn;
  parallel_ranges(n, kParMin, kParMax, [&](int, int lo, int hi) {
    for (int w = lo; w < hi; ++w) {
      const int bw = vert[w];
      int c = 0;
      for (int k = po[bw]; k < po[bw + 1]; ++k) c += dfn[psrc[k]] != kNone;
      qoff[w + 1] = c;
    }
  });
  for (int w = 0; w < n; ++w) qoff[w + 1] += qoff[w];
  qdfn.resize(qoff[n]);
  parallel_ranges(n, kParMin, kParMax, [&](int, int lo, int hi) {
    for (int w = lo; w < hi; ++w) {
      const int bw = vert[w];
      int x = qoff[w];
      for (int k = po[bw]; k < po[bw + 1]; ++k)
        if (dfn[psrc[k]] != kNone) qdfn[x++] = dfn[psrc[k]];
    }
  });
  for (int w = n - 1; w >= 1; --w) {
    for (int k = qoff[w]; k < qoff[w + 1]; ++k) {
      const int u = eval(qdfn[k]);
      if (semi[u] < semi[w]) semi[w] = semi[u];
    }
    // add w to bucket of its semidominator
    bucket_next[w] = bucket_head[semi[w]];
    bucket_head[semi[w]] = w;
    anc[w] = par[w];  // link
    for (int v = bucket_head[par[w]]; v != kNone; v = bucket_next[v]) {
      int u = eval(v);
      idom[v] = semi[u] < semi[v] ? u : par[w];
    }
    bucket_head[par[w]] = kNone;
  }
  for (int w = 1; w < n; ++w)
    if (idom[w] != semi[w]) idom[w] = idom[idom[w]];
  idom[0] = 0;
  *idom_out = std::move(idom);
  *dfn_out = std::move(dfn);
  *preorder_out = std::move(vert);
}

// The single target data region (see ingest.h) of one ingested CFG:
// in_region, kernel ids, the region's entry and exit edges, the kernel whose
// entry opens it, and the exit edges added to the edge constants (eid_ent
// updated for the new ones).
template <class Dom>
void find_data_region(const ompdart_cfg *c, Ingest *g, const std::vector<int32_t> &so, const int32_t *succ,
                      const std::vector<int32_t> &po, const std::vector<int32_t> &psrc,
                      const std::vector<int32_t> &peid, const std::vector<uint8_t> &reach,
                      const std::vector<int32_t> &pre, const std::vector<int32_t> &dfn,
                      const std::vector<int32_t> &idom, Dom dominates, std::vector<int32_t> *eid_ent) {
  const int N = g->N;
  g->region_mode = true;
  g->kernel.assign(c->region, c->region + N);
  int nk = 0;
  for (int b = 0; b < N; ++b) nk = std::max(nk, c->region[b] + 1);
  g->kern_off = {0, nk};
  g->in_region.assign(N, 0);
  g->start_kernel = {kNone};
  g->entry_in_region = {0};
  g->rin_off = {0, 0};
  g->rout_off = {0, 0};
  // kernel blocks (cap 1) and bodies of loops holding one (cap 2), their headers
  std::vector<uint8_t> cap(N, 0), hcap(N, 0);
  bool any = false;
  for (int b = 0; b < N; ++b)
    if (reach[b] && c->region[b] >= 0) cap[b] = 1, any = true;
  if (!any) return;
  for (int l = 0; l < g->L; ++l) {
    bool holds = false;
    for (int x = g->body_off[l]; x < g->body_off[l + 1] && !holds; ++x) holds = c->region[g->body_blk[x]] >= 0;
    if (!holds) continue;
    hcap[g->loop_head[l]] = 1;
    for (int x = g->body_off[l]; x < g->body_off[l + 1]; ++x) cap[g->body_blk[x]] |= 2;
  }
  // S: meet of the kernel blocks and capturing headers in the dominator
  // tree (DFS numbers: an immediate dominator has a smaller one)
  auto meet = [](int a, int b, const std::vector<int32_t> &par) {
    while (a != b) {
      if (a > b) a = par[a];
      else b = par[b];
    }
    return a;
  };
  int S = kNone;
  for (int b = 0; b < N; ++b)
    if ((cap[b] & 1) || hcap[b]) S = S == kNone ? dfn[b] : meet(S, dfn[b], idom);
  S = pre[S];
  // post-dominators: Lengauer-Tarjan on the reversed graph rooted at a
  // virtual exit X = N whose successors are the exit blocks; a block's
  // successors there are its reachable predecessors
  const int X = N;
  std::vector<int32_t> so2(N + 2, 0), su2, po2(N + 2, 0), ps2;
  for (int b = 0; b < N; ++b) {
    int n = 0;
    for (int k = po[b]; k < po[b + 1]; ++k) n += reach[psrc[k]];
    so2[b + 1] = n;
  }
  for (int b = 0; b < N; ++b) so2[X + 1] += reach[b] && so[b] == so[b + 1];
  for (int b = 0; b <= N; ++b) so2[b + 1] += so2[b];
  su2.resize(so2[N + 1]);
  for (int b = 0, x = 0; b < N; ++b)
    for (int k = po[b]; k < po[b + 1]; ++k)
      if (reach[psrc[k]]) su2[x++] = psrc[k];
  for (int b = 0, x = so2[X]; b < N; ++b)
    if (reach[b] && so[b] == so[b + 1]) su2[x++] = b;
  // predecessors in the reversed graph: the forward successors, and X for an exit
  for (int b = 0; b < N; ++b) po2[b + 1] = reach[b] ? (so[b + 1] - so[b]) + (so[b] == so[b + 1]) : 0;
  for (int b = 0; b <= N; ++b) po2[b + 1] += po2[b];
  ps2.resize(po2[N + 1]);
  for (int b = 0; b < N; ++b) {
    if (!reach[b]) continue;
    int x = po2[b];
    for (int e = so[b]; e < so[b + 1]; ++e) ps2[x++] = succ[e];
    if (so[b] == so[b + 1]) ps2[x++] = X;
  }
  std::vector<int32_t> pre2, dfn2, ipd;
  lengauer_tarjan(N + 1, X, so2, su2.data(), po2, ps2, &pre2, &dfn2, &ipd);
  const int n2 = (int)pre2.size();
  std::vector<int32_t> sz2(n2, 1), tin2(n2, 0), nxt2(n2, 0);
  for (int w = n2 - 1; w >= 1; --w) sz2[ipd[w]] += sz2[w];
  nxt2[0] = 1;
  for (int w = 1; w < n2; ++w) {
    tin2[w] = nxt2[ipd[w]];
    nxt2[ipd[w]] += sz2[w];
    nxt2[w] = tin2[w] + 1;
  }
  // E: meet, in the post-dominator tree, of the blocks the captured blocks lead to outside themselves
  int E = kNone;
  bool to_x = false;
  for (int b = 0; b < N; ++b) {
    if (!cap[b]) continue;
    for (int e = so[b]; e < so[b + 1]; ++e) {
      const int t = succ[e];
      if (cap[t]) continue;
      if (dfn2[t] == kNone) to_x = true;
      else E = E == kNone ? dfn2[t] : meet(E, dfn2[t], ipd);
    }
  }
  if (to_x || E == kNone) E = 0;  // the virtual exit (DFS number 0)
  const int Eb = pre2[E];         // X when the region runs to the virtual exit
  for (int b = 0; b < N; ++b) {
    if (!reach[b] || b == Eb || !dominates(S, b)) continue;
    const int d = dfn2[b];
    if (E != 0 && (d == kNone || !(tin2[E] <= tin2[d] && tin2[d] < tin2[E] + sz2[E]))) continue;
    g->in_region[b] = 1;
  }
  // boundary edges; the exit edges join the edge constants
  for (int b = 0; b < N; ++b) {
    if (!reach[b]) continue;
    for (int e = so[b]; e < so[b + 1]; ++e) {
      const int t = succ[e];
      if (!g->in_region[b] && g->in_region[t]) g->rin_eid.push_back(e);
      if (g->in_region[b] && !g->in_region[t]) g->rout_eid.push_back(e);
    }
  }
  g->rin_off = {0, (int32_t)g->rin_eid.size()};
  g->rout_off = {0, (int32_t)g->rout_eid.size()};
  g->entry_in_region = {g->in_region[c->entry]};
  for (int e : g->rout_eid) {
    int &k = (*eid_ent)[e];
    if (k == kNone) {
      k = g->K++;
      g->ent_loop.push_back(kNone);
      g->ent_src.push_back((int32_t)(std::upper_bound(so.begin(), so.end(), e) - so.begin()) - 1);
      g->ent_eid.push_back(e);
      g->ent_rx.push_back(1);
    } else {
      g->ent_rx[k] = 1;
    }
  }
  // the kernel whose entry edges are exactly the region's entry edges (and
  // that holds the CFG's entry iff the region starts there) opens the region
  std::vector<int32_t> rin = g->rin_eid;
  std::sort(rin.begin(), rin.end());
  for (int k = 0; k < nk; ++k) {
    std::vector<int32_t> ke;
    for (int t = 0; t < N; ++t) {
      if (!reach[t] || c->region[t] != k) continue;
      for (int q = po[t]; q < po[t + 1]; ++q)
        if (reach[psrc[q]] && c->region[psrc[q]] != k) ke.push_back(peid[q]);
    }
    std::sort(ke.begin(), ke.end());
    const bool holds_entry = c->region[c->entry] == k;
    if (ke == rin && (bool)g->entry_in_region[0] == holds_entry && (holds_entry || !rin.empty())) {
      g->start_kernel[0] = k;
      break;
    }
  }
}

}  // namespace

int ingest(const ompdart_cfg *c, Ingest *g, std::string *err, bool data_region, bool all_edges) {
  if (!check_format(c, err)) return OMPDART_E_INVALID;
  if (data_region && c->region &&
      first_bad(c->n_blocks, [&](int b) { return c->region[b] < -1 || c->region[b] >= c->n_blocks; }) <
          c->n_blocks) {
    if (err) *err = "kernel ids (region) must be -1 or in [0, n_blocks)";
    return OMPDART_E_INVALID;
  }
  const int N = c->n_blocks;
  g->N = N;
  g->E = c->succ_off[N];
  g->A = c->acc_off[N];
  g->V = c->n_vars;
  g->W = (c->n_vars + 63) / 64;
  g->entry = c->entry;
  std::vector<int32_t> so(c->succ_off, c->succ_off + N + 1);
  const int32_t *succ = c->succ;
  TraceScope trace("ingest: predecessors", N);

  // predecessor CSR with edge ids
  std::vector<int32_t> po(N + 1, 0), psrc(g->E), peid(g->E);
  for (int e = 0; e < g->E; ++e) po[succ[e] + 1]++;
  for (int b = 0; b < N; ++b) po[b + 1] += po[b];
  {
    std::vector<int32_t> fill(po.begin(), po.end() - 1);
    for (int b = 0; b < N; ++b)
      for (int e = so[b]; e < so[b + 1]; ++e) {
        int k = fill[succ[e]]++;
        psrc[k] = b;
        peid[k] = e;
      }
  }

  // dominators on the reachable subgraph
  trace.next("ingest: dominators", N);
  std::vector<int32_t> pre, dfn, idom;
  lengauer_tarjan(N, c->entry, so, succ, po, psrc, &pre, &dfn, &idom);
  const int n_reach = (int)pre.size();
  std::vector<uint8_t> reach(N, 0);
  for (int b : pre) reach[b] = 1;

  // the dominator tree as preorder intervals over DFS numbers:
  // a dom b  <=>  tin[a] <= tin[b] < tin[a] + sz[a].  An immediate
  // dominator has a smaller DFS number than the block it dominates, so the
  // subtree sizes add up in decreasing DFS order and the intervals are
  // handed out in increasing DFS order (no tree walk).
  std::vector<int32_t> sz(n_reach, 1), tin(n_reach, 0), nxt(n_reach, 0);
  for (int w = n_reach - 1; w >= 1; --w) sz[idom[w]] += sz[w];
  nxt[0] = 1;
  for (int w = 1; w < n_reach; ++w) {
    const int u = idom[w];
    tin[w] = nxt[u];
    nxt[u] += sz[w];
    nxt[w] = tin[w] + 1;
  }
  auto dominates = [&](int a, int b) {  // a and b reachable
    const int da = dfn[a], db = dfn[b];
    return tin[da] <= tin[db] && tin[db] < tin[da] + sz[da];
  };

  // natural loops; headers in decreasing DFS preorder = inner loops first
  trace.next("ingest: natural loops", n_reach);
  std::vector<uint8_t> is_head(n_reach, 0);
  parallel_ranges(n_reach, kParMin, kParMax, [&](int, int lo, int hi) {
    for (int i = lo; i < hi; ++i) {
      const int h = pre[i];
      for (int k = po[h]; k < po[h + 1]; ++k)
        if (reach[psrc[k]] && dominates(h, psrc[k])) {
          is_head[i] = 1;
          break;
        }
    }
  });
  std::vector<int32_t> headers;
  for (int i = n_reach - 1; i >= 0; --i)
    if (is_head[i]) headers.push_back(pre[i]);
  const int L = (int)headers.size();
  // each natural loop's body: the header and every block reaching a latch
  // without passing through the header (independent per loop: flooded in
  // parallel, each thread with its own marks)
  std::vector<std::vector<int32_t>> bodies(L);
  parallel_ranges(L, std::max(1, kParMin / 64), kParMax, [&](int, int lo, int hi) {
    std::vector<int32_t> mark(N, kNone), stk;
    for (int l = lo; l < hi; ++l) {
      const int h = headers[l];
      auto &bd = bodies[l];
      bd.push_back(h);
      mark[h] = l;
      stk.clear();
      for (int k = po[h]; k < po[h + 1]; ++k) {
        const int t = psrc[k];
        if (reach[t] && dominates(h, t) && mark[t] != l) {
          mark[t] = l;
          stk.push_back(t);
        }
      }
      while (!stk.empty()) {
        const int b = stk.back();
        stk.pop_back();
        bd.push_back(b);
        for (int k = po[b]; k < po[b + 1]; ++k) {
          const int p = psrc[k];
          if (reach[p] && mark[p] != l) {
            mark[p] = l;
            stk.push_back(p);
          }
        }
      }
    }
  });
  // innermost loop of each block and the loop tree, inner loops first
  std::vector<int32_t> inner(N, kNone), lparent(L, kNone);
  for (int l = 0; l < L; ++l) {
    const int h = headers[l];
    for (int b : bodies[l]) {
      if (inner[b] == kNone) {
        inner[b] = l;
      } else if (b != h || inner[b] != l) {
        // b belongs to an already-built (inner) loop: link that loop chain
        int x = inner[b];
        while (lparent[x] != kNone && lparent[x] != l) x = lparent[x];
        if (x != l && lparent[x] == kNone) lparent[x] = l;
      }
    }
  }
  std::vector<int32_t> ldepth(L, 0);
  for (int l = L - 1; l >= 0; --l) {  // outer loops have larger ids here
    ldepth[l] = lparent[l] == kNone ? 1 : 0;
  }
  // depth by walking parents (parents have larger ids: processed later)
  for (int l = 0; l < L; ++l) {
    int d = 1;
    for (int x = lparent[l]; x != kNone; x = lparent[x]) ++d;
    ldepth[l] = d;
  }
  auto common_depth = [&](int a, int b) -> int {  // depth of the deepest loop holding both
    int la = inner[a], lb = inner[b];
    int da = la == kNone ? 0 : ldepth[la], db = lb == kNone ? 0 : ldepth[lb];
    while (da > db) { la = lparent[la]; --da; }
    while (db > da) { lb = lparent[lb]; --db; }
    while (la != lb) { la = lparent[la]; lb = lparent[lb]; --da; }
    return da;
  };

  // loop-ordered DFS: at every block visit successors that leave the most
  // loops first, so that their subtrees finish first and every loop body
  // ends up as one run of positions right after its header.
  trace.next("ingest: loop-ordered DFS", n_reach);
  std::vector<int32_t> post;
  post.reserve(pre.size());
  {
    std::vector<uint8_t> seen(N, 0);
    std::vector<int32_t> sorted_succ(g->E);
    parallel_ranges(N, kParMin, kParMax, [&](int, int lo, int hi) {
      std::vector<std::pair<int, int32_t>> key;
      for (int b = lo; b < hi; ++b) {
        if (!reach[b]) continue;
        int n = so[b + 1] - so[b];
        int32_t *dst = sorted_succ.data() + so[b];
        for (int k = 0; k < n; ++k) dst[k] = succ[so[b] + k];
        if (n > 1) {  // stable: equal depths keep the successor order
          key.resize(n);
          for (int k = 0; k < n; ++k) key[k] = {common_depth(b, dst[k]), dst[k]};
          std::stable_sort(key.begin(), key.end(),
                           [](const std::pair<int, int32_t> &x, const std::pair<int, int32_t> &y) {
                             return x.first < y.first;
                           });
          for (int k = 0; k < n; ++k) dst[k] = key[k].second;
        }
      }
    });
    std::vector<std::pair<int32_t, int32_t>> st;
    st.push_back({c->entry, so[c->entry]});
    seen[c->entry] = 1;
    while (!st.empty()) {
      auto &t = st.back();
      if (t.second < so[t.first + 1]) {
        int s = sorted_succ[t.second++];
        if (!seen[s]) {
          seen[s] = 1;
          st.push_back({s, so[s]});
        }
      } else {
        post.push_back(t.first);
        st.pop_back();
      }
    }
  }
  const int M = (int)post.size();
  g->M = M;
  g->order.assign(post.rbegin(), post.rend());
  g->pos.assign(N, kNone);
  parallel_ranges(M, kParMin, kParMax, [&](int, int lo, int hi) {
    for (int i = lo; i < hi; ++i) g->pos[g->order[i]] = i;
  });

  // reducibility: every retreating edge must be a back edge
  g->reducible = first_bad(M, [&](int i) {
                   const int u = g->order[i];
                   for (int e = so[u]; e < so[u + 1]; ++e) {
                     const int v = succ[e];
                     if (g->pos[v] <= i && !dominates(v, u)) return true;
                   }
                   return false;
                 }) == M;

  // loops renumbered by header position
  trace.next("ingest: loop tables", L);
  std::vector<int32_t> perm(L);
  for (int l = 0; l < L; ++l) perm[l] = l;
  std::sort(perm.begin(), perm.end(), [&](int a, int b) { return g->pos[headers[a]] < g->pos[headers[b]]; });
  std::vector<int32_t> newid(L);
  for (int k = 0; k < L; ++k) newid[perm[k]] = k;
  g->L = L;
  g->loop_head.resize(L);
  g->loop_parent.resize(L);
  g->loop_depth.resize(L);
  g->loop_end.resize(L);
  g->body_off.assign(L + 1, 0);
  for (int k = 0; k < L; ++k) g->body_off[k + 1] = g->body_off[k] + (int32_t)bodies[perm[k]].size();
  g->body_blk.resize(g->body_off[L]);
  uint8_t split[kParMax] = {};  // a body that is not one run of positions, per thread
  parallel_ranges(L, std::max(1, kParMin / 16), kParMax, [&](int t, int lo, int hi) {
    for (int k = lo; k < hi; ++k) {
      const int l = perm[k];
      g->loop_head[k] = headers[l];
      g->loop_parent[k] = lparent[l] == kNone ? kNone : newid[lparent[l]];
      g->loop_depth[k] = ldepth[l];
      std::vector<int32_t> &bd = bodies[l];  // not needed in build order any more
      std::sort(bd.begin(), bd.end(), [&](int a, int b) { return g->pos[a] < g->pos[b]; });
      const int p0 = g->pos[bd.front()], p1 = g->pos[bd.back()];
      if (bd.front() != headers[l] || p1 - p0 + 1 != (int)bd.size()) split[t] = 1;
      g->loop_end[k] = p1 + 1;
      std::copy(bd.begin(), bd.end(), g->body_blk.begin() + g->body_off[k]);
    }
  });
  g->contiguous = std::none_of(split, split + kParMax, [](uint8_t x) { return x != 0; });
  g->inner_loop.assign(N, kNone);
  for (int b = 0; b < N; ++b)
    if (inner[b] != kNone) g->inner_loop[b] = newid[inner[b]];

  // loop-entry edges: p -> header with p outside the body, by loop and in
  // predecessor order (counted, then filled, in parallel over loops)
  std::vector<int32_t> eid_ent(g->E, kNone), ent_off(L + 1, 0);
  auto is_entry = [&](int k, int q) {
    const int p = psrc[q];
    if (!reach[p]) return false;
    // p outside body(k)  <=>  k is not an ancestor-or-self of inner(p)
    for (int x = g->inner_loop[p]; x != kNone; x = g->loop_parent[x])
      if (x == k) return false;
    return true;
  };
  const int loops_per_thread = std::max(1, kParMin / 16);
  parallel_ranges(L, loops_per_thread, kParMax, [&](int, int lo, int hi) {
    for (int k = lo; k < hi; ++k) {
      const int h = g->loop_head[k];
      int n = 0;
      for (int q = po[h]; q < po[h + 1]; ++q) n += is_entry(k, q);
      ent_off[k + 1] = n;
    }
  });
  for (int k = 0; k < L; ++k) ent_off[k + 1] += ent_off[k];
  g->K = ent_off[L];
  g->ent_loop.resize(g->K);
  g->ent_src.resize(g->K);
  g->ent_eid.resize(g->K);
  parallel_ranges(L, loops_per_thread, kParMax, [&](int, int lo, int hi) {
    for (int k = lo; k < hi; ++k) {
      const int h = g->loop_head[k];
      int x = ent_off[k];
      for (int q = po[h]; q < po[h + 1]; ++q) {
        if (!is_entry(k, q)) continue;
        eid_ent[peid[q]] = x;
        g->ent_loop[x] = k;
        g->ent_src[x] = psrc[q];
        g->ent_eid[x] = peid[q];
        ++x;
      }
    }
  });

  if (all_edges) {
    // eager `to' placement: a constant may sit on any edge, so every
    // reachable edge gets an entry (after the loop-entry ones, in position
    // order of the edge's target)
    for (int i = 0; i < M; ++i) {
      const int b = g->order[i];
      for (int q = po[b]; q < po[b + 1]; ++q) {
        if (!reach[psrc[q]] || eid_ent[peid[q]] != kNone) continue;
        eid_ent[peid[q]] = g->K++;
        g->ent_loop.push_back(kNone);
        g->ent_src.push_back(psrc[q]);
        g->ent_eid.push_back(peid[q]);
      }
    }
  }
  g->ent_rx.assign(g->K, 0);
  if (data_region && c->region) find_data_region(c, g, so, succ, po, psrc, peid, reach, pre, dfn, idom, dominates,
                                                 &eid_ent);
  g->ent_dst.resize(g->K);
  for (int k = 0; k < g->K; ++k) g->ent_dst[k] = succ[g->ent_eid[k]];

  // position-ordered edge lists (counted, then filled, in parallel over positions)
  trace.next("ingest: edge lists", M);
  g->fin_off.assign(M + 1, 0);
  g->out_off.assign(M + 1, 0);
  g->is_exit.assign(M, 0);
  parallel_ranges(M, kParMin, kParMax, [&](int, int lo, int hi) {
    for (int i = lo; i < hi; ++i) {
      const int b = g->order[i];
      int n = 0;
      for (int q = po[b]; q < po[b + 1]; ++q) n += reach[psrc[q]];
      g->fin_off[i + 1] = n;
      g->out_off[i + 1] = so[b + 1] - so[b];
      g->is_exit[i] = so[b] == so[b + 1];
    }
  });
  for (int i = 0; i < M; ++i) {
    g->fin_off[i + 1] += g->fin_off[i];
    g->out_off[i + 1] += g->out_off[i];
  }
  g->fin_src.resize(g->fin_off[M]);
  g->fin_eid.resize(g->fin_off[M]);
  g->fin_ent.resize(g->fin_off[M]);
  g->out_dst.resize(g->out_off[M]);
  parallel_ranges(M, kParMin, kParMax, [&](int, int lo, int hi) {
    for (int i = lo; i < hi; ++i) {
      const int b = g->order[i];
      int x = g->fin_off[i];
      for (int q = po[b]; q < po[b + 1]; ++q) {
        if (!reach[psrc[q]]) continue;
        g->fin_src[x] = psrc[q];
        g->fin_eid[x] = peid[q];
        g->fin_ent[x] = eid_ent[peid[q]];
        ++x;
      }
      std::copy(succ + so[b], succ + so[b + 1], g->out_dst.begin() + g->out_off[i]);
    }
  });
  g->exit_blocks.clear();
  for (int b = 0; b < N; ++b)
    if (reach[b] && so[b] == so[b + 1]) g->exit_blocks.push_back(b);
  g->chunk_off.assign({0, M});
  g->max_chunk = M;
  g->cfg_pos_off.assign({0, M});
  g->cfg_blk_off.assign({0, N});
  return OMPDART_OK;
}

void concat_ingests(const std::vector<const Ingest *> &parts, Ingest *o) {
  *o = Ingest();
  // every part's offsets first, then the parts copied in parallel
  struct Off {
    int64_t n, e, m, l, k, fin, out, x, body;
  };
  const int P = (int)parts.size();
  std::vector<Off> off(P + 1, Off{0, 0, 0, 0, 0, 0, 0, 0, 0});
  for (int q = 0; q < P; ++q) {
    const Ingest *g = parts[q];
    off[q + 1] = Off{off[q].n + g->N, off[q].e + g->E, off[q].m + g->M, off[q].l + g->L, off[q].k + g->K,
                     off[q].fin + (int64_t)g->fin_src.size(), off[q].out + (int64_t)g->out_dst.size(),
                     off[q].x + (int64_t)g->exit_blocks.size(), off[q].body + (int64_t)g->body_blk.size()};
    o->A += g->A;
    o->V = g->V;
    o->W = g->W;
    o->reducible = o->reducible && g->reducible;
    o->contiguous = o->contiguous && g->contiguous;
  }
  const Off &t = off[P];
  o->N = (int)t.n;
  o->E = (int)t.e;
  o->M = (int)t.m;
  o->L = (int)t.l;
  o->K = (int)t.k;
  o->order.resize(t.m);
  o->pos.resize(t.n);
  o->fin_off.resize(t.m + 1);
  o->fin_src.resize(t.fin);
  o->fin_eid.resize(t.fin);
  o->fin_ent.resize(t.fin);
  o->out_off.resize(t.m + 1);
  o->out_dst.resize(t.out);
  o->is_exit.resize(t.m);
  o->exit_blocks.resize(t.x);
  o->loop_head.resize(t.l);
  o->loop_parent.resize(t.l);
  o->loop_depth.resize(t.l);
  o->loop_end.resize(t.l);
  o->body_off.resize(t.l + 1);
  o->body_blk.resize(t.body);
  o->inner_loop.resize(t.n);
  o->ent_loop.resize(t.k);
  o->ent_src.resize(t.k);
  o->ent_eid.resize(t.k);
  o->ent_dst.resize(t.k);
  o->ent_rx.resize(t.k);
  o->cfg_pos_off.resize(P + 1);
  o->cfg_blk_off.resize(P + 1);
  for (int q = 0; q <= P; ++q) o->cfg_blk_off[q] = (int32_t)off[q].n;
  // region mode: per-CFG regions laid end to end (a part without kernels
  // or without the mode contributes an empty region)
  for (int q = 0; q < P; ++q) o->region_mode = o->region_mode || parts[q]->region_mode;
  std::vector<int32_t> kern_base(P + 1, 0), rin_base(P + 1, 0), rout_base(P + 1, 0);
  if (o->region_mode) {
    for (int q = 0; q < P; ++q) {
      const Ingest *g = parts[q];
      kern_base[q + 1] = kern_base[q] + (g->region_mode ? g->kern_off.back() : 0);
      rin_base[q + 1] = rin_base[q] + (int32_t)g->rin_eid.size();
      rout_base[q + 1] = rout_base[q] + (int32_t)g->rout_eid.size();
    }
    o->in_region.assign(t.n, 0);
    o->kernel.assign(t.n, -1);
    o->kern_off = kern_base;
    o->rin_eid.resize(rin_base[P]);
    o->rout_eid.resize(rout_base[P]);
    o->rin_off = rin_base;
    o->rout_off = rout_base;
    o->start_kernel.assign(P, -1);
    o->entry_in_region.assign(P, 0);
  }
  o->fin_off[t.m] = (int32_t)t.fin;
  o->out_off[t.m] = (int32_t)t.out;
  o->body_off[t.l] = (int32_t)t.body;
  o->cfg_pos_off[P] = (int32_t)t.m;
  parallel_ranges(P, 64, 8, [&](int, int lo_p, int hi_p) {
    for (int q = lo_p; q < hi_p; ++q) {
      const Ingest *g = parts[q];
      const Off &f = off[q];
      const int bo = (int)f.n, eo = (int)f.e, po = (int)f.m, lo = (int)f.l, ko = (int)f.k;
      o->cfg_pos_off[q] = po;
      for (int i = 0; i < g->M; ++i) {
        o->order[po + i] = g->order[i] + bo;
        o->fin_off[po + i] = g->fin_off[i] + (int32_t)f.fin;
        o->out_off[po + i] = g->out_off[i] + (int32_t)f.out;
        o->is_exit[po + i] = g->is_exit[i];
      }
      for (int b = 0; b < g->N; ++b) {
        o->pos[bo + b] = g->pos[b] < 0 ? -1 : g->pos[b] + po;
        o->inner_loop[bo + b] = g->inner_loop[b] < 0 ? -1 : g->inner_loop[b] + lo;
      }
      for (size_t k = 0; k < g->fin_src.size(); ++k) {
        o->fin_src[f.fin + k] = g->fin_src[k] + bo;
        o->fin_eid[f.fin + k] = g->fin_eid[k];  // edge ids stay local to their CFG
        o->fin_ent[f.fin + k] = g->fin_ent[k] < 0 ? -1 : g->fin_ent[k] + ko;
      }
      for (size_t k = 0; k < g->out_dst.size(); ++k) o->out_dst[f.out + k] = g->out_dst[k] + bo;
      for (size_t k = 0; k < g->exit_blocks.size(); ++k) o->exit_blocks[f.x + k] = g->exit_blocks[k] + bo;
      for (int l = 0; l < g->L; ++l) {
        o->loop_head[lo + l] = g->loop_head[l] + bo;
        o->loop_parent[lo + l] = g->loop_parent[l] < 0 ? -1 : g->loop_parent[l] + lo;
        o->loop_depth[lo + l] = g->loop_depth[l];
        o->loop_end[lo + l] = g->loop_end[l] + po;
        o->body_off[lo + l] = g->body_off[l] + (int32_t)f.body;
      }
      for (size_t k = 0; k < g->body_blk.size(); ++k) o->body_blk[f.body + k] = g->body_blk[k] + bo;
      for (int k = 0; k < g->K; ++k) {
        o->ent_loop[ko + k] = g->ent_loop[k] < 0 ? -1 : g->ent_loop[k] + lo;
        o->ent_src[ko + k] = g->ent_src[k] + bo;
        o->ent_eid[ko + k] = g->ent_eid[k] + eo;
        o->ent_dst[ko + k] = g->ent_dst[k] + bo;
        o->ent_rx[ko + k] = g->ent_rx[k];
      }
      if (o->region_mode && g->region_mode) {
        std::copy(g->in_region.begin(), g->in_region.end(), o->in_region.begin() + bo);
        std::copy(g->kernel.begin(), g->kernel.end(), o->kernel.begin() + bo);
        std::copy(g->rin_eid.begin(), g->rin_eid.end(), o->rin_eid.begin() + rin_base[q]);
        std::copy(g->rout_eid.begin(), g->rout_eid.end(), o->rout_eid.begin() + rout_base[q]);
        o->start_kernel[q] = g->start_kernel[0];
        o->entry_in_region[q] = g->entry_in_region[0];
      }
    }
  });
  o->entry = parts.empty() ? 0 : parts[0]->entry;
  o->chunk_off.assign({0, o->M});
  o->max_chunk = o->M;
}

// Single-entry cut before position i (0 < i < M): every edge that crosses
// it (source before i, target at or after i) targets order[i], and no edge
// goes from at-or-after i back to before i.  Then the whole influence of
// positions < i on positions >= i is one value -- the one entering order[i]
// -- and the same holds for the backward problem in the other direction.
void make_chunks(Ingest *g, int target) {
  const int M = g->M;
  g->chunk_off.clear();
  g->chunk_off.push_back(0);
  if (target <= 0) target = M + 1;  // one chunk per CFG
  // fwd[i]: edges with pos(src) < i <= pos(dst), counted by difference
  // arrays; into[i]: edges into order[i] from positions < i; back[i]:
  // edges with pos(dst) < i <= pos(src).  Positions in parallel, the
  // counts by atomic adds (most land next to the position's own).
  std::vector<int32_t> fwd(M + 1, 0), back(M + 1, 0), into(M, 0);  // counts of edges: below 2^31
  auto add = [](auto *x, auto v) { __atomic_fetch_add(x, v, __ATOMIC_RELAXED); };
  parallel_ranges(M, kParMin, kParMax, [&](int, int lo, int hi) {
    for (int j = lo; j < hi; ++j) {
      for (int k = g->out_off[j]; k < g->out_off[j + 1]; ++k) {
        const int pd = g->pos[g->out_dst[k]];
        if (pd > j) {
          add(&fwd[j + 1], 1);
          add(&fwd[pd + 1], -1);
          add(&into[pd], 1);
        } else {
          add(&back[pd + 1], 1);
          add(&back[j + 1], -1);
        }
      }
    }
  });
  std::vector<uint8_t> ok(M + 1, 0);
  int32_t f = 0, bk = 0;
  for (int i = 0; i <= M; ++i) {
    f += fwd[i];
    bk += back[i];
    if (i > 0 && i < M) ok[i] = (bk == 0) && (f == into[i]);
  }
  // the boundaries between the CFGs of a batch are always cuts (no edge
  // crosses them)
  std::vector<uint8_t> force(M + 1, 0);
  for (int x : g->cfg_pos_off)
    if (x > 0 && x < M) force[x] = 1;
  int start = 0;
  g->max_chunk = 0;
  for (int i = 1; i < M; ++i) {
    if (force[i] || (ok[i] && i - start >= target)) {
      g->chunk_off.push_back(i);
      g->max_chunk = std::max(g->max_chunk, i - start);
      start = i;
    }
  }
  g->chunk_off.push_back(M);
  g->max_chunk = std::max(g->max_chunk, M - start);
}

}  // namespace ompdart
