// program.cpp -- interprocedural analysis of a whole program
// (ompdart_analyze_program): callee summaries bottom-up, then every
// function analysed top-down in the contexts its call sites give it
// (Sec. IV-C side effects at call sites; Sec. IV-D per function).
//
//   1. heights in the call DAG (a leaf is 0; recursion is rejected);
//   2. bottom-up, one device run per height: each function's call table
//      row for a site is its callee's summary mapped into the function's
//      numbering (map_summary), then all functions of the height are
//      summarised together (summarize_run);
//   3. top-down, one batch per height (highest first, so every caller is
//      done before its callees): a root runs in its own boundary rows; a
//      called function runs once per distinct context its call sites pass
//      on.  A site's context per caller instance is the caller's state at
//      the call (validity the callee starts from, liveness after the call)
//      mapped into the callee's numbering; a site passes on at most
//      max_contexts of them (sorted, the excess merged into the last by the
//      meet: validity AND, liveness OR), except that a context whose meet
//      would leave a variable valid nowhere that either holds somewhere
//      stays a context of its own.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/ompdart.h"
#include "solver.h"

using namespace ompdart;

namespace {

typedef std::vector<uint64_t> Row;

struct Ctx {  // one context: rows in the callee's numbering
  Row eh, ed, xl;
  bool operator<(const Ctx &o) const {
    if (eh != o.eh) return eh < o.eh;
    if (ed != o.ed) return ed < o.ed;
    return xl < o.xl;
  }
  bool operator==(const Ctx &o) const { return eh == o.eh && ed == o.ed && xl == o.xl; }
};

int words(int n_vars) { return (n_vars + 63) / 64; }

// caller rows -> callee rows through var_map (callee v denotes caller
// var_map[v]); a callee variable that denotes nothing of the caller (a
// local) starts valid on the host only and is dead after the exit
Ctx map_context(const uint64_t *eh, const uint64_t *ed, const uint64_t *xl, const int32_t *var_map, int callee_vars,
                int caller_vars) {
  const int W = words(callee_vars);
  Ctx c{Row(W, 0), Row(W, 0), Row(W, 0)};
  for (int v = 0; v < callee_vars; ++v) {
    const int t = var_map ? var_map[v] : v;
    const uint64_t b = 1ull << (v & 63);
    if (t < 0 || t >= caller_vars) {
      c.eh[v >> 6] |= b;
      continue;
    }
    const uint64_t tb = 1ull << (t & 63);
    if (eh[t >> 6] & tb) c.eh[v >> 6] |= b;
    if (ed[t >> 6] & tb) c.ed[v >> 6] |= b;
    if (xl[t >> 6] & tb) c.xl[v >> 6] |= b;
  }
  return c;
}

}  // namespace

extern "C" {

void ompdart_program_result_free(ompdart_program_result *r) {
  if (!r) return;
  for (int i = 0; i < r->n_instances; ++i) {
    ompdart_result_free(r->inst[i].result);
    free(r->inst[i].entry_h);
    free(r->inst[i].entry_d);
    free(r->inst[i].exit_live);
  }
  free(r->inst);
  free(r->summaries);
  free(r->summary_off);
  free(r->height);
  free(r->status);
  free(r);
}

int ompdart_analyze_program(const ompdart_program *Pin, const ompdart_opts *opts, ompdart_program_result **out) {
  set_last_error_text("");
  if (!Pin || !out || Pin->n_funcs < 0 || (Pin->n_funcs > 0 && (!Pin->funcs || !Pin->site_off)))
    return set_error(OMPDART_E_INVALID, "bad program");
  // functions given in device memory: their arrays copied to the host first
  StagedCfgs staged;
  ompdart_program prog = *Pin;
  {
    std::string serr;
    const int src = stage_cfgs(Pin->funcs, Pin->n_funcs, &staged, &prog.funcs, &serr);
    if (src) return set_error(src, serr);
  }
  const ompdart_program *P = &prog;
  *out = nullptr;
  ompdart_opts o{};
  if (opts) o = *opts;
  const int F = P->n_funcs;
  const int S = F ? P->site_off[F] : 0;
  const int max_ctx = P->max_contexts > 0 ? P->max_contexts : 4;
  if (S && (!P->site_callee || !P->map_off || !P->var_map)) return set_error(OMPDART_E_INVALID, "bad call sites");
  for (int f = 0; f < F; ++f) {
    if (P->site_off[f + 1] < P->site_off[f]) return set_error(OMPDART_E_INVALID, "site_off must be non-decreasing");
    const ompdart_cfg &c = P->funcs[f];
    if (c.n_blocks < 1 || !c.acc_off || (c.acc_off[c.n_blocks] && !c.acc))
      return set_error(OMPDART_E_INVALID, "bad function CFG");
    const int ns = P->site_off[f + 1] - P->site_off[f];
    for (int i = 0; i < c.acc_off[c.n_blocks]; ++i)
      if ((c.acc[i] >> 31) && (int)(c.acc[i] & 0x7FFFFFFFu) >= ns)
        return set_error(OMPDART_E_INVALID, "call access row beyond the function's call sites");
  }
  for (int s = 0; s < S; ++s) {
    const int g = P->site_callee[s];
    if (g < 0 || g >= F) return set_error(OMPDART_E_INVALID, "call site callee out of range");
    if (P->map_off[s + 1] - P->map_off[s] != P->funcs[g].n_vars)
      return set_error(OMPDART_E_INVALID, "a site's var_map must have one entry per callee variable");
  }
  // ---- 1. heights (iterative DFS; a back edge is recursion)
  std::vector<int32_t> height(F, -1), state(F, 0), has_caller(F, 0);
  for (int s = 0; s < S; ++s) has_caller[P->site_callee[s]] = 1;
  for (int r = 0; r < F; ++r) {
    if (state[r]) continue;
    std::vector<std::pair<int, int>> st{{r, P->site_off[r]}};
    state[r] = 1;
    while (!st.empty()) {
      auto &t = st.back();
      if (t.second < P->site_off[t.first + 1]) {
        const int g = P->site_callee[t.second++];
        if (state[g] == 1) return set_error(OMPDART_E_INVALID, "the call graph has a cycle (recursion)");
        if (!state[g]) {
          state[g] = 1;
          st.push_back({g, P->site_off[g]});
        }
      } else {
        int h = 0;
        for (int s = P->site_off[t.first]; s < P->site_off[t.first + 1]; ++s)
          h = std::max(h, height[P->site_callee[s]] + 1);
        height[t.first] = h;
        state[t.first] = 2;
        st.pop_back();
      }
    }
  }
  const int H = F ? *std::max_element(height.begin(), height.end()) + 1 : 0;
  std::vector<std::vector<int>> at_height(H);
  for (int f = 0; f < F; ++f) at_height[height[f]].push_back(f);
  // ---- 2. summaries bottom-up; call tables of every function
  std::vector<Row> summary(F), table(F);
  std::vector<int32_t> fstatus(F, OMPDART_OK);
  for (int h = 0; h < H; ++h) {
    std::vector<ompdart_cfg> cfgs;
    std::vector<uint64_t *> rows;
    for (int f : at_height[h]) {
      const ompdart_cfg &c = P->funcs[f];
      const int W = words(c.n_vars), ns = P->site_off[f + 1] - P->site_off[f];
      table[f].assign((size_t)std::max(ns, 1) * 7 * W, 0);
      for (int k = 0; k < ns; ++k) {
        const int s = P->site_off[f] + k, g = P->site_callee[s];
        if (fstatus[g]) {
          fstatus[f] = fstatus[g];  // a callee without a summary
          continue;
        }
        map_summary(summary[g].data(), P->funcs[g].n_vars, P->var_map + P->map_off[s], c.n_vars,
                    table[f].data() + (size_t)k * 7 * W);
      }
      summary[f].assign((size_t)7 * W, 0);
      ompdart_cfg cc = c;
      cc.call_planes = ns ? table[f].data() : nullptr;
      cc.n_calls = ns;
      cfgs.push_back(cc);
      rows.push_back(summary[f].data());
    }
    std::vector<int32_t> st(cfgs.size(), OMPDART_OK);
    int rc = summarize_run(cfgs.data(), (int)cfgs.size(), o, rows.data(), st.data());
    if (rc) return rc;
    for (size_t i = 0; i < cfgs.size(); ++i)
      if (st[i] && !fstatus[at_height[h][i]]) fstatus[at_height[h][i]] = st[i];
  }
  // ---- 3. contexts top-down, one batch per height
  std::vector<std::vector<Ctx>> ctxs(F);
  for (int f = 0; f < F; ++f)
    if (!has_caller[f]) {  // a root: its own boundary rows
      const ompdart_cfg &c = P->funcs[f];
      const int W = words(c.n_vars);
      Ctx x{Row(W), Row(W), Row(W)};
      for (int w = 0; w < W; ++w) {
        const uint64_t t = (w == W - 1 && c.n_vars % 64) ? (1ull << (c.n_vars % 64)) - 1 : ~0ull;
        x.eh[w] = (c.entry_host_valid ? c.entry_host_valid[w] : ~0ull) & t;
        x.ed[w] = (c.entry_dev_valid ? c.entry_dev_valid[w] : 0ull) & t;
        x.xl[w] = (c.exit_host_live ? c.exit_host_live[w] : ~0ull) & t;
      }
      ctxs[f].push_back(x);
    }
  std::vector<ompdart_instance> inst;
  for (int h = H - 1; h >= 0; --h) {
    struct Item { int f; Ctx c; };
    std::vector<Item> items;
    for (int f : at_height[h]) {
      std::sort(ctxs[f].begin(), ctxs[f].end());
      ctxs[f].erase(std::unique(ctxs[f].begin(), ctxs[f].end()), ctxs[f].end());
      for (const Ctx &c : ctxs[f]) items.push_back({f, c});
    }
    if (items.empty()) continue;
    std::vector<ompdart_cfg> cfgs(items.size());
    for (size_t i = 0; i < items.size(); ++i) {
      const int f = items[i].f, ns = P->site_off[f + 1] - P->site_off[f];
      cfgs[i] = P->funcs[f];
      cfgs[i].call_planes = ns ? table[f].data() : nullptr;
      cfgs[i].n_calls = ns;
      cfgs[i].entry_host_valid = items[i].c.eh.data();
      cfgs[i].entry_dev_valid = items[i].c.ed.data();
      cfgs[i].exit_host_live = items[i].c.xl.data();
    }
    std::vector<int32_t> st(items.size(), OMPDART_OK);
    std::vector<ompdart_result *> res(items.size(), nullptr);
    int rc = ompdart_analyze_batch(cfgs.data(), (int)items.size(), &o, res.data(), st.data());
    if (rc) {
      for (auto *r : res) ompdart_result_free(r);
      for (auto &x : inst) ompdart_result_free(x.result);
      return rc;
    }
    // contexts each site passes on, per callee
    std::map<int, std::vector<Ctx>> per_site;  // site -> contexts (callee numbering)
    for (size_t i = 0; i < items.size(); ++i) {
      const int f = items[i].f;
      const ompdart_cfg &c = P->funcs[f];
      const int W = words(c.n_vars);
      ompdart_instance x{};
      x.func = f;
      x.status = st[i] ? st[i] : fstatus[f];
      x.result = res[i];
      x.entry_h = (uint64_t *)malloc(sizeof(uint64_t) * W);
      x.entry_d = (uint64_t *)malloc(sizeof(uint64_t) * W);
      x.exit_live = (uint64_t *)malloc(sizeof(uint64_t) * W);
      if (x.entry_h) memcpy(x.entry_h, items[i].c.eh.data(), sizeof(uint64_t) * W);
      if (x.entry_d) memcpy(x.entry_d, items[i].c.ed.data(), sizeof(uint64_t) * W);
      if (x.exit_live) memcpy(x.exit_live, items[i].c.xl.data(), sizeof(uint64_t) * W);
      inst.push_back(x);
      if (!res[i]) continue;
      const ompdart_result &r = *res[i];
      for (int j = 0; j < r.n_call_sites; ++j) {
        const int k = (int)(c.acc[r.call_site_acc[j]] & 0x7FFFFFFFu);
        const int s = P->site_off[f] + k, g = P->site_callee[s];
        per_site[s].push_back(map_context(r.call_entry_h + (size_t)j * W, r.call_entry_d + (size_t)j * W,
                                          r.call_exit_live + (size_t)j * W, P->var_map + P->map_off[s],
                                          P->funcs[g].n_vars, c.n_vars));
      }
    }
    for (auto &kv : per_site) {
      std::vector<Ctx> &v = kv.second;
      std::sort(v.begin(), v.end());
      v.erase(std::unique(v.begin(), v.end()), v.end());
      if ((int)v.size() > max_ctx) {
        // merge the excess into the last kept one by the meet, except a
        // context whose meet would leave a variable valid nowhere that one
        // of the two holds somewhere: it stays a context of its own
        Ctx m = v[max_ctx - 1];
        std::vector<Ctx> alone;
        const size_t Wn = m.eh.size();
        for (size_t e = max_ctx; e < v.size(); ++e) {
          const Ctx &c = v[e];
          Ctx t{Row(Wn), Row(Wn), Row(Wn)};
          bool hole = false;
          for (size_t w = 0; w < Wn; ++w) {
            t.eh[w] = m.eh[w] & c.eh[w];
            t.ed[w] = m.ed[w] & c.ed[w];
            t.xl[w] = m.xl[w] | c.xl[w];
            hole |= ((m.eh[w] | m.ed[w] | c.eh[w] | c.ed[w]) & ~(t.eh[w] | t.ed[w])) != 0;
          }
          if (hole)
            alone.push_back(c);
          else
            m = std::move(t);
        }
        v.resize(max_ctx - 1);
        v.push_back(std::move(m));
        v.insert(v.end(), alone.begin(), alone.end());
      }
      const int g = P->site_callee[kv.first];
      ctxs[g].insert(ctxs[g].end(), v.begin(), v.end());
    }
  }
  // ---- result
  ompdart_program_result *R = (ompdart_program_result *)calloc(1, sizeof(ompdart_program_result));
  if (!R) return set_error(OMPDART_E_NOMEM, "host allocation failed");
  R->n_instances = (int32_t)inst.size();
  R->inst = (ompdart_instance *)calloc(std::max<size_t>(inst.size(), 1), sizeof(ompdart_instance));
  R->summary_off = (int64_t *)calloc(std::max(F, 1), sizeof(int64_t));
  R->height = (int32_t *)calloc(std::max(F, 1), sizeof(int32_t));
  R->status = (int32_t *)calloc(std::max(F, 1), sizeof(int32_t));
  size_t tot = 0;
  for (int f = 0; f < F; ++f) tot += summary[f].size();
  R->summaries = (uint64_t *)calloc(std::max<size_t>(tot, 1), sizeof(uint64_t));
  R->levels = H;
  if (!R->inst || !R->summary_off || !R->height || !R->status || !R->summaries) {
    for (auto &x : inst) ompdart_result_free(x.result);
    ompdart_program_result_free(R);
    return set_error(OMPDART_E_NOMEM, "host allocation failed");
  }
  std::copy(inst.begin(), inst.end(), R->inst);
  size_t off = 0;
  for (int f = 0; f < F; ++f) {
    R->summary_off[f] = (int64_t)off;
    std::copy(summary[f].begin(), summary[f].end(), R->summaries + off);
    off += summary[f].size();
    R->height[f] = height[f];
    R->status[f] = fstatus[f];
  }
  *out = R;
  return OMPDART_OK;
}

}  // extern "C"
