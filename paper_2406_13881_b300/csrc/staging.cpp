// staging.cpp -- CFGs whose arrays live in device memory (ompdart_cfg.mem =
// OMPDART_MEM_DEVICE).  Ingestion (validation, orderings, dominators,
// loops; Sec. IV-B) runs on the host, so the entry points copy such a
// CFG's arrays into host buffers first and hand the copies on.  A device
// array that several CFGs share (one function analysed in several calling
// contexts) is copied once, so those CFGs keep sharing one ingestion.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <unordered_map>

#include "solver.h"

namespace ompdart {

namespace {

int stage_fail(std::string *err, const std::string &msg) {
  if (err) *err = msg;
  return OMPDART_E_INVALID;
}

bool on_device(const void *p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// host copy of `bytes' bytes at device address p (one copy per distinct
// (address, size)); nullptr with *rc set on failure
const void *copy_in(StagedCfgs *st, const void *p, size_t bytes, const char *what, int *rc, std::string *err) {
  if (!p) return nullptr;
  auto key = std::make_pair(p, bytes);
  auto it = st->seen.find(key);
  if (it != st->seen.end()) return it->second;
  if (!on_device(p)) {
    *rc = stage_fail(err, std::string("mem = OMPDART_MEM_DEVICE but ") + what + " is not device memory");
    return nullptr;
  }
  st->bufs.emplace_back(bytes ? bytes : 1);
  void *h = st->bufs.back().data();
  if (bytes) {
    const cudaError_t ce = cudaMemcpy(h, p, bytes, cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) {
      (void)cudaGetLastError();
      *rc = OMPDART_E_CUDA;
      if (err) *err = std::string("copying ") + what + " from the device: " + cudaGetErrorString(ce);
      return nullptr;
    }
  }
  st->seen.emplace(key, h);
  return h;
}

int stage_one(const ompdart_cfg &in, StagedCfgs *st, ompdart_cfg *out, std::string *err) {
  *out = in;
  out->mem = OMPDART_MEM_HOST;
  if (in.n_blocks < 1 || in.n_vars < 1 || !in.succ_off || !in.acc_off)
    return stage_fail(err, "malformed CFG header");
  const size_t N = (size_t)in.n_blocks, W = (size_t)(in.n_vars + 63) / 64;
  int rc = OMPDART_OK;
  auto so = static_cast<const int32_t *>(copy_in(st, in.succ_off, (N + 1) * 4, "succ_off", &rc, err));
  if (rc) return rc;
  auto ao = static_cast<const int32_t *>(copy_in(st, in.acc_off, (N + 1) * 4, "acc_off", &rc, err));
  if (rc) return rc;
  const long long E = so[N], A = ao[N];
  if (E < 0 || A < 0) return stage_fail(err, "malformed CSR (negative edge or access count)");
  if ((E && !in.succ) || (A && !in.acc)) return stage_fail(err, "malformed CSR (NULL successor or access array)");
  out->succ_off = so;
  out->acc_off = ao;
  out->succ = static_cast<const int32_t *>(copy_in(st, in.succ, (size_t)E * 4, "succ", &rc, err));
  if (rc) return rc;
  out->acc = static_cast<const uint32_t *>(copy_in(st, in.acc, (size_t)A * 4, "acc", &rc, err));
  if (rc) return rc;
  out->entry_host_valid =
      static_cast<const uint64_t *>(copy_in(st, in.entry_host_valid, W * 8, "entry_host_valid", &rc, err));
  if (rc) return rc;
  out->entry_dev_valid =
      static_cast<const uint64_t *>(copy_in(st, in.entry_dev_valid, W * 8, "entry_dev_valid", &rc, err));
  if (rc) return rc;
  out->exit_host_live =
      static_cast<const uint64_t *>(copy_in(st, in.exit_host_live, W * 8, "exit_host_live", &rc, err));
  if (rc) return rc;
  if (in.call_planes && in.n_calls > 0)
    out->call_planes = static_cast<const uint64_t *>(
        copy_in(st, in.call_planes, (size_t)in.n_calls * 7 * W * 8, "call_planes", &rc, err));
  if (rc) return rc;
  out->region = static_cast<const int32_t *>(copy_in(st, in.region, N * 4, "region", &rc, err));
  if (rc) return rc;
  out->scalar_vars = static_cast<const uint64_t *>(copy_in(st, in.scalar_vars, W * 8, "scalar_vars", &rc, err));
  return rc;
}

}  // namespace

int stage_cfgs(const ompdart_cfg *in, int n, StagedCfgs *st, const ompdart_cfg **out, std::string *err,
               bool per_cfg) {
  *out = in;
  bool any = false;
  for (int i = 0; i < n; ++i) any |= in[i].mem != OMPDART_MEM_HOST;
  if (!any) return OMPDART_OK;
  st->cfgs.assign(in, in + n);
  st->rc.assign(n, OMPDART_OK);
  st->err.assign(n, std::string());
  for (int i = 0; i < n; ++i) {
    if (in[i].mem == OMPDART_MEM_HOST) continue;
    int rc = in[i].mem == OMPDART_MEM_DEVICE
                 ? stage_one(in[i], st, &st->cfgs[i], &st->err[i])
                 : stage_fail(&st->err[i], "mem must be OMPDART_MEM_HOST or OMPDART_MEM_DEVICE");
    if (rc) {
      if (!per_cfg) {
        if (err) *err = st->err[i];
        return rc;
      }
      st->rc[i] = rc;
      st->cfgs[i] = ompdart_cfg{};  // rejected by ingestion; the caller reports rc[i]
      st->cfgs[i].n_blocks = -1;
    }
  }
  *out = st->cfgs.data();
  return OMPDART_OK;
}

int firstprivate_view(const ompdart_cfg &in, StagedCfgs *st, ompdart_cfg *out, std::vector<uint64_t> *fp,
                      int *n_kernels, std::string *err) {
  *out = in;
  fp->clear();
  *n_kernels = 0;
  if (!in.region) return OMPDART_OK;
  const int N = in.n_blocks, W = (in.n_vars + 63) / 64;
  int nk = 0;
  for (int b = 0; b < N; ++b) {
    if (in.region[b] < -1 || in.region[b] >= N) {
      if (err) *err = "kernel ids (region) must be -1 or in [0, n_blocks)";
      return OMPDART_E_INVALID;
    }
    nk = std::max(nk, in.region[b] + 1);
  }
  *n_kernels = nk;
  fp->assign((size_t)nk * W, 0);
  if (!in.scalar_vars || !nk) return OMPDART_OK;
  auto scalar = [&](int v) { return (in.scalar_vars[v >> 6] >> (v & 63)) & 1ull; };
  // per (kernel, scalar): bit 1 read on the device, bit 2 written (either space)
  std::unordered_map<long long, uint8_t> use;
  for (int b = 0; b < N; ++b) {
    const int k = in.region[b];
    if (k < 0) continue;
    for (int i = in.acc_off[b]; i < in.acc_off[b + 1]; ++i) {
      const uint32_t a = in.acc[i];
      const int v = (int)(a & 0xFFFFFFu);
      if ((a >> 31) || !scalar(v)) continue;
      uint8_t &u = use[(long long)k * in.n_vars + v];
      const int kind = (int)((a >> 24) & 3u);
      if (kind & 2) u |= 2;
      if ((kind & 1) && ((a >> 26) & 1u)) u |= 1;
    }
  }
  bool any = false;
  for (const auto &kv : use)
    if (kv.second == 1) {
      const int k = (int)(kv.first / in.n_vars), v = (int)(kv.first % in.n_vars);
      (*fp)[(size_t)k * W + (v >> 6)] |= 1ull << (v & 63);
      any = true;
    }
  if (!any) return OMPDART_OK;
  const size_t A = (size_t)in.acc_off[N];
  st->bufs.emplace_back(std::max<size_t>(A, 1) * 4);
  uint32_t *acc = reinterpret_cast<uint32_t *>(st->bufs.back().data());
  std::memcpy(acc, in.acc, A * 4);
  for (int b = 0; b < N; ++b) {
    const int k = in.region[b];
    if (k < 0) continue;
    for (int i = in.acc_off[b]; i < in.acc_off[b + 1]; ++i) {
      const uint32_t a = acc[i];
      const int v = (int)(a & 0xFFFFFFu);
      if ((a >> 31) || !((a >> 26) & 1u) || !scalar(v)) continue;
      if (((*fp)[(size_t)k * W + (v >> 6)] >> (v & 63)) & 1ull) acc[i] = a & ~(1u << 26);  // a host read
    }
  }
  out->acc = acc;
  return OMPDART_OK;
}

}  // namespace ompdart
