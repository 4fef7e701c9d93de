// staging.cpp -- CFGs whose arrays live in device memory (ompdart_cfg.mem =
// OMPDART_MEM_DEVICE).  Ingestion (validation, orderings, dominators,
// loops; Sec. IV-B) runs on the host, so the entry points copy such a
// CFG's arrays into host buffers first and hand the copies on.  A device
// array that several CFGs share (one function analysed in several calling
// contexts) is copied once, so those CFGs keep sharing one ingestion.
#include <cuda_runtime.h>

#include <cstring>
#include <string>

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

}  // namespace ompdart
