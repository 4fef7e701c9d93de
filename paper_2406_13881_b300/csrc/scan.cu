// scan.cu -- chunked scan solver (placeholder until the fast path lands).
#include <string>

#include "ingest.h"
#include "plan.cuh"

namespace ompdart {
struct ScanState {};
int scan_supported(const Ingest &) { return 0; }
ScanState *scan_create(const Ingest &, DevPlan &, cudaStream_t, std::string *err) {
  if (err) *err = "scan solver unavailable";
  return nullptr;
}
int enqueue_scan_solver(ScanState *, const DevPlan &, cudaStream_t) { return 0; }
int enqueue_scan_edges(ScanState *, const DevPlan &, cudaStream_t) { return 0; }
void scan_destroy(ScanState *st) { delete st; }
}  // namespace ompdart
