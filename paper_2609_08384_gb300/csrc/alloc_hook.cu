// Allocation entry points with the failure hook of brahms_fail_next_allocations.
#include <atomic>

#include "alloc_hook.h"
#include "brahms.h"

namespace {
std::atomic<int> g_fail_next{0};

// true if this allocation is one of those asked to fail
bool take_failure() {
  int n = g_fail_next.load(std::memory_order_acquire);
  while (n > 0) {
    if (g_fail_next.compare_exchange_weak(n, n - 1, std::memory_order_acq_rel)) return true;
  }
  return false;
}
}  // namespace

namespace brahms {

cudaError_t dev_alloc(void** p, size_t bytes) {
  if (take_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

cudaError_t pinned_alloc(void** p, size_t bytes) {
  if (take_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost(p, bytes);
}

}  // namespace brahms

extern "C" brahms_status brahms_fail_next_allocations(int count) {
  if (count < 0) return BRAHMS_E_ARG;
  g_fail_next.store(count, std::memory_order_release);
  return BRAHMS_OK;
}

extern "C" int brahms_pending_allocation_failures(void) { return g_fail_next.load(std::memory_order_acquire); }
