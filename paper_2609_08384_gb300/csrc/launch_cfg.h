// Per-device, thread-safe record of the one-time launch configuration of a
// kernel (its dynamic shared-memory limit).
//
// cudaFuncSetAttribute acts on the current device only, so a kernel that
// needs more than 48 KB of dynamic shared memory must be configured once on
// every device it runs on.  The record is one bit per device (devices 0..63;
// any other device is configured before every launch) in an atomic word, so
// host threads launching concurrently never read a torn flag; two threads may
// both set the attribute on a first launch, which is harmless.  The attribute
// belongs to the device's context: after cudaDeviceReset the record is stale
// and a launch that needs the raised limit fails with an error (it does not
// fault); such a process must not launch through this library again.
#pragma once

#include <atomic>

#include <cuda_runtime.h>

namespace brahms {

struct SmemOnce {
  std::atomic<unsigned long long> mask{0};
};

template <class K>
inline cudaError_t raise_smem_limit(K kernel, size_t smem, SmemOnce& once) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ULL << dev) : 0ULL;
  if (bit && (once.mask.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && bit) once.mask.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// The same for a kernel launched with varying shared memory: the largest
// limit set so far on each device.
struct SmemMax {
  std::atomic<size_t> bytes[64] = {};
};

template <class K>
inline cudaError_t raise_smem_limit_to(K kernel, size_t smem, SmemMax& rec) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool tracked = dev >= 0 && dev < 64;
  if (tracked && rec.bytes[dev].load(std::memory_order_acquire) >= smem) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && tracked) {
    size_t cur = rec.bytes[dev].load(std::memory_order_acquire);
    while (cur < smem && !rec.bytes[dev].compare_exchange_weak(cur, smem, std::memory_order_acq_rel)) {
    }
  }
  return e;
}

}  // namespace brahms
