// Allocation-free variant of the per-field energy reduction.
//
// brahms_energy() reduces into per-block partial sums kept in the context's
// workspace.  Some callers cannot give the library any device memory of its
// own: hosts whose device memory is entirely owned by another allocator,
// plugin environments that forbid a library from calling cudaMalloc, and
// latency-critical loops that cannot afford cudaMalloc/cudaFree (which may
// synchronise the whole device).  brahms_energy_static() serves them: the
// caller passes the fields and a device output array, and the partial sums
// live in the fixed array below, which every GPU that loads this library
// holds until the process exits.
#include <cmath>
#include <mutex>

#include <cuda.h>
#include <cuda_runtime.h>

#include "brahms.h"

namespace {

constexpr int kStaticFields = 3;     // at most this many fields per call
constexpr int kStaticBlocks = 1024;  // partial sums per field
constexpr int kStaticThreads = 256;

// 3 x 1024 doubles = 24 KiB of device memory per GPU.
static __device__ __align__(256) double g_energy_scratch[kStaticFields * kStaticBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // context the address belongs to (0: unknown)

// Identity of the calling thread's current CUDA context, through the driver
// entry points (no link against libcuda); false if none is current yet or
// the entry points are missing.
bool current_context_id(unsigned long long* id) {
  typedef CUresult (*GetCurrentFn)(CUcontext*);
  typedef CUresult (*GetIdFn)(CUcontext, unsigned long long*);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetIdFn>(p);
    cudaGetLastError();
  });
  if (!get_current || !get_id) return false;
  CUcontext c = nullptr;
  if (get_current(&c) != CUDA_SUCCESS || !c) return false;
  return get_id(c, id) == CUDA_SUCCESS;
}

// Device address of g_energy_scratch on the current device (the name is only
// a host-side handle).  It is looked up once per device, and again when the
// device's context is not the one the address was taken in: a
// cudaDeviceReset destroys the context and the library's module with it, and
// the module loads at a new address in the next context.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  unsigned long long id = 0;
  bool have_id = current_context_id(&id);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev] || !have_id || g_scratch_ctx[dev] != id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_energy_scratch);
    if (e != cudaSuccess) return e;
    if (!have_id) have_id = current_context_id(&id);  // the lookup made the device's context current
    g_scratch_ptr[dev] = static_cast<double*>(p);
    g_scratch_ctx[dev] = have_id ? id : 0;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

struct StaticFields {
  const float2* f[kStaticFields];
};

__device__ __forceinline__ double warp_sum_static(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double block_sum_static(double s) {
  __shared__ double red[kStaticThreads / 32];
  s = warp_sum_static(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double v = 0.0;
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    v = warp_sum_static(v);
  }
  return v;
}

// partial[f * nblocks + b] = sum over this block's grid-stride share of |A_f|^2
__global__ void __launch_bounds__(kStaticThreads)
    energy_static_partial_kernel(StaticFields fs, long long n, double* partial) {
  const float2* a = fs.f[blockIdx.y];
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 v = a[i];
    s = fma((double)v.x, (double)v.x, fma((double)v.y, (double)v.y, s));
  }
  s = block_sum_static(s);
  if (threadIdx.x == 0) partial[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// out[f] = weight[f] * sum of the nblocks partials of field f
struct StaticWeights {
  double w[kStaticFields];
};
__global__ void __launch_bounds__(kStaticThreads)
    energy_static_final_kernel(const double* partial, int nblocks, StaticWeights w, double* out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) s += partial[blockIdx.x * nblocks + i];
  s = block_sum_static(s);
  if (threadIdx.x == 0) out[blockIdx.x] = w.w[blockIdx.x] * s;
}

}  // namespace

extern "C" brahms_status brahms_energy_static(const void* const* fields, int nfields, int nx, int ny, int nt,
                                              double dx, double dy, double dt, const brahms_field_params* fp,
                                              double* energy_j_dev, void* cuda_stream) {
  if (!fields || !fp || !energy_j_dev) return BRAHMS_E_ARG;
  if (nfields < 1 || nfields > kStaticFields) return BRAHMS_E_SIZE;
  if (nx < 1 || ny < 1 || nt < 1) return BRAHMS_E_ARG;
  const long long n = (long long)nx * ny * nt;
  if (n > (1LL << 40)) return BRAHMS_E_SIZE;
  if (!(dx > 0) || !(dy > 0) || !(dt > 0)) return BRAHMS_E_ARG;
  StaticFields fs{};
  StaticWeights w{};
  const double c0 = 299792458.0, eps0 = 8.8541878128e-12;
  for (int f = 0; f < nfields; ++f) {
    if (!fields[f] || !std::isfinite(fp[f].n)) return BRAHMS_E_ARG;
    fs.f[f] = static_cast<const float2*>(fields[f]);
    w.w[f] = 0.5 * c0 * eps0 * fp[f].n * dx * dy * dt;
  }
  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return BRAHMS_E_CUDA;
  long long want = (n + kStaticThreads * 16 - 1) / (kStaticThreads * 16);
  const int nblocks = (int)(want < 1 ? 1 : (want > kStaticBlocks ? kStaticBlocks : want));
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // every partial read below is written by this call first
  energy_static_partial_kernel<<<dim3(nblocks, nfields), kStaticThreads, 0, s>>>(fs, n, scratch);
  energy_static_final_kernel<<<nfields, kStaticThreads, 0, s>>>(scratch, nblocks, w, energy_j_dev);
  return cudaPeekAtLastError() == cudaSuccess ? BRAHMS_OK : BRAHMS_E_CUDA;
}
