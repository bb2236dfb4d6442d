// tau-pass with TMA double buffering.
//
// Persistent CTAs walk the tau-tiles (16 neighbouring x columns x NT values
// of one (field, y)).  While a tile is transformed, multiplied and
// transformed back, thread 0 has already asked the Tensor Memory Accelerator
// for the next tile: cp.async.bulk.tensor copies it into the other shared
// buffer and completes an mbarrier transaction count.  The TMA box is the
// tile itself (16 complex = 128 bytes of x, one y, up to 256 tau; two boxes
// for NT = 512), written to shared memory tau-major with the 16 columns
// contiguous -- exactly the column-exchange layout of the FFT, so the tile is
// transformed in place.  Results are stored from registers with coalesced
// 128-byte rows.  Every mbarrier wait is bounded by %globaltimer (the limit
// is an argument, 2 s by default); on expiry the kernel records an error
// flag, waits for its copies in flight (bounded by 2 s, whatever the limit,
// so that no copy can land in shared memory after the CTA has left) and
// returns.
#include <cuda.h>

#include "kernels.cuh"
#include "launch_cfg.h"

namespace brahms {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long gtimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; false on timeout.  The first probe does not block
// (test_wait); a zero limit gives up right there if the phase is not complete,
// so that a test can make the wait run out (try_wait may itself suspend the
// thread until the copy lands, which would hide a short limit).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns) {
  if (mbar_test_wait(bar, parity)) return true;
  if (limit_ns == 0) return false;
  const unsigned long long t0 = gtimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (gtimer_ns() - t0 > limit_ns) return false;
  }
  return true;
}

constexpr unsigned long long kTmaDrainNs = 2000000000ULL;  // 2 s

}  // namespace

template <class PL>
__host__ __device__ constexpr int tma_box_t() { return PL::N < 256 ? PL::N : 256; }
template <class PL, int TX>
__host__ __device__ constexpr size_t tma_smem_bytes() {
  return 2 * (size_t)PL::N * TX * 8 + (tw_in_smem<PL>() ? (size_t)tw_table_size<PL>() * 16 : 0) + 16;
}

template <class PL, int TX>
__global__ void __launch_bounds__(PL::T * TX, PL::T * TX <= 256 ? 2 : 1)
    tpass_tma_kernel(const __grid_constant__ CUtensorMap tm, const AxisArgs p, int* err, unsigned long long wait_ns) {
  constexpr int N = PL::N, E = PL::E, T = PL::T;
  constexpr int BOX = tma_box_t<PL>();
  constexpr int NBOX = N / BOX;
  constexpr uint32_t TILE_BYTES = (uint32_t)(N * TX * 8);
  constexpr int R0 = fft_radix<PL, false>(0), RL = fft_radix<PL, false>(PL::NP - 1);
  constexpr int S0 = N / R0, SL = N / RL;
  extern __shared__ __align__(1024) unsigned char smraw[];
  float2* buf[2] = {reinterpret_cast<float2*>(smraw), reinterpret_cast<float2*>(smraw) + N * TX};
  float4* tws = reinterpret_cast<float4*>(buf[1] + N * TX);
  unsigned long long* bars =
      reinterpret_cast<unsigned long long*>(reinterpret_cast<unsigned char*>(tws) +
                                            (tw_in_smem<PL>() ? (size_t)tw_table_size<PL>() * 16 : 0));
  // TMA destinations must be 128-byte aligned
  if (smem_u32(smraw) & 127u) {
    if (threadIdx.x == 0) atomicExch(err, 2);
    return;
  }

  if constexpr (tw_in_smem<PL>())
    for (int i = threadIdx.x; i < tw_table_size<PL>(); i += blockDim.x) tws[i] = p.tw[i];
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars[0])), "r"(1) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bars[1])), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const long long ntiles = p.ntiles;
  // thread 0: start the copy of tile tl into buffer b
  auto issue = [&](long long tl, int b) {
    const int xt = (int)(tl % p.xtiles);
    const long long rest = tl / p.xtiles;
    const int y = (int)(rest % p.ny), f = (int)(rest / p.ny);
    const uint32_t bar = smem_u32(&bars[b]);
    // earlier generic-proxy accesses to this buffer precede the async-proxy writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(TILE_BYTES) : "memory");
#pragma unroll
    for (int q = 0; q < NBOX; ++q) {
      const uint32_t dst = smem_u32(buf[b] + (size_t)q * BOX * TX);
      asm volatile(
          "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
          "[%6];" ::"r"(dst),
          "l"(reinterpret_cast<uint64_t>(&tm)), "r"(2 * TX * xt), "r"(y), "r"(q * BOX), "r"(f), "r"(bar)
          : "memory");
    }
  };

  const int lt = threadIdx.x;
  const int tx = lt % TX, t = lt / TX;
  uint32_t phase[2] = {0u, 0u};
  long long tile = blockIdx.x;
  if (threadIdx.x == 0 && tile < ntiles) issue(tile, 0);
  int k = 0;
  for (; tile < ntiles; tile += gridDim.x, ++k) {
    const int b = k & 1;
    const long long next = tile + gridDim.x;
    const bool pending_next = next < ntiles;
    if (threadIdx.x == 0 && pending_next) issue(next, b ^ 1);
    const bool ok = mbar_wait(smem_u32(&bars[b]), phase[b], wait_ns);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicExch(err, 1);
        // let the copies in flight land (bounded) before the CTA exits
        mbar_wait(smem_u32(&bars[b]), phase[b], kTmaDrainNs);
        if (pending_next) mbar_wait(smem_u32(&bars[b ^ 1]), phase[b ^ 1], kTmaDrainNs);
      }
      break;
    }
    phase[b] ^= 1u;
    // coordinates of this tile
    const int xt = (int)(tile % p.xtiles);
    const long long rest = tile / p.xtiles;
    const int y = (int)(rest % p.ny), f = (int)(rest / p.ny);
    const int x = xt * TX + tx;
    const bool act = x < p.nx;
    const XchCol<TX> xc{buf[b], tx};
    float2 v[E];
#pragma unroll
    for (int bb = 0; bb < E / R0; ++bb)
#pragma unroll
      for (int r = 0; r < R0; ++r) v[bb * R0 + r] = xc.ld(t + bb * T + r * S0);
    using TWA = typename std::conditional<tw_in_smem<PL>(), TwShared, TwGlobal>::type;
    const TWA tw{tw_in_smem<PL>() ? tws : p.tw};
    fft_run<PL, false, 0, XchCol<TX>, SyncBlock, TWA>(v, t, xc, tw);
    float2 dxy = make_float2(0.f, 0.f);
    if (act) {
      const float2 dx = p.px[f * p.nx + x], dy = p.py[f * p.ny + y];
      dxy = cadd(cadd(dx, dy), cmul(dx, dy));
    }
    if (p.conj_p) dxy.y = -dxy.y;
    const float2* pt = p.pt + f * p.nt;
    const float tsign = p.conj_p ? -1.f : 1.f;
#pragma unroll
    for (int bb = 0; bb < E / RL; ++bb)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int kk = t + bb * T + r * SL;
        float2 dt = pt[kk];
        dt.y *= tsign;
        float2 w = v[bb * RL + r];
        w = make_float2(fmaf(w.x, p.scale, w.x * p.scale_lo), fmaf(w.y, p.scale, w.y * p.scale_lo));
        v[bb * RL + r] = mul_one_plus(w, cadd(cadd(dxy, dt), cmul(dxy, dt)));
      }
    fft_run<PL, true, 0, XchCol<TX>, SyncBlock, TWA>(v, t, xc, tw);
    if (act) {
      float2* base = p.data + (long long)f * p.fstride + (long long)y * p.nx + x;
      const long long stride = (long long)p.nx * p.ny;
#pragma unroll
      for (int bb = 0; bb < E / R0; ++bb)
#pragma unroll
        for (int r = 0; r < R0; ++r) base[(t + bb * T + r * S0) * stride] = v[bb * R0 + r];
    }
    __syncthreads();  // buffer b is free for the copy issued in the next iteration
  }
}

// ----------------------------------------------- prefetching tau-pass
// Persistent CTAs, two per SM, each with one 64 KB prefetch buffer: a tile
// is copied from the buffer into registers, the CTA synchronises, thread 0
// starts the copy of the CTA's next tile into the same buffer, and the tile
// is transformed, multiplied, transformed back and stored while that copy is
// in flight.  The FFT exchanges go through a separate half-size buffer, one
// real component at a time, so that two CTAs' buffers fit in an SM; the
// twiddles are read through L1.  Tiles are taken from the last down (as the
// plain tau-pass).  Waits are bounded as in the double-buffered kernel.
template <class PL>
__host__ __device__ constexpr size_t pre_smem_bytes() {
  return (size_t)PL::N * 16 * 8 + (size_t)PL::N * 16 * 4 + 16;
}

template <class PL>
__global__ void __launch_bounds__(PL::T * 16, 2)
    tpass_pre_kernel(const __grid_constant__ CUtensorMap tm, const AxisArgs p, int* err, unsigned long long wait_ns) {
  constexpr int TX = 16;
  constexpr int N = PL::N, E = PL::E, T = PL::T;
  constexpr int BOX = tma_box_t<PL>();
  constexpr int NBOX = N / BOX;
  constexpr uint32_t TILE_BYTES = (uint32_t)(N * TX * 8);
  constexpr int R0 = fft_radix<PL, false>(0), RL = fft_radix<PL, false>(PL::NP - 1);
  constexpr int S0 = N / R0, SL = N / RL;
  extern __shared__ __align__(1024) unsigned char smraw[];
  float2* pre = reinterpret_cast<float2*>(smraw);
  float* xre = reinterpret_cast<float*>(pre + N * TX);
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(xre + N * TX);
  if (smem_u32(smraw) & 127u) {
    if (threadIdx.x == 0) atomicExch(err, 2);
    return;
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const long long ntiles = p.ntiles;
  auto issue = [&](long long tl) {
    const int xt = (int)(tl % p.xtiles);
    const long long rest = tl / p.xtiles;
    const int y = (int)(rest % p.ny), f = (int)(rest / p.ny);
    const uint32_t b = smem_u32(bar);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(TILE_BYTES) : "memory");
#pragma unroll
    for (int q = 0; q < NBOX; ++q) {
      const uint32_t dst = smem_u32(pre + (size_t)q * BOX * TX);
      asm volatile(
          "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
          "[%6];" ::"r"(dst),
          "l"(reinterpret_cast<uint64_t>(&tm)), "r"(2 * TX * xt), "r"(y), "r"(q * BOX), "r"(f), "r"(b)
          : "memory");
    }
  };

  const int tx = threadIdx.x % TX, t = threadIdx.x / TX;
  const TwGlobal tw{p.tw};
  const XchColSplit<TX> xc{xre, tx};
  uint32_t phase = 0u;
  long long k = blockIdx.x;  // tile ntiles-1-k
  if (threadIdx.x == 0 && k < ntiles) issue(ntiles - 1 - k);
  for (; k < ntiles; k += gridDim.x) {
    const long long tile = ntiles - 1 - k;
    const bool ok = mbar_wait(smem_u32(bar), phase, wait_ns);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicExch(err, 1);
        mbar_wait(smem_u32(bar), phase, kTmaDrainNs);  // the copy in flight lands before the CTA leaves
      }
      return;
    }
    phase ^= 1u;
    float2 v[E];
#pragma unroll
    for (int bb = 0; bb < E / R0; ++bb)
#pragma unroll
      for (int r = 0; r < R0; ++r) v[bb * R0 + r] = pre[(t + bb * T + r * S0) * TX + tx];
    __syncthreads();  // the buffer is free: fetch the next tile while this one is transformed
    if (threadIdx.x == 0 && k + gridDim.x < ntiles) issue(ntiles - 1 - (k + gridDim.x));
    const int xt = (int)(tile % p.xtiles);
    const long long rest = tile / p.xtiles;
    const int y = (int)(rest % p.ny), f = (int)(rest / p.ny);
    const int x = xt * TX + tx;
    const bool act = x < p.nx;
    fft_run<PL, false, 0, XchColSplit<TX>, SyncBlock, TwGlobal>(v, t, xc, tw);
    float2 dxy = make_float2(0.f, 0.f);
    if (act) {
      const float2 dx = p.px[f * p.nx + x], dy = p.py[f * p.ny + y];
      dxy = cadd(cadd(dx, dy), cmul(dx, dy));
    }
    if (p.conj_p) dxy.y = -dxy.y;
    const float2* pt = p.pt + f * p.nt;
    const float tsign = p.conj_p ? -1.f : 1.f;
#pragma unroll
    for (int bb = 0; bb < E / RL; ++bb)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int kk = t + bb * T + r * SL;
        float2 dt = pt[kk];
        dt.y *= tsign;
        float2 w = v[bb * RL + r];
        w = make_float2(fmaf(w.x, p.scale, w.x * p.scale_lo), fmaf(w.y, p.scale, w.y * p.scale_lo));
        v[bb * RL + r] = mul_one_plus(w, cadd(cadd(dxy, dt), cmul(dxy, dt)));
      }
    fft_run<PL, true, 0, XchColSplit<TX>, SyncBlock, TwGlobal>(v, t, xc, tw);
    if (act) {
      float2* base = p.data + (long long)f * p.fstride + (long long)y * p.nx + x;
      const long long stride = (long long)p.nx * p.ny;
#pragma unroll
      for (int bb = 0; bb < E / R0; ++bb)
#pragma unroll
        for (int r = 0; r < R0; ++r) base[(t + bb * T + r * S0) * stride] = v[bb * R0 + r];
    }
  }
  // a CTA whose last wait succeeded has no copy in flight here
}

// ------------------------------------------------------------------- host
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

bool tma_tau_supported(int nx, int nt) { return (nt == 256 || nt == 512) && nx >= 16; }

// Tensor map of a [nf][nt][ny][nx] complex64 array seen as floats:
// dims (2 nx, ny, nt, nf), box (2 tx, 1, min(nt, 256), 1).
cudaError_t make_tau_tensor_map(void* map128, const float2* data, int nx, int ny, int nt, int nf, int tx) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || !tma_tau_supported(nx, nt)) return cudaErrorNotSupported;
  CUtensorMap* m = reinterpret_cast<CUtensorMap*>(map128);
  const cuuint64_t dims[4] = {(cuuint64_t)2 * nx, (cuuint64_t)ny, (cuuint64_t)nt, (cuuint64_t)nf};
  const cuuint64_t strides[3] = {(cuuint64_t)8 * nx, (cuuint64_t)8 * nx * ny, (cuuint64_t)8 * nx * ny * nt};
  const cuuint32_t box[4] = {(cuuint32_t)(2 * tx), 1, (cuuint32_t)(nt < 256 ? nt : 256), 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float2*>(data), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <class PL, int TX>
static cudaError_t launch_tma(const void* map128, const AxisArgs& a0, int* err, unsigned long long wait_ns,
                              cudaStream_t s) {
  const size_t smem = tma_smem_bytes<PL, TX>();
  static SmemOnce once;
  cudaError_t e = raise_smem_limit(tpass_tma_kernel<PL, TX>, smem, once);
  if (e != cudaSuccess) return e;
  // resident CTAs on the current device (asked at every launch: a few
  // microseconds against a launch of about half a millisecond)
  int dev = 0, per_sm = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tpass_tma_kernel<PL, TX>, PL::T * TX, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  AxisArgs a = a0;  // tiles of TX columns
  a.xtiles = (a.nx + TX - 1) / TX;
  a.ntiles = a0.ntiles / a0.xtiles * a.xtiles;
  long long grid = (long long)sms * per_sm;
  if (grid > a.ntiles) grid = a.ntiles;
  if (grid <= 0) return cudaSuccess;
  CUtensorMap m;
  memcpy(&m, map128, sizeof(m));
  tpass_tma_kernel<PL, TX><<<(unsigned)grid, PL::T * TX, smem, s>>>(m, a, err, wait_ns);
  return cudaPeekAtLastError();
}

template <class PL>
static cudaError_t launch_pre(const void* map128, const AxisArgs& a0, int* err, unsigned long long wait_ns,
                              cudaStream_t s) {
  AxisArgs a = a0;  // tiles of 16 columns
  a.xtiles = (a.nx + 15) / 16;
  a.ntiles = a0.ntiles / a0.xtiles * a.xtiles;
  constexpr size_t smem = pre_smem_bytes<PL>();
  static SmemOnce once;
  cudaError_t e = raise_smem_limit(tpass_pre_kernel<PL>, smem, once);
  if (e != cudaSuccess) return e;
  int dev = 0, per_sm = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tpass_pre_kernel<PL>, PL::T * 16, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  long long grid = (long long)sms * per_sm;
  if (grid > a.ntiles) grid = a.ntiles;
  if (grid <= 0) return cudaSuccess;
  CUtensorMap m;
  memcpy(&m, map128, sizeof(m));
  tpass_pre_kernel<PL><<<(unsigned)grid, PL::T * 16, smem, s>>>(m, a, err, wait_ns);
  return cudaPeekAtLastError();
}

cudaError_t run_tpass_prop_tma(int nt, int tx, const void* map128, const AxisArgs& a, int* err,
                               unsigned long long wait_ns, cudaStream_t s) {
  if (tx == 1) {  // prefetching form (16-column tiles)
    switch (nt) {
      case 256: return launch_pre<TauPlan<256>>(map128, a, err, wait_ns, s);
      case 512: return launch_pre<TauPlan<512>>(map128, a, err, wait_ns, s);
      default: return cudaErrorNotSupported;
    }
  }
  if (tx == 8) {
    switch (nt) {
      case 256: return launch_tma<TauPlan<256>, 8>(map128, a, err, wait_ns, s);
      case 512: return launch_tma<TauPlan<512>, 8>(map128, a, err, wait_ns, s);
      default: return cudaErrorNotSupported;
    }
  }
  switch (nt) {
    case 256: return launch_tma<TauPlan<256>, 16>(map128, a, err, wait_ns, s);
    case 512: return launch_tma<TauPlan<512>, 16>(map128, a, err, wait_ns, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace brahms
