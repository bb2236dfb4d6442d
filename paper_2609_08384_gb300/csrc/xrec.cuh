// Launcher of the recording forward x-pass (the plain x-pass that also writes
// the real-space states entering its B and A half steps), shared by the
// map-free (k_xrec.cu) and mismatch-map (k_xrec_map.cu) instantiations.
#pragma once

#include "kernels.cuh"
#include "launch_cfg.h"

namespace brahms {

template <int NX, int F, bool MAP>
cudaError_t launch_record(const XPassArgs& a0, cudaStream_t s) {
  XPassArgs a = a0;
  fill_stage_factors(a);
  constexpr int ROWS = xpass_rows<NX>();
  constexpr int THREADS = xpass_threads<NX>();
  const size_t smem = (size_t)xpass_smem_floats2<NX>(F) * sizeof(float2);
  static SmemOnce once;
  cudaError_t e = raise_smem_limit(xpass_kernel<NX, F, MAP, true>, smem, once);
  if (e != cudaSuccess) return e;
  const long long grid = (a.rows + ROWS - 1) / ROWS;
  if (grid <= 0) return cudaSuccess;
  xpass_kernel<NX, F, MAP, true><<<(unsigned)grid, THREADS, smem, s>>>(a);
  return cudaPeekAtLastError();
}

}  // namespace brahms
