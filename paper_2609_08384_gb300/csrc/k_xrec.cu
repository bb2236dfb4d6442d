// The recording forward x-pass of the adjoint's segment recomputation: the
// plain x-pass that also writes the real-space states entering its B and A
// half steps (the forward states the reverse x-pass linearises about).
// Under a transverse mismatch map the instantiations of k_xrec_map.cu run.
#include "xrec.cuh"

namespace brahms {

cudaError_t run_xpass_record(int nx, int nf, const XPassArgs& a, cudaStream_t s) {
  if (a.emap) return run_xpass_record_map(nx, nf, a, s);
  switch (nx) {
#define BRAHMS_XR_CASE(N) \
  case N:                 \
    return nf == 3 ? launch_record<N, 3, false>(a, s) : launch_record<N, 2, false>(a, s);
    BRAHMS_FOR_EACH_SIZE(BRAHMS_XR_CASE)
#undef BRAHMS_XR_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace brahms
