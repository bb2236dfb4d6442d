// The recording forward x-pass under a transverse mismatch map (per-point
// stage phases); a translation unit of its own so that it compiles in
// parallel with the map-free instantiations of k_xrec.cu.
#include "xrec.cuh"

namespace brahms {

cudaError_t run_xpass_record_map(int nx, int nf, const XPassArgs& a, cudaStream_t s) {
  switch (nx) {
#define BRAHMS_XRM_CASE(N) \
  case N:                  \
    return nf == 3 ? launch_record<N, 3, true>(a, s) : launch_record<N, 2, true>(a, s);
    BRAHMS_FOR_EACH_SIZE(BRAHMS_XRM_CASE)
#undef BRAHMS_XRM_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace brahms
