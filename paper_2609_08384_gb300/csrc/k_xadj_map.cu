// The reverse x-pass under a transverse mismatch map (kernel in xadj.cuh); a
// translation unit of its own so that it compiles in parallel with the
// map-free instantiations of k_xadj.cu.
#include "xadj.cuh"

namespace brahms {

cudaError_t run_xpass_adjoint_map(int nx, int nf, const XAdjArgs& a, long long* ncta, cudaStream_t s) {
  switch (nx) {
#define BRAHMS_XAM_CASE(N) \
  case N:                  \
    return nf == 3 ? launch_adjoint<N, 3, true>(a, ncta, s) : launch_adjoint<N, 2, true>(a, ncta, s);
    BRAHMS_FOR_EACH_SIZE(BRAHMS_XAM_CASE)
#undef BRAHMS_XAM_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace brahms
