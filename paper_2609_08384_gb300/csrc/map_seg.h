// Stage phase factors of one x-pass under a map that changes along z, for
// passes that do not run in z order (the adjoint's recomputation and reverse
// sweep): the map's share of the phase at the start of step j is formed from
// the step counts of every segment before it,
//   Q_j(x, y) = sum_s c_s(j) m_s(x, y),  c_s(j) = dz * #{i < j : step i in segment s},
// instead of the running sum a forward propagation keeps.
#pragma once

#include <cuda_runtime.h>

namespace brahms {

constexpr int kMapSegMax = 16;  // segments the adjoint takes

struct MapSegArgs {
  const double* maps;  // [nseg][ny][nx]
  float2* emap;        // [4][ny][nx], as MapArgs
  long long nxy;
  int nseg;
  int sB, sA;                             // segments of the B step and of the A step
  double cB[kMapSegMax], cA[kMapSegMax];  // c_s of the B step and of the A step
  double phiB, dkB, phiA, dkA, dz;
};
cudaError_t run_map_tables_seg(const MapSegArgs& a, cudaStream_t s);

}  // namespace brahms
