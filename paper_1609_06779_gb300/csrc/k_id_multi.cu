// Inverse dynamics and the adjoint's reverse sweep over length classes (one
// launch, a team per class).
#include "fd_adjoint.cuh"
#include "fd_launch.h"

namespace fdk {

cudaError_t launch_id_multi(const KArgs &a, int prec, const ClassTable &ct, cudaStream_t s) {
  const unsigned g = static_cast<unsigned>(ct.blk[ct.n]);
  if (g == 0) return cudaSuccess;
  if (prec == 0) id_multi_kernel<double><<<g, BLOCK, 0, s>>>(a, ct);
  else id_multi_kernel<float><<<g, BLOCK, 0, s>>>(a, ct);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_rnea_multi(const KArgs &a, int prec, const ClassTable &ct,
                                      cudaStream_t s) {
  const unsigned g = static_cast<unsigned>(ct.blk[ct.n]);
  if (g == 0) return cudaSuccess;
  if (prec == 0) adjoint_multi_kernel<double><<<g, BLOCK, 0, s>>>(a, ct);
  else adjoint_multi_kernel<float><<<g, BLOCK, 0, s>>>(a, ct);
  return cudaGetLastError();
}

}  // namespace fdk
