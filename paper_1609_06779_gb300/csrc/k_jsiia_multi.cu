// JSIIA kernels over length classes (one launch, a team per class).
#include "fd_kernels.cuh"
#include "fd_launch.h"

namespace fdk {

cudaError_t launch_jsiia_multi(const KArgs &a, int prec, const ClassTable &ct, cudaStream_t s) {
  const unsigned g = static_cast<unsigned>(ct.blk[ct.n]);
  if (g == 0) return cudaSuccess;
  if (prec == 0) jsiia_multi_kernel<double, double><<<g, BLOCK, 0, s>>>(a, ct);
  else if (prec == 1) jsiia_multi_kernel<float, float><<<g, BLOCK, 0, s>>>(a, ct);
  else jsiia_multi_kernel<float, double><<<g, BLOCK, 0, s>>>(a, ct);
  return cudaGetLastError();
}

}  // namespace fdk
