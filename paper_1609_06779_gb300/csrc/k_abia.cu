// ABIA kernels: instantiations and launcher.
#include "fd_kernels.cuh"
#include "fd_launch.h"

namespace fdk {

cudaError_t launch_abia(const KArgs &a, int prec, cudaStream_t s) {
  const unsigned g = grid_for(a.n_problems, 1);
  if (prec == 0) abia_kernel<double, double><<<g, BLOCK, 0, s>>>(a);
  else if (prec == 1) abia_kernel<float, float><<<g, BLOCK, 0, s>>>(a);
  else abia_kernel<float, double><<<g, BLOCK, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fdk
