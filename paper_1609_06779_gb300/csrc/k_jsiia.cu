// JSIIA kernels: instantiations and launcher.
#include "fd_kernels.cuh"
#include "fd_launch.h"

namespace fdk {

template <class T, class TA>
static cudaError_t go(const KArgs &a, int team, cudaStream_t s) {
  const unsigned g = grid_for(a.n_problems, team);
  switch (team) {
    case 1: jsiia_kernel<T, TA, 1><<<g, BLOCK, 0, s>>>(a); break;
    case 2: jsiia_kernel<T, TA, 2><<<g, BLOCK, 0, s>>>(a); break;
    case 4: jsiia_kernel<T, TA, 4><<<g, BLOCK, 0, s>>>(a); break;
    case 8: jsiia_kernel<T, TA, 8><<<g, BLOCK, 0, s>>>(a); break;
    case 16: jsiia_kernel<T, TA, 16><<<g, BLOCK, 0, s>>>(a); break;
    case 32: jsiia_kernel<T, TA, 32><<<g, BLOCK, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_jsiia(const KArgs &a, int prec, int team, cudaStream_t s) {
  if (prec == 0) return go<double, double>(a, team, s);
  if (prec == 1) return go<float, float>(a, team, s);
  return go<float, double>(a, team, s);
}

}  // namespace fdk
