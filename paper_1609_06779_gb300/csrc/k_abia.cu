// ABIA kernels: instantiations and launcher.
#include "fd_kernels.cuh"
#include "fd_launch.h"

namespace fdk {

template <class T, class TA>
static cudaError_t launch_abia_t(const KArgs &a, int team, cudaStream_t s) {
  const unsigned g = grid_for(a.n_problems, team);
  switch (team) {
    case 1: abia_kernel<T, TA><<<g, BLOCK, 0, s>>>(a); break;
    case 8: abia_team_kernel<T, TA, 8><<<g, BLOCK, 0, s>>>(a); break;
    case 16: abia_team_kernel<T, TA, 16><<<g, BLOCK, 0, s>>>(a); break;
    case 32: abia_team_kernel<T, TA, 32><<<g, BLOCK, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_abia(const KArgs &a, int prec, int team, cudaStream_t s) {
  if (prec == 0) return launch_abia_t<double, double>(a, team, s);
  if (prec == 1) return launch_abia_t<float, float>(a, team, s);
  return launch_abia_t<float, double>(a, team, s);
}

}  // namespace fdk
