// ABIA kernels: instantiations and launcher.
#include "fd_kernels.cuh"
#include "fd_launch.h"

namespace fdk {

template <class T, class TA, bool TWO>
static cudaError_t launch_abia_t(const KArgs &a, int team, cudaStream_t s) {
  const unsigned g = grid_for(a.n_problems, team);
  switch (team) {
    case 1: abia_kernel<T, TA, TWO><<<g, BLOCK, 0, s>>>(a); break;
    case 8: abia_team_kernel<T, TA, 8, TWO><<<g, BLOCK, 0, s>>>(a); break;
    case 16: abia_team_kernel<T, TA, 16, TWO><<<g, BLOCK, 0, s>>>(a); break;
    case 32: abia_team_kernel<T, TA, 32, TWO><<<g, BLOCK, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class T, class TA>
static cudaError_t launch_abia_m(const KArgs &a, int team, cudaStream_t s) {
  return a.mode == MODE_FD2 ? launch_abia_t<T, TA, true>(a, team, s)
                            : launch_abia_t<T, TA, false>(a, team, s);
}

cudaError_t launch_abia(const KArgs &a, int prec, int team, cudaStream_t s) {
  if (prec == 0) return launch_abia_m<double, double>(a, team, s);
  if (prec == 1) return launch_abia_m<float, float>(a, team, s);
  return launch_abia_m<float, double>(a, team, s);
}

}  // namespace fdk
