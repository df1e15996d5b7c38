// CFA kernels: instantiations and launcher.
#include "fd_kernels.cuh"
#include "fd_launch.h"

namespace fdk {

template <class T, class TA>
static cudaError_t go(const KArgs &a, int team, cudaStream_t s) {
  const unsigned g = grid_for(a.n_problems, team);
  switch (team) {
    FDK_TEAM_CASES(cfa_kernel, T, TA)
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_cfa(const KArgs &a, int prec, int team, cudaStream_t s) {
  if (prec == 0) return go<double, double>(a, team, s);
  if (prec == 1) return go<float, float>(a, team, s);
  return go<float, double>(a, team, s);
}

}  // namespace fdk
