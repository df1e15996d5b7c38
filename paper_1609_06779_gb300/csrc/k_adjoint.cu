// Reverse inverse dynamics kernels for the adjoint: instantiations and launcher.
#include "fd_adjoint.cuh"
#include "fd_launch.h"

namespace fdk {

template <class T>
static cudaError_t go(const KArgs &a, int team, cudaStream_t s) {
  const unsigned g = grid_for(a.n_problems, team);
  switch (team) {
    FDK_TEAM_CASES(adjoint_rnea_kernel, T)
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_adjoint_rnea(const KArgs &a, int prec, int team, cudaStream_t s) {
  return prec == 0 ? go<double>(a, team, s) : go<float>(a, team, s);
}

}  // namespace fdk
