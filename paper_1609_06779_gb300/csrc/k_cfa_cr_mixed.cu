// CFA kernels with block cyclic reduction for T = float, TA = double.
#include "fd_kernels.cuh"
#include "fd_launch.h"

namespace fdk {

cudaError_t launch_cfa_cr_mixed(const KArgs &a, int team, cudaStream_t s) {
  const unsigned g = grid_for(a.n_problems, team);
  switch (team) {
    FDK_TEAM_CASES(cfa_cr_kernel, float, double)
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace fdk
