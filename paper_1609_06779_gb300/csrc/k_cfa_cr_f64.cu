// CFA kernels with block cyclic reduction for T = double, TA = double.
#include "fd_kernels.cuh"
#include "fd_launch.h"

namespace fdk {

cudaError_t launch_cfa_cr_f64(const KArgs &a, int team, cudaStream_t s) {
  const unsigned g = grid_for(a.n_problems, team);
  switch (team) {
    FDK_TEAM_CASES(cfa_cr_kernel, double, double)
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace fdk
