// CFA by cyclic reduction (two right-hand sides) kernels for T = double, TA = double (one translation unit per precision).
#include "fd_kernels.cuh"
#include "fd_launch.h"

namespace fdk {

cudaError_t launch_cfa_cr2_f64(const KArgs &a, int team, cudaStream_t s) {
  const unsigned g = grid_for(a.n_problems, team);
  switch (team) {
    FDK_TEAM_CASES(cfa_cr2_kernel, double, double)
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace fdk
