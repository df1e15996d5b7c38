// CFA kernels with the hybrid partition / cyclic-reduction solve for T = double,
// TA = double, one right-hand side (one translation unit per precision and mode).
#include "fd_kernels.cuh"
#include "fd_launch.h"

namespace fdk {

cudaError_t launch_cfa_hy2_f64(const KArgs &a, int team, cudaStream_t s);

cudaError_t launch_cfa_hy_f64(const KArgs &a, int team, cudaStream_t s) {
  if (a.mode == MODE_FD2) return launch_cfa_hy2_f64(a, team, s);
  const unsigned g = grid_for(a.n_problems, team);
  switch (team) {
    FDK_TEAM_CASES(cfa_hy_kernel, double, double, false)
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace fdk
