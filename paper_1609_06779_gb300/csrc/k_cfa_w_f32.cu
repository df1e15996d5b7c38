// CFA with a general projection W_i = Wc_i Q_i, T = TA = float (one translation
// unit per precision).
#include "fd_kernels.cuh"
#include "fd_launch.h"

namespace fdk {

cudaError_t launch_cfa_w_f32(const KArgs &a, int team, cudaStream_t s) {
  const unsigned g = grid_for(a.n_problems, team);
  switch (team) {
    FDK_TEAM_CASES(cfa_w_kernel, float, float)
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace fdk
