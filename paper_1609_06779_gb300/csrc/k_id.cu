// Inverse dynamics (Eq. 2a-2d) kernels: instantiations and launcher.
#include "fd_kernels.cuh"
#include "fd_launch.h"

namespace fdk {

template <class T>
static cudaError_t go(const KArgs &a, int team, cudaStream_t s) {
  const unsigned g = grid_for(a.n_problems, team);
  switch (team) {
    FDK_TEAM_CASES(id_kernel, T)
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_id(const KArgs &a, int prec, int team, cudaStream_t s) {
  return prec == 0 ? go<double>(a, team, s) : go<float>(a, team, s);
}

}  // namespace fdk
