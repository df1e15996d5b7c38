// cfa_hy kernels over length classes (one launch, a team per class) for
// T = double, TA = double, two right-hand sides (MODE_FD2).
#include "fd_kernels.cuh"
#include "fd_launch.h"

namespace fdk {

cudaError_t launch_cfa_hy2_multi_f64(const KArgs &a, const ClassTable &ct, cudaStream_t s) {
  const unsigned g = static_cast<unsigned>(ct.blk[ct.n]);
  if (g == 0) return cudaSuccess;
  cfa_multi_kernel<double, double, 2, true><<<g, BLOCK, 0, s>>>(a, ct);
  return cudaGetLastError();
}

}  // namespace fdk
