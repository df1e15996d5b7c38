// cfa_hy kernels over length classes (one launch, a team per class) for
// T = float, TA = double, one right-hand side (one translation unit per precision
// and mode).
#include "fd_kernels.cuh"
#include "fd_launch.h"

namespace fdk {

cudaError_t launch_cfa_hy2_multi_mixed(const KArgs &a, const ClassTable &ct, cudaStream_t s);

cudaError_t launch_cfa_hy_multi_mixed(const KArgs &a, const ClassTable &ct, cudaStream_t s) {
  if (a.mode == MODE_FD2) return launch_cfa_hy2_multi_mixed(a, ct, s);
  const unsigned g = static_cast<unsigned>(ct.blk[ct.n]);
  if (g == 0) return cudaSuccess;
  cfa_multi_kernel<float, double, 2, false><<<g, BLOCK, 0, s>>>(a, ct);
  return cudaGetLastError();
}

}  // namespace fdk
