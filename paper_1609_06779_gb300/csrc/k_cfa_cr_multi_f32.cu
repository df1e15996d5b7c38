// cfa_cr kernels over length classes (one launch, a team per class) for
// T = float, TA = float, one right-hand side (one translation unit per precision
// and mode).
#include "fd_kernels.cuh"
#include "fd_launch.h"

namespace fdk {

cudaError_t launch_cfa_cr2_multi_f32(const KArgs &a, const ClassTable &ct, cudaStream_t s);

cudaError_t launch_cfa_cr_multi_f32(const KArgs &a, const ClassTable &ct, cudaStream_t s) {
  if (a.mode == MODE_FD2) return launch_cfa_cr2_multi_f32(a, ct, s);
  const unsigned g = static_cast<unsigned>(ct.blk[ct.n]);
  if (g == 0) return cudaSuccess;
  cfa_multi_kernel<float, float, 1, false><<<g, BLOCK, 0, s>>>(a, ct);
  return cudaGetLastError();
}

}  // namespace fdk
