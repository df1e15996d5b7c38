// ABIA kernels over length classes (one launch, a team per class).
#include "fd_kernels.cuh"
#include "fd_launch.h"

namespace fdk {

template <class T, class TA>
static void go(const KArgs &a, const ClassTable &ct, unsigned g, cudaStream_t s) {
  if (a.mode == MODE_FD2) abia_multi_kernel<T, TA, true><<<g, BLOCK, 0, s>>>(a, ct);
  else abia_multi_kernel<T, TA, false><<<g, BLOCK, 0, s>>>(a, ct);
}

cudaError_t launch_abia_multi(const KArgs &a, int prec, const ClassTable &ct, cudaStream_t s) {
  const unsigned g = static_cast<unsigned>(ct.blk[ct.n]);
  if (g == 0) return cudaSuccess;
  if (prec == 0) go<double, double>(a, ct, g, s);
  else if (prec == 1) go<float, float>(a, ct, g, s);
  else go<float, double>(a, ct, g, s);
  return cudaGetLastError();
}

}  // namespace fdk
