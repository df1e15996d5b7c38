// Kinematic-tree kernels (ABIA, JSIIA, inverse dynamics; one thread per tree) in
// FP64 and FP32.
#include "fd_tree.cuh"
#include "fd_launch.h"

namespace fdk {

// algo: 0 ABIA, 1 JSIIA, -1 inverse dynamics; prec: 0 FP64, 1 FP32
cudaError_t launch_tree(const KArgs &a, int algo, int prec, cudaStream_t s) {
  const unsigned g = static_cast<unsigned>((static_cast<int64_t>(a.n_problems) + 127) / 128);
  if (g == 0) return cudaSuccess;
  if (prec == 0) {
    if (algo == 0) tree_abia_kernel<double, double><<<g, 128, 0, s>>>(a);
    else if (algo == 1) tree_jsiia_kernel<double, double><<<g, 128, 0, s>>>(a);
    else tree_id_kernel<double><<<g, 128, 0, s>>>(a);
  } else if (prec == 1) {
    if (algo == 0) tree_abia_kernel<float, float><<<g, 128, 0, s>>>(a);
    else if (algo == 1) tree_jsiia_kernel<float, float><<<g, 128, 0, s>>>(a);
    else tree_id_kernel<float><<<g, 128, 0, s>>>(a);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// the loop-closure correction after the tree JSIIA (FP64)
cudaError_t launch_tree_loops(const KArgs &a, cudaStream_t s) {
  const unsigned g = static_cast<unsigned>((static_cast<int64_t>(a.n_problems) + 127) / 128);
  if (g == 0) return cudaSuccess;
  tree_loop_kernel<<<g, 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fdk
