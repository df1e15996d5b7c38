// Inverse dynamics (Eq. 2a-2d) kernels: instantiations and launcher.
#include "fd_kernels.cuh"
#include "fd_launch.h"

namespace fdk {

template <class T>
static cudaError_t go(const KArgs &a, int team, cudaStream_t s) {
  const unsigned g = grid_for(a.n_problems, team);
  switch (team) {
    case 1: id_kernel<T, 1><<<g, BLOCK, 0, s>>>(a); break;
    case 2: id_kernel<T, 2><<<g, BLOCK, 0, s>>>(a); break;
    case 4: id_kernel<T, 4><<<g, BLOCK, 0, s>>>(a); break;
    case 8: id_kernel<T, 8><<<g, BLOCK, 0, s>>>(a); break;
    case 16: id_kernel<T, 16><<<g, BLOCK, 0, s>>>(a); break;
    case 32: id_kernel<T, 32><<<g, BLOCK, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_id(const KArgs &a, int prec, int team, cudaStream_t s) {
  return prec == 0 ? go<double>(a, team, s) : go<float>(a, team, s);
}

}  // namespace fdk
