// ABIA with the articulated-inertia recursion as a parallel scan (FP64): launcher.
#include "fd_abia_scan.cuh"
#include "fd_launch.h"

namespace fdk {

template <int P, bool TWO>
static cudaError_t go2(const KArgs &a, cudaStream_t s) {
  const unsigned g = grid_for(a.n_problems, P);
  const size_t smem = static_cast<size_t>(block_for<P>()) * SCAN_SLOT * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(abia_scan_kernel<P, TWO>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  abia_scan_kernel<P, TWO><<<g, block_for<P>(), smem, s>>>(a);
  return cudaGetLastError();
}

template <int P>
static cudaError_t go(const KArgs &a, cudaStream_t s) {
  return a.mode == MODE_FD2 ? go2<P, true>(a, s) : go2<P, false>(a, s);
}

cudaError_t launch_abia_scan(const KArgs &a, int prec, int team, cudaStream_t s) {
  if (prec != 0) return cudaErrorInvalidValue;
  switch (team) {
    case 8: return go<8>(a, s);
    case 16: return go<16>(a, s);
    case 32: return go<32>(a, s);
    case 64: return go<64>(a, s);
    case 128: return go<128>(a, s);
    case 256: return go<256>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fdk
