// fd_launch.h -- host-side launchers of the kernels (one translation unit each).
#pragma once

#include <cuda_runtime.h>

#include "fd_layout.h"

namespace fdk {

constexpr int BLOCK = 128;

// prec: 0 = double, 1 = float, 2 = float with double accumulation.
cudaError_t launch_id(const KArgs &a, int prec, int team, cudaStream_t s);
cudaError_t launch_cfa(const KArgs &a, int prec, int team, cudaStream_t s);
cudaError_t launch_jsiia(const KArgs &a, int prec, int team, cudaStream_t s);
cudaError_t launch_abia(const KArgs &a, int prec, cudaStream_t s);

inline unsigned grid_for(int n_problems, int team) {
  const long long threads = static_cast<long long>(n_problems) * team;
  return static_cast<unsigned>((threads + BLOCK - 1) / BLOCK);
}

}  // namespace fdk
