// fd_launch.h -- host-side launchers of the kernels (one translation unit each).
#pragma once

#include <cuda_runtime.h>

#include "fd_layout.h"

namespace fdk {

constexpr int BLOCK = 128;

// prec: 0 = double, 1 = float, 2 = float with double accumulation.
cudaError_t launch_id(const KArgs &a, int prec, int team, cudaStream_t s);
cudaError_t launch_cfa(const KArgs &a, int prec, int team, cudaStream_t s);
cudaError_t launch_cfa_w(const KArgs &a, int prec, int team, cudaStream_t s);
cudaError_t launch_tree(const KArgs &a, int algo, int prec, cudaStream_t s);
cudaError_t launch_tree_loops(const KArgs &a, cudaStream_t s);
cudaError_t launch_cfa_cr(const KArgs &a, int prec, int team, cudaStream_t s);
cudaError_t launch_cfa_hy(const KArgs &a, int prec, int team, cudaStream_t s);
cudaError_t launch_jsiia(const KArgs &a, int prec, int team, cudaStream_t s);
// team 1: one thread per problem; 8, 16, 32: rows of the articulated inertia
// spread over six lanes of the team.
cudaError_t launch_abia(const KArgs &a, int prec, int team, cudaStream_t s);
inline bool abia_team_ok(int team) { return team == 1 || team == 8 || team == 16 || team == 32; }
cudaError_t launch_adjoint_rnea(const KArgs &a, int prec, int team, cudaStream_t s);
// ABIA with the articulated-inertia recursion as a scan: FP64 (prec 0), teams 8 .. 256.
cudaError_t launch_abia_scan(const KArgs &a, int prec, int team, cudaStream_t s);
inline bool abia_scan_team_ok(int team) { return team >= 8 && team <= 256; }

// One launch over the length classes of `ct` (teams of 1 .. 128 lanes, one per
// class; ABIA 1, 8, 16 or 32), grid ct.blk[ct.n] blocks of BLOCK threads.
cudaError_t launch_id_multi(const KArgs &a, int prec, const ClassTable &ct, cudaStream_t s);
cudaError_t launch_cfa_multi(const KArgs &a, int prec, const ClassTable &ct, cudaStream_t s);
cudaError_t launch_cfa_cr_multi(const KArgs &a, int prec, const ClassTable &ct, cudaStream_t s);
cudaError_t launch_cfa_hy_multi(const KArgs &a, int prec, const ClassTable &ct, cudaStream_t s);
cudaError_t launch_jsiia_multi(const KArgs &a, int prec, const ClassTable &ct, cudaStream_t s);
cudaError_t launch_abia_multi(const KArgs &a, int prec, const ClassTable &ct, cudaStream_t s);
cudaError_t launch_adjoint_rnea_multi(const KArgs &a, int prec, const ClassTable &ct,
                                      cudaStream_t s);

inline unsigned grid_for(int n_problems, int team) {
  const int block = team > BLOCK ? team : BLOCK;
  const long long threads = static_cast<long long>(n_problems) * team;
  return static_cast<unsigned>((threads + block - 1) / block);
}

// Team sizes the kernels are built for: one thread up to a 256-thread block.
#define FDK_TEAM_CASES(KERNEL, ...)                                               \
  case 1: KERNEL<__VA_ARGS__, 1><<<g, block_for<1>(), 0, s>>>(a); break;          \
  case 2: KERNEL<__VA_ARGS__, 2><<<g, block_for<2>(), 0, s>>>(a); break;          \
  case 4: KERNEL<__VA_ARGS__, 4><<<g, block_for<4>(), 0, s>>>(a); break;          \
  case 8: KERNEL<__VA_ARGS__, 8><<<g, block_for<8>(), 0, s>>>(a); break;          \
  case 16: KERNEL<__VA_ARGS__, 16><<<g, block_for<16>(), 0, s>>>(a); break;       \
  case 32: KERNEL<__VA_ARGS__, 32><<<g, block_for<32>(), 0, s>>>(a); break;       \
  case 64: KERNEL<__VA_ARGS__, 64><<<g, block_for<64>(), 0, s>>>(a); break;       \
  case 128: KERNEL<__VA_ARGS__, 128><<<g, block_for<128>(), 0, s>>>(a); break;    \
  case 256: KERNEL<__VA_ARGS__, 256><<<g, block_for<256>(), 0, s>>>(a); break;

}  // namespace fdk
